"""Counter-based SplitMix64 and the block sampler.

The method draws W_k i.i.d. uniformly from M fixed selectors (Sec. 1, the
definition of {W_k}); with row-block selectors, that is a block index drawn
uniformly with replacement.  Both the CUDA library and this oracle implement
the same counter-based generator from its published definition:

  SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014): state s_i = seed + (i+1)*GAMMA mod 2^64, output
  mix(s_i) with the "variant 13" finaliser constants.

A draw is addressed by (seed, stream, counter) -> output index
stream * 2^40 + counter, so each stream is a disjoint window of the sequence.
Bounded integers in [0, K) use Lemire's multiply-shift on the top 32 bits
(Lemire, "Fast random integer generation in an interval", TOMACS 2019), so the
decision is integer arithmetic on both sides.
"""
from __future__ import annotations

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
STREAM_SHIFT = 40

STREAM_BLOCKS = 2   # view-block index per step
STREAM_RAYS = 3     # ray ids of random-ray blocks
STREAM_CYCLIC = 7   # the per-epoch permutations of the random cyclic order


def mix64(z: int) -> int:
    z &= MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def splitmix64(seed: int, index: int) -> int:
    """The index-th (0-based) output of SplitMix64 seeded with `seed`."""
    return mix64((seed + (index + 1) * GAMMA) & MASK64)


def draw(seed: int, stream: int, counter: int) -> int:
    return splitmix64(seed, (stream << STREAM_SHIFT) + counter)


def bounded(u: int, K: int) -> int:
    """Integer in [0, K) from a 64-bit draw: ((u >> 32) * K) >> 32."""
    return ((u >> 32) * K) >> 32


def uniform01(u: int) -> float:
    """Double in [0, 1): (u >> 11) * 2^-53."""
    return (u >> 11) * (1.0 / 9007199254740992.0)


def view_block(seed: int, k: int, n_blocks: int) -> int:
    """Block index tau_k (k = 1, 2, ...) drawn uniformly with replacement."""
    return bounded(draw(seed, STREAM_BLOCKS, k - 1), n_blocks)


def random_rays(seed: int, k: int, ell: int, n_avail: int) -> list[int]:
    """ell ray ids for step k, each uniform in [0, n_avail), drawn independently."""
    base = (k - 1) * ell
    return [bounded(draw(seed, STREAM_RAYS, base + i), n_avail) for i in range(ell)]


def cyclic_permutation(seed: int, epoch: int, n_blocks: int) -> list[int]:
    """The order in which epoch `epoch` (0-based) visits the blocks under the
    random cyclic order (Sec. 4.3's walnut experiment): the Fisher-Yates
    shuffle (Durstenfeld's form) of 0..M-1, where swap i, for i = M-1 down to
    1, exchanges entries i and j = bounded(draw(seed, 7, epoch*M + M-1-i), i+1)."""
    perm = list(range(n_blocks))
    base = epoch * n_blocks
    for i in range(n_blocks - 1, 0, -1):
        j = bounded(draw(seed, STREAM_CYCLIC, base + (n_blocks - 1 - i)), i + 1)
        perm[i], perm[j] = perm[j], perm[i]
    return perm


_PERM_CACHE: dict = {}


def cyclic_block(seed: int, k: int, n_blocks: int) -> int:
    """Block index tau_k (k = 1, 2, ...) under the random cyclic order."""
    epoch, pos = divmod(k - 1, n_blocks)
    key = (seed, epoch, n_blocks)
    if key not in _PERM_CACHE:
        if len(_PERM_CACHE) > 256:
            _PERM_CACHE.clear()
        _PERM_CACHE[key] = cyclic_permutation(seed, epoch, n_blocks)
    return _PERM_CACHE[key][pos]


def distinct_rays(seed: int, k: int, ell: int, n_avail: int) -> list[int]:
    """ell distinct ray ids of [0, n_avail) for step k by Floyd's algorithm
    (Bentley and Floyd, "A sample of brilliance", CACM 1987): for i = 0..ell-1,
    j = n_avail - ell + i and t uniform in [0, j] (draw (k-1)*ell + i of the
    ray stream); t joins the sample unless it is already there, in which case
    j joins.  Returned in insertion order."""
    if ell > n_avail:
        raise ValueError("fewer rays than the block needs")
    base = (k - 1) * ell
    chosen: set[int] = set()
    out = []
    for i in range(ell):
        j = n_avail - ell + i
        t = bounded(draw(seed, STREAM_RAYS, base + i), j + 1)
        v = j if t in chosen else t
        chosen.add(v)
        out.append(v)
    return out
