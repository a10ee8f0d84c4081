"""Pins for the oracle's counter-based generator and block sampler (Sec. 1: W_k i.i.d. uniform)."""
import os

import numpy as np

from oracle import rng

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.txt")


def _golden():
    outs, buckets = [], None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = line.split()
        if f[0] == "buckets":
            buckets = (int(f[1]), int(f[2]), [int(v) for v in f[3:]])
        else:
            outs.append((int(f[0]), int(f[1]), int(f[2])))
    return outs, buckets


def test_splitmix64_reference_outputs():
    outs, _ = _golden()
    assert outs
    for seed, i, want in outs:
        assert rng.splitmix64(seed, i) == want


def test_splitmix64_reference_buckets():
    _, (seed, count, want) = _golden()
    got = [0] * 5
    for i in range(count):
        got[int(rng.uniform01(rng.splitmix64(seed, i)) * 5)] += 1
    assert got == want


def test_streams_are_windows_of_one_sequence():
    seed = 99
    assert rng.draw(seed, 0, 7) == rng.splitmix64(seed, 7)
    assert rng.draw(seed, 2, 5) == rng.splitmix64(seed, (2 << 40) + 5)


def test_bounded_is_top_bits_for_powers_of_two():
    for i in range(200):
        u = rng.splitmix64(7, i)
        for j in (1, 5, 16, 31):
            assert rng.bounded(u, 1 << j) == u >> (64 - j)


def test_bounded_range_and_uniformity():
    K = 7
    counts = np.zeros(K, dtype=np.int64)
    for i in range(70000):
        v = rng.bounded(rng.splitmix64(11, i), K)
        assert 0 <= v < K
        counts[v] += 1
    expected = 70000 / K
    chi2 = float(((counts - expected) ** 2 / expected).sum())
    assert chi2 < 22.5  # 6 dof, p ~ 0.001


def test_view_blocks_uniform_with_replacement():
    M, draws = 60, 30000
    seq = [rng.view_block(1, k, M) for k in range(1, draws + 1)]
    counts = np.bincount(seq, minlength=M)
    expected = draws / M
    chi2 = float(((counts - expected) ** 2 / expected).sum())
    assert chi2 < 104.0  # 59 dof, p ~ 0.0002
    # with replacement: repeats among the first M draws are expected
    assert len(set(seq[:M])) < M


def test_random_rays_in_range_and_distinct_streams():
    rays = rng.random_rays(5, 3, 64, 1000)
    assert len(rays) == 64 and all(0 <= v < 1000 for v in rays)
    assert rays != rng.random_rays(5, 4, 64, 1000)
    assert rays == [rng.bounded(rng.draw(5, rng.STREAM_RAYS, 2 * 64 + i), 1000) for i in range(64)]


# ------------------------------------------------------------ sampling without replacement
def test_cyclic_order_visits_every_block_once_per_epoch():
    for V, seed in ((1, 3), (2, 4), (7, 5), (60, 1), (180, 2)):
        for epoch in range(4):
            seen = [rng.cyclic_block(seed, epoch * V + i, V) for i in range(1, V + 1)]
            assert sorted(seen) == list(range(V)), (V, seed, epoch)


def test_cyclic_epochs_differ():
    V = 60
    perms = {tuple(rng.cyclic_permutation(9, e, V)) for e in range(20)}
    assert len(perms) == 20


def test_cyclic_permutation_is_uniform():
    # Fisher-Yates draws each of the M! orders with probability 1/M!; a swap
    # index drawn from [0, i) instead of [0, i] (Sattolo's cycles) reaches only
    # (M-1)! of them, and any bias in the swaps shows in the counts
    import itertools
    V, E = 4, 24000
    counts = dict.fromkeys(itertools.permutations(range(V)), 0)
    for e in range(E):
        counts[tuple(rng.cyclic_permutation(21, e, V))] += 1
    exp = E / len(counts)
    chi2 = sum((c - exp) ** 2 / exp for c in counts.values())
    assert min(counts.values()) > 0
    assert chi2 < 60.0, chi2          # 23 degrees of freedom: p < 1e-4 above 55


def test_floyd_rays_are_distinct_and_in_range():
    for n, ell, seed in ((5, 4, 1), (10, 10, 2), (1000, 37, 3), (65340, 363, 4)):
        for k in range(1, 40):
            ids = rng.distinct_rays(seed, k, ell, n)
            assert len(ids) == ell and len(set(ids)) == ell
            assert all(0 <= v < n for v in ids)
    assert sorted(rng.distinct_rays(5, 3, 10, 10)) == list(range(10))


def test_floyd_sample_is_uniform_over_subsets():
    # Floyd's algorithm gives every ell-subset of the n ids probability 1 / C(n, ell)
    import itertools
    n, ell, K = 6, 3, 20000
    counts = {frozenset(c): 0 for c in itertools.combinations(range(n), ell)}
    for k in range(1, K + 1):
        counts[frozenset(rng.distinct_rays(17, k, ell, n))] += 1
    exp = K / len(counts)
    chi2 = sum((c - exp) ** 2 / exp for c in counts.values())
    assert chi2 < 50.0, chi2          # 19 degrees of freedom: p < 1e-4 above 47


def test_floyd_rejects_blocks_larger_than_the_rays():
    import pytest
    with pytest.raises(ValueError):
        rng.distinct_rays(1, 1, 11, 10)
