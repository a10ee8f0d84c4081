// Task list of the tiled Cholesky factorisation (host code, no CUDA): the
// order in which the persistent factorisation's CTAs claim tasks.  Kept in a
// header of its own so that a host test can run the list's counter protocol.
#pragma once
#include <cstdint>
#include <vector>

namespace slim {

// One task of the right-looking tiled factorisation.
//   kPotrf (k):      factor diagonal tile (k,k) and form its inverse
//   kTrsm  (i,k):    L_ik = A_ik L_kk^{-T}
//   kUpd   (i,m,k):  A_im -= L_ik L_mk^T   (update from panel k)
//   kPanel (k+1,k):  the critical path of one panel in one task:
//                    TRSM(k+1,k), then A_{k+1,k+1} -= L_{k+1,k} L_{k+1,k}^T,
//                    then POTRF(k+1)
//   kUpd4  (i,m,k):  kUpd of the four tiles (i..i+1, m..m+1) at once
// Tile counter (i,m) counts the updates applied to tile (i,m), plus one when
// the tile is final: kUpd(i,m,k) waits for tiles (i,k), (m,k) final and
// (i,m) at k; kTrsm(i,m) for (m,m) final and (i,m) at m; kPanel(k+1,k) for
// (k,k) final, (k+1,k) and (k+1,k+1) at k, and adds 1 to (k+1,k) and 2 to
// (k+1,k+1).
struct CholTask {
  uint16_t type, i, m, k;
};
enum : uint16_t { kPotrf = 0, kTrsm = 1, kUpd = 2, kPanel = 3, kUpd4 = 4 };

// Task list in a dependency-compatible order: every task depends only on
// tasks earlier in the list, so CTAs that claim tasks through an atomic
// ticket always make progress.  With `grouped`, the trailing updates of a
// step come as 2x2 groups of tiles (kUpd4, top-left tile (i, m)) where the
// tiles are below the diagonal or on it.
inline std::vector<CholTask> build_chol_tasks(int T, bool grouped) {
  // Right-looking order with a lookahead of one panel.  The critical path of
  // panel k+1 (TRSM of tile (k+1,k), its update of the diagonal tile, and the
  // diagonal factorisation) is one task placed right after panel k's, ahead of
  // panel k's remaining trailing updates.
  std::vector<CholTask> t;
  t.push_back({kPotrf, 0, 0, 0});
  for (int i = 2; i < T; ++i) t.push_back({kTrsm, (uint16_t)i, 0, 0});
  for (int k = 0; k + 1 < T; ++k) {
    const int n1 = k + 1;
    t.push_back({kPanel, (uint16_t)n1, (uint16_t)n1, (uint16_t)k});
    for (int i = n1 + 1; i < T; ++i) t.push_back({kUpd, (uint16_t)i, (uint16_t)n1, (uint16_t)k});
    for (int i = n1 + 2; i < T; ++i) t.push_back({kTrsm, (uint16_t)i, (uint16_t)n1, (uint16_t)n1});
    if (!grouped) {
      for (int m = k + 2; m < T; ++m)
        for (int i = m; i < T; ++i) t.push_back({kUpd, (uint16_t)i, (uint16_t)m, (uint16_t)k});
      continue;
    }
    // columns m, m+1 together: the diagonal tile (m, m) alone, then 2x2
    // groups of rows i, i+1 (i >= m+1, so (m+1, m+1) is a group's diagonal
    // tile), a last odd row as two tiles; a last odd column tile by tile
    for (int m = k + 2; m < T; m += 2) {
      if (m + 1 >= T) {
        for (int i = m; i < T; ++i) t.push_back({kUpd, (uint16_t)i, (uint16_t)m, (uint16_t)k});
        continue;
      }
      t.push_back({kUpd, (uint16_t)m, (uint16_t)m, (uint16_t)k});
      int i = m + 1;
      for (; i + 1 < T; i += 2) t.push_back({kUpd4, (uint16_t)i, (uint16_t)m, (uint16_t)k});
      if (i < T) {
        t.push_back({kUpd, (uint16_t)i, (uint16_t)m, (uint16_t)k});
        t.push_back({kUpd, (uint16_t)i, (uint16_t)(m + 1), (uint16_t)k});
      }
    }
  }
  return t;
}

}  // namespace slim
