// Runs the factorisation's task list in claim order on the host with the
// tile-counter protocol of the kernel: at its turn every task's waits must
// already hold (so CTAs claiming tasks in order always make progress), every
// tile must receive each update k < its column exactly once, and every tile
// of the lower triangle must end final (counter = column + 1).
// Exit status 0 when every T in [1, 40] passes, grouped and not.
#include <cstdio>
#include <map>
#include <set>
#include <utility>
#include <vector>

#include "slim_chol_tasks.h"

using slim::CholTask;

namespace {

struct Run {
  int T;
  std::map<std::pair<int, int>, int> cnt;
  std::map<std::pair<int, int>, std::set<int>> applied;
  int c(int a, int b) { auto it = cnt.find({a, b}); return it == cnt.end() ? 0 : it->second; }
  bool apply(int a, int b, int k) {
    if (!applied[{a, b}].insert(k).second) return false;   // an update applied twice
    cnt[{a, b}] = c(a, b) + 1;
    return true;
  }
};

bool check(int T, bool grouped) {
  Run s{T, {}, {}};
  std::vector<CholTask> list = slim::build_chol_tasks(T, grouped);
#ifdef PLANT_EARLY_UPDATE
  // planted mistake: the first grouped update moved ahead of the panel it needs
  for (size_t a = 1; a < list.size(); ++a)
    if (list[a].type == slim::kUpd4) {
      std::swap(list[a], list[1]);
      break;
    }
#endif
  for (const CholTask& t : list) {
    const int i = t.i, m = t.m, k = t.k;
    switch (t.type) {
      case slim::kPotrf:
        if (s.c(k, k) < k) return false;
        s.cnt[{k, k}] = s.c(k, k) + 1;
        break;
      case slim::kTrsm:
        if (s.c(m, m) < m + 1 || s.c(i, m) < m) return false;
        s.cnt[{i, m}] = s.c(i, m) + 1;
        break;
      case slim::kUpd:
        if (i < m || s.c(i, k) < k + 1 || s.c(m, k) < k + 1 || s.c(i, m) < k) return false;
        if (!s.apply(i, m, k)) return false;
        break;
      case slim::kUpd4:
        for (int r : {i, i + 1, m, m + 1})
          if (s.c(r, k) < k + 1) return false;
        for (int a = i; a <= i + 1; ++a)
          for (int b = m; b <= m + 1; ++b) {
            if (a < b || s.c(a, b) < k) return false;   // the kernel writes lower tiles only
            if (!s.apply(a, b, k)) return false;
          }
        break;
      case slim::kPanel:
        if (s.c(k, k) < k + 1 || s.c(i, k) < k || s.c(i, i) < k) return false;
        s.cnt[{i, k}] = s.c(i, k) + 1;
        if (!s.applied[{i, i}].insert(k).second) return false;
        s.cnt[{i, i}] = s.c(i, i) + 2;
        break;
      default:
        return false;
    }
  }
  for (int a = 0; a < T; ++a)
    for (int b = 0; b <= a; ++b) {
      if (s.c(a, b) != b + 1) return false;
      if ((int)s.applied[{a, b}].size() != b) return false;
    }
  return true;
}

}  // namespace

int main() {
  int bad = 0;
  for (int T = 1; T <= 40; ++T)
    for (bool g : {false, true})
      if (!check(T, g)) {
        std::printf("task list fails: T=%d grouped=%d\n", T, (int)g);
        ++bad;
      }
  std::printf("%s\n", bad ? "FAIL" : "ok");
  return bad ? 1 : 0;
}
