// Host build of the index walks of the ghost fill (csrc/mpw_index.cuh) with
// plain C++ stand-ins for the CUDA qualifiers.  Prints the number of
// mismatches of the strided block walk against the quotient/remainder
// decomposition, and of the hollow-box enumeration (32- and 64-bit forms)
// against each other and against an exact single cover of the shell.
#include <algorithm>
#include <cstdio>
#include <vector>

using std::max;
#define __device__
#define __forceinline__ inline
#include "../../paper_2002_00088_gb300/csrc/mpw_index.cuh"

template <int STRIDE>
static long walk_mismatches(long& checked) {
  long bad = 0;
  for (int d0 = 1; d0 <= 70; ++d0)
    for (int d1 = 1; d1 <= 40; d1 += (d1 < 12 ? 1 : 3))
      for (int d2 = 1; d2 <= 34; d2 += (d2 < 8 ? 1 : 5)) {
        const int n = d0 * d1 * d2;
        for (int tid = 0; tid < STRIDE; tid += 5) {
          mpw::BlockWalk<STRIDE> w(tid, d0, d1, d2);
          for (int e = tid; e < 2 * n; e += STRIDE, w.next()) {
            const int f = e >= n, r = e - f * n;
            if (w.f != f || w.o0 != r % d0 || w.o1 != (r / d0) % d1 || w.o2 != r / (d0 * d1)) ++bad;
            ++checked;
          }
        }
      }
  return bad;
}

int main() {
  long checked = 0;
  const long walk_bad = walk_mismatches<256>(checked) + walk_mismatches<128>(checked);
  std::printf("walk_checked %ld\nwalk_mismatches %ld\n", checked, walk_bad);
  long shell_bad = 0, points = 0;
  const int dims[][3] = {{262, 262, 262}, {134, 134, 134}, {6, 7, 8}, {5, 5, 5}, {7, 6, 5},
                         {40, 9, 12},     {3, 3, 3},       {70, 70, 70}, {1030, 1030, 7}};
  for (const auto& d : dims) {
    const int O[3] = {d[0], d[1], d[2]}, th = 3;
    const int Ix = max(O[0] - 2 * th, 0), Iy = max(O[1] - 2 * th, 0), Iz = max(O[2] - 2 * th, 0);
    const long long total = (long long)O[0] * O[1] * O[2] - (long long)Ix * Iy * Iz;
    std::vector<char> seen((size_t)O[0] * O[1] * O[2], 0);
    for (long long idx = 0; idx < total; ++idx) {
      int x, y, z, x2, y2, z2;
      mpw::shell_point_t<long long>(idx, O, th, x, y, z);
      mpw::shell_point_t<unsigned>((unsigned)idx, O, th, x2, y2, z2);
      if (x != x2 || y != y2 || z != z2) ++shell_bad;
      const bool inner = x >= th && x < O[0] - th && y >= th && y < O[1] - th && z >= th && z < O[2] - th;
      if (x < 0 || y < 0 || z < 0 || x >= O[0] || y >= O[1] || z >= O[2] || inner) {
        ++shell_bad;
        continue;
      }
      char& s = seen[((size_t)z * O[1] + y) * O[0] + x];
      if (s) ++shell_bad;
      s = 1;
      ++points;
    }
    for (int z = 0; z < O[2]; ++z)  // every shell point visited
      for (int y = 0; y < O[1]; ++y)
        for (int x = 0; x < O[0]; ++x) {
          const bool inner = x >= th && x < O[0] - th && y >= th && y < O[1] - th && z >= th && z < O[2] - th;
          if (!inner && !seen[((size_t)z * O[1] + y) * O[0] + x]) ++shell_bad;
        }
  }
  std::printf("shell_points %ld\nshell_mismatches %ld\n", points, shell_bad);
  return 0;
}
