// Host-side checks of integer helpers that the kernels use (compiled and run
// by tests/test_host_helpers.py; no GPU needed):
//   wide_tile / wide_tile_count: the 128 x 256 tile order of the wide split
//     product visits every tile that reaches the diagonal exactly once;
//   fixed40: v rounded to the 2^-40 grid, within half a unit, and exact sums.
#include <cmath>
#include <cstdio>
#include <random>
#include <set>
#include <utility>

#include "sp2_common.cuh"
#include "sp2_tc.cuh"

static int check_wide_tiles() {
  int bad = 0;
  for (int T = 1; T <= 160; ++T) {
    const int T2 = (T + 1) / 2;
    int expect = 0;
    for (int I = 0; I < T; ++I) expect += T2 - I / 2;  // pairs P >= I / 2
    const int cnt = sp2::tc::wide_tile_count(T);
    if (cnt != expect) {
      std::printf("T=%d: count %d, expected %d\n", T, cnt, expect);
      ++bad;
    }
    std::set<std::pair<int, int>> seen;
    for (int t = 0; t < cnt; ++t) {
      int I, P;
      sp2::tc::wide_tile<8>(t, T, I, P);
      if (I < 0 || I >= T || P < 0 || P >= T2 || P < I / 2 || !seen.insert({I, P}).second) {
        std::printf("T=%d: tile %d -> (%d, %d) out of range or repeated\n", T, t, I, P);
        ++bad;
        break;
      }
    }
    if ((int)seen.size() != expect) ++bad;
    int I, P;
    sp2::tc::wide_tile<8>(cnt, T, I, P);
    if (I != -1) ++bad;  // past the end
  }
  return bad;
}

static int check_fixed40() {
  std::mt19937_64 g(7);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  int bad = 0;
  long long sum = 0;
  double exact = 0.0;
  for (int i = 0; i < 1000000; ++i) {
    const double mag = std::pow(2.0, -45.0 + 51.0 * std::fabs(U(g)));  // 2^-45 .. 2^6
    const float v = (float)(U(g) * mag);
    const long long q = sp2::fixed40(v);
    const double scaled = (double)v * 1099511627776.0;  // v 2^40, exact in FP64
    if (std::fabs((double)q - scaled) > 0.5) {
      if (bad < 5) std::printf("fixed40(%a) = %lld, v 2^40 = %.3f\n", v, q, scaled);
      ++bad;
    }
    if (i < 4096) {  // a sum of grid values is the integer sum (no rounding)
      sum += q;
      exact += (double)q;
    }
  }
  if ((double)sum != exact) ++bad;
  return bad;
}

int main() {
  const int a = check_wide_tiles(), b = check_fixed40();
  std::printf("wide_tile failures %d, fixed40 failures %d\n", a, b);
  return (a || b) ? 1 : 0;
}
