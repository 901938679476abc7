// Host check of the population offset widths of the FP32 sweep
// (fp32::pop_idx_kind and PopIdx in fp32_device.cuh): no GPU is used.  For
// node counts on either side of each bound it prints the width chosen and
// whether the largest component offset, 18 N + N - 1, is exact in the
// offset type (computed the way the kernels compute it); the Python test
// parses the lines.
#include <cstdio>

#include "../../paper_1907_04732_gb300/csrc/fp32_device.cuh"

template <int W>
static bool last_offset_exact(long long N) {
  using T = lbe::fp32::PopIdx<W>;
  const T v = (T)18 * (T)N + (T)(N - 1);
  return (long double)v == (long double)(19LL * N - 1);
}

int main() {
  const long long cases[] = {1,          1048576,     113025455,   113025456,  115343360,
                             226050910,  226050911,   226050912,   2147483647};
  for (long long N : cases) {
    const int k = lbe::fp32::pop_idx_kind(N);
    const bool exact = k == 0 ? last_offset_exact<0>(N) : (k == 1 ? last_offset_exact<1>(N) : last_offset_exact<2>(N));
    std::printf("N=%lld kind=%d exact=%d\n", N, k, exact ? 1 : 0);
  }
  return 0;
}
