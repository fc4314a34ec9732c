// Instantiations of the persistent tensor-core scan in its penalty form:
// the block selection and the attribute filter of Alg. 2 are folded into the
// MMA (a one-hot code chunk per row against a -P chunk per probe), so the
// epilogue only compares scores (see scan_tc_kernel.cuh).
#include "scan_tc_kernel.cuh"

namespace caps {

int tc_launch_pen(const CUtensorMap& map, const TcArgs& a, int metric, int words_pad, int kp,
                  int64_t grid, size_t smem, cudaStream_t s, int N) {
#define CAPS_PEN(WPV, KPV)                                                                     \
  if (N == 64)                                                                                 \
    return metric == CAPS_L2 ? launch_tc<CAPS_L2, WPV, KPV, 64, true>(map, a, grid, smem, s)   \
                             : launch_tc<CAPS_IP, WPV, KPV, 64, true>(map, a, grid, smem, s);  \
  return metric == CAPS_L2 ? launch_tc<CAPS_L2, WPV, KPV, 128, true>(map, a, grid, smem, s)   \
                           : launch_tc<CAPS_IP, WPV, KPV, 128, true>(map, a, grid, smem, s)
  if (kp == 10) {
    switch (words_pad) {
      case 1: CAPS_PEN(1, 10);
      case 2: CAPS_PEN(2, 10);
      case 4: CAPS_PEN(4, 10);
    }
  } else if (kp == 16) {
    switch (words_pad) {
      case 1: CAPS_PEN(1, 16);
      case 2: CAPS_PEN(2, 16);
      case 4: CAPS_PEN(4, 16);
    }
  }
#undef CAPS_PEN
  return fail(CAPS_EINVAL, "unsupported attribute word count or list length (penalty form)");
}

}  // namespace caps
