// Instantiations of the persistent tensor-core scan on e4m3 rows (form 1,
// per-row and per-query scales, fp32 accumulation): the block selection and
// the attribute filter are tested per (probe, row) in the epilogue, which
// multiplies each passing pair's dot product by the two scales (see
// scan_tc_kernel.cuh).
#include "scan_tc_kernel.cuh"

namespace caps {

int tc_launch_f8(const CUtensorMap& map, const TcArgs& a, int metric, int words_pad, int kp, int N,
                 int64_t grid, size_t smem, cudaStream_t s) {
#define CAPS_F8(WPV, KPV)                                                                       \
  if (N == 128)                                                                                 \
    return metric == CAPS_L2                                                                    \
               ? launch_tc<CAPS_L2, WPV, KPV, 128, false, true>(map, a, grid, smem, s)         \
               : launch_tc<CAPS_IP, WPV, KPV, 128, false, true>(map, a, grid, smem, s);        \
  return metric == CAPS_L2 ? launch_tc<CAPS_L2, WPV, KPV, 256, false, true>(map, a, grid, smem, s) \
                           : launch_tc<CAPS_IP, WPV, KPV, 256, false, true>(map, a, grid, smem, s)
  if (kp == 10) {
    switch (words_pad) {
      case 1: CAPS_F8(1, 10);
      case 2: CAPS_F8(2, 10);
      case 4: CAPS_F8(4, 10);
    }
  } else if (kp == 16) {
    switch (words_pad) {
      case 1: CAPS_F8(1, 16);
      case 2: CAPS_F8(2, 16);
      case 4: CAPS_F8(4, 16);
    }
  } else if (kp == 32) {
    switch (words_pad) {
      case 1: CAPS_F8(1, 32);
      case 2: CAPS_F8(2, 32);
      case 4: CAPS_F8(4, 32);
    }
  }
#undef CAPS_F8
  return fail(CAPS_EINVAL, "unsupported attribute word count or list length (e4m3 form)");
}

}  // namespace caps
