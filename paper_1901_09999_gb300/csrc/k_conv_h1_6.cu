// Instantiations of the image convolution (k_conv.cuh) for half widths 1..6.
#include "k_conv.cuh"

namespace psfm {
namespace conv {

cudaError_t launch_range_1_6(int h, const ConvParams& P, cudaStream_t st) {
  switch (h) {
#define PSFM_CASE(n) \
  case n:            \
    return launch_hw<n>(P, st);
    PSFM_CASE(1) PSFM_CASE(2) PSFM_CASE(3) PSFM_CASE(4) PSFM_CASE(5) PSFM_CASE(6)
#undef PSFM_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace conv
}  // namespace psfm
