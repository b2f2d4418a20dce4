// Instantiations of the image convolution (k_conv.cuh) for half widths 7..10.
#include "k_conv.cuh"

namespace psfm {
namespace conv {

cudaError_t launch_range_7_10(int h, const ConvParams& P, cudaStream_t st) {
  switch (h) {
#define PSFM_CASE(n) \
  case n:            \
    return launch_hw<n>(P, st);
    PSFM_CASE(7) PSFM_CASE(8) PSFM_CASE(9) PSFM_CASE(10)
#undef PSFM_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace conv
}  // namespace psfm
