// Instantiations of the image convolution (k_conv.cuh) for half widths 11..13.
#include "k_conv.cuh"

namespace psfm {
namespace conv {

cudaError_t launch_range_11_13(int h, const ConvParams& P, cudaStream_t st) {
  switch (h) {
#define PSFM_CASE(n) \
  case n:            \
    return launch_hw<n>(P, st);
    PSFM_CASE(11) PSFM_CASE(12) PSFM_CASE(13)
#undef PSFM_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace conv
}  // namespace psfm
