// Instantiations of the image convolution (k_conv.cuh) for half widths 18..19.
#include "k_conv.cuh"

namespace psfm {
namespace conv {

cudaError_t launch_range_18_19(int h, const ConvParams& P, cudaStream_t st) {
  switch (h) {
#define PSFM_CASE(n) \
  case n:            \
    return launch_hw<n>(P, st);
    PSFM_CASE(18) PSFM_CASE(19)
#undef PSFM_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace conv
}  // namespace psfm
