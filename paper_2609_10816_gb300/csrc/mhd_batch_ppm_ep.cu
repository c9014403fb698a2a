// mhd_batch_ppm_ep.cu -- the batched stage kernels for PPM-EP reconstruction (a translation
// unit of their own, so that the reconstructions' kernels compile in parallel).
#include "mhd_batch.cuh"

namespace mhd {

template <>
StageKernel batch_kernel<REC_PPM_EP>(int which, int rs, int emf) {
  return batch_kernel_impl<REC_PPM_EP>(which, rs, emf);
}

}  // namespace mhd
