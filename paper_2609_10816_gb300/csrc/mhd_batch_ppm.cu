// mhd_batch_ppm.cu -- the batched stage kernels for PPM reconstruction (a translation
// unit of their own, so that the reconstructions' kernels compile in parallel).
#include "mhd_batch.cuh"

namespace mhd {

template <>
StageKernel batch_kernel<REC_PPM>(int which, int rs, int emf) {
  return batch_kernel_impl<REC_PPM>(which, rs, emf);
}

}  // namespace mhd
