// mhd_batch_plm_mc.cu -- the batched stage kernels for PLM with the monotonised-central limiter reconstruction (a translation
// unit of their own, so that the reconstructions' kernels compile in parallel).
#include "mhd_batch.cuh"

namespace mhd {

template <>
StageKernel batch_kernel<REC_PLM_MC>(int which, int rs, int emf) {
  return batch_kernel_impl<REC_PLM_MC>(which, rs, emf);
}

}  // namespace mhd
