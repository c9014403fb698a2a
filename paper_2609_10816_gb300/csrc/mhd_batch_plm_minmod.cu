// mhd_batch_plm_minmod.cu -- the batched stage kernels for PLM with the minmod limiter reconstruction (a translation
// unit of their own, so that the reconstructions' kernels compile in parallel).
#include "mhd_batch.cuh"

namespace mhd {

template <>
StageKernel batch_kernel<REC_PLM_MINMOD>(int which, int rs, int emf) {
  return batch_kernel_impl<REC_PLM_MINMOD>(which, rs, emf);
}

}  // namespace mhd
