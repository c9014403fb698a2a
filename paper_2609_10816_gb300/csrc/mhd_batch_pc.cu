// mhd_batch_pc.cu -- the batched stage kernels for piecewise-constant reconstruction (a translation
// unit of their own, so that the reconstructions' kernels compile in parallel).
#include "mhd_batch.cuh"

namespace mhd {

template <>
StageKernel batch_kernel<REC_PC>(int which, int rs, int emf) {
  return batch_kernel_impl<REC_PC>(which, rs, emf);
}

}  // namespace mhd
