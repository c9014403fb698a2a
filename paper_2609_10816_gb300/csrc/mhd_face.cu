// mhd_face.cu -- face-sweep kernels of the single-box step (body in mhd_face.cuh).
#include <algorithm>

#include "mhd_face.cuh"

namespace mhd {

// blocks of 128 threads the compiler must fit per SM (register budget of the face sweep)
#ifndef MHD_FACE_MINB
#define MHD_FACE_MINB 1
#endif

template <int RC, int RS>
__global__ void __launch_bounds__(128, MHD_FACE_MINB) k_face(Dev D, int dir, int seg) {
  if (D.work) {
    for_each_segment(D.work + dir, sweep_threads(D, dir, seg), [&](long long t) {
      Line ln;
      int m0, m1;
      if (sweep_line_at(D, dir, seg, t, ln, m0, m1)) face_seg<RC, RS>(D, dir, ln, m0, m1);
    });
    return;
  }
  Line ln;
  int m0, m1;
  if (!sweep_line(D, dir, seg, ln, m0, m1)) return;
  face_seg<RC, RS>(D, dir, ln, m0, m1);
}

template <int RC, int RS>
static void launch_face_t(const Dev& d, int dir, int seg, cudaStream_t st) {
  const int bs = 128;
  if (d.work) {
    const long long res = resident_blocks((const void*)k_face<RC, RS>, bs);
    seg = fill_seg(d, dir, seg, res * bs);
    const long long blocks = std::min((sweep_threads(d, dir, seg) + bs - 1) / bs, res);
    cudaMemsetAsync(d.work + dir, 0, sizeof(unsigned long long), st);
    k_face<RC, RS><<<(unsigned)blocks, bs, 0, st>>>(d, dir, seg);
    return;
  }
  const long long threads = sweep_threads(d, dir, seg);
  k_face<RC, RS><<<(unsigned)((threads + bs - 1) / bs), bs, 0, st>>>(d, dir, seg);
}

template <int RC>
static void launch_face_r(const Dev& d, int dir, int rs, int seg, cudaStream_t st) {
  switch (rs) {
    case RS_HLL: launch_face_t<RC, RS_HLL>(d, dir, seg, st); break;
    case RS_HLLD: launch_face_t<RC, RS_HLLD>(d, dir, seg, st); break;
    default: launch_face_t<RC, RS_LLF>(d, dir, seg, st); break;
  }
}

void launch_face(const Dev& d, int dir, int recon, int rs, int seg, cudaStream_t st) {
  switch (recon) {
    case REC_PC: launch_face_r<REC_PC>(d, dir, rs, seg, st); break;
    case REC_PLM_MC: launch_face_r<REC_PLM_MC>(d, dir, rs, seg, st); break;
    case REC_PLM_MINMOD: launch_face_r<REC_PLM_MINMOD>(d, dir, rs, seg, st); break;
    case REC_PPM: launch_face_r<REC_PPM>(d, dir, rs, seg, st); break;
    default: launch_face_r<REC_PPM_EP>(d, dir, rs, seg, st); break;
  }
}

}  // namespace mhd
