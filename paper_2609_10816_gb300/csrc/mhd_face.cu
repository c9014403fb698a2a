// mhd_face.cu -- face-sweep kernels of the single-box step (body in mhd_face.cuh).
#include <algorithm>

#include "mhd_face.cuh"

namespace mhd {

// blocks of 128 threads the compiler must fit per SM (register budget of the face sweep)
#ifndef MHD_FACE_MINB
#define MHD_FACE_MINB 1
#endif

// one direction, one thread per segment (the form without work cursors: mhd_step_noalloc)
template <int RC, int RS>
__global__ void __launch_bounds__(128, MHD_FACE_MINB) k_face(Dev D, int dir, int seg) {
  Line ln;
  int m0, m1;
  if (!sweep_line(D, dir, seg, ln, m0, m1)) return;
  face_seg<RC, RS>(D, dir, ln, m0, m1);
}

// The three face sweeps of a stage as one persistent launch: the segments of the x, y and z
// sweeps form one work list behind one cursor, so that the grid drains one tail per stage instead
// of one per direction (a warp takes 32 segments of up to 64 faces at a time, and the last ones
// run while the other SMs idle). A warp's 32 segments lie on an 8 x 4 patch of lines where the box
// allows (sweep_line_at), so that its lanes take the same Riemann-fan branch more often.
template <int RC, int RS>
__global__ void __launch_bounds__(128, MHD_FACE_MINB) k_faces(Dev D, int s0, int s1, int s2) {
  const long long t0 = sweep_threads(D, 0, s0), t1 = sweep_threads(D, 1, s1), t2 = sweep_threads(D, 2, s2);
  for_each_segment(D.work, t0 + t1 + t2, [&](long long t) {
    int dir = 0, seg = s0;
    if (t >= t0) {
      t -= t0;
      dir = 1;
      seg = s1;
      if (t >= t1) {
        t -= t1;
        dir = 2;
        seg = s2;
      }
    }
    Line ln;
    int m0, m1;
    if (sweep_line_at(D, dir, seg, t, ln, m0, m1, false, true)) face_seg<RC, RS>(D, dir, ln, m0, m1);
  });
}

template <int RC, int RS>
static void launch_faces_t(const Dev& d, int seg, cudaStream_t st) {
  const int bs = 128;
  const long long res = resident_blocks((const void*)k_faces<RC, RS>, bs);
  int sg[3];
  long long tot = 0;
  for (int dir = 0; dir < 3; ++dir) {
    sg[dir] = fill_seg(d, dir, seg, res * bs);
    tot += sweep_threads(d, dir, sg[dir]);
  }
  const long long blocks = std::min((tot + bs - 1) / bs, res);
  cudaMemsetAsync(d.work, 0, sizeof(unsigned long long), st);
  k_faces<RC, RS><<<(unsigned)blocks, bs, 0, st>>>(d, sg[0], sg[1], sg[2]);
}

template <int RC, int RS>
static void launch_face_t(const Dev& d, int dir, int seg, cudaStream_t st) {
  const int bs = 128;
  const long long threads = sweep_threads(d, dir, seg);
  k_face<RC, RS><<<(unsigned)((threads + bs - 1) / bs), bs, 0, st>>>(d, dir, seg);
}

template <int RC>
static void launch_face_r(const Dev& d, int dir, int rs, int seg, cudaStream_t st) {
  if (dir < 0) {  // all three directions in one launch
    switch (rs) {
      case RS_HLL: launch_faces_t<RC, RS_HLL>(d, seg, st); break;
      case RS_HLLD: launch_faces_t<RC, RS_HLLD>(d, seg, st); break;
      default: launch_faces_t<RC, RS_LLF>(d, seg, st); break;
    }
    return;
  }
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

int launch_faces(const Dev& d, int recon, int rs, int seg, cudaStream_t st) {
  if (!d.work) {  // no work cursors: one launch per direction, one thread per segment
    for (int dir = 0; dir < 3; ++dir) launch_face(d, dir, recon, rs, seg, st);
    return 3;
  }
  launch_face(d, -1, recon, rs, seg, st);
  return 1;
}

}  // namespace mhd
