// mhd_edge.cu -- edge-sweep kernels of the single-box step (bodies in mhd_edge.cuh).
#include <algorithm>

#include "mhd_edge.cuh"

namespace mhd {

// one thread per segment (the form without work cursors: mhd_step_noalloc)
template <int RC, int EMF>
__global__ void __launch_bounds__(128) k_edge_bt(Dev D, int e, int seg) {
  const int dir = (e + 2) % 3;
  Line ln;
  int m0, m1;
  if (!sweep_line(D, dir, seg, ln, m0, m1, dir == 0)) return;
  edge_bt_seg<RC, EMF>(D, e, ln, m0, m1);
}

template <int RC>
__global__ void __launch_bounds__(128) k_b25_cell_to_face(Dev D, int e, int to_a, int seg) {
  Line ln;
  int m0, m1;
  const int dir = to_a ? (e + 1) % 3 : (e + 2) % 3;
  if (!sweep_line(D, dir, seg, ln, m0, m1, dir == 0)) return;
  b25_seg<RC>(D, e, to_a, ln, m0, m1);
}

template <int RC, int EMF>
__global__ void __launch_bounds__(128) k_edge_lr(Dev D, int e, int seg) {
  const int dir = (e + 1) % 3;
  Line ln;
  int m0, m1;
  if (!sweep_line(D, dir, seg, ln, m0, m1, dir == 0)) return;
  edge_lr_seg<RC, EMF>(D, e, ln, m0, m1);
}

// The three edge sweeps of one kind (LR: lines along a = e + 1, else along c = e + 2) as one
// persistent launch: the segments of the e = 0, 1, 2 sweeps form one work list behind one cursor,
// so that the grid drains one tail instead of three. Along y and z a warp's segments lie on an
// 8 x 4 patch of lines where the box allows (sweep_line_at).
template <int RC, int EMF, bool LR>
__global__ void __launch_bounds__(128) k_edges(Dev D, int s0, int s1, int s2) {
  const int sg[3] = {s0, s1, s2};
  long long tot[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) tot[e] = sweep_threads(D, LR ? (e + 1) % 3 : (e + 2) % 3, sg[e]);
  for_each_segment(D.work + (LR ? 6 : 3), tot[0] + tot[1] + tot[2], [&](long long t) {
    int e = 0;
    if (t >= tot[0]) {
      t -= tot[0];
      e = 1;
      if (t >= tot[1]) {
        t -= tot[1];
        e = 2;
      }
    }
    const int dir = LR ? (e + 1) % 3 : (e + 2) % 3;
    Line ln;
    int m0, m1;
    if (sweep_line_at(D, dir, sg[e], t, ln, m0, m1, dir == 0, dir != 0)) {
      if (LR) edge_lr_seg<RC, EMF>(D, e, ln, m0, m1);
      else edge_bt_seg<RC, EMF>(D, e, ln, m0, m1);
    }
  });
}

template <int RC, int EMF, bool LR>
static void launch_edges_t(const Dev& d, int seg, cudaStream_t st) {
  const int bs = 128;
  const long long res = resident_blocks((const void*)k_edges<RC, EMF, LR>, bs);
  int sg[3];
  long long tot = 0;
  for (int e = 0; e < 3; ++e) {
    const int dir = LR ? (e + 1) % 3 : (e + 2) % 3;
    sg[e] = edge_sweep_seg(d, dir, seg);
    if (dir != 0) sg[e] = fill_seg(d, dir, sg[e], res * bs);
    tot += sweep_threads(d, dir, sg[e]);
  }
  const long long blocks = std::min((tot + bs - 1) / bs, res);
  cudaMemsetAsync(d.work + (LR ? 6 : 3), 0, sizeof(unsigned long long), st);
  k_edges<RC, EMF, LR><<<(unsigned)blocks, bs, 0, st>>>(d, sg[0], sg[1], sg[2]);
}

template <int RC, int EMF>
static void launch_bt_t(const Dev& d, int seg, cudaStream_t st) {
  if (d.work) {
    launch_edges_t<RC, EMF, false>(d, seg, st);
    return;
  }
  const int bs = 128;
  for (int e = 0; e < 3; ++e) {
    const int c = (e + 2) % 3;
    const int sg = edge_sweep_seg(d, c, seg);
    k_edge_bt<RC, EMF><<<(unsigned)((sweep_threads(d, c, sg) + bs - 1) / bs), bs, 0, st>>>(d, e, sg);
  }
}
template <int RC, int EMF>
static void launch_lr_t(const Dev& d, int seg, cudaStream_t st) {
  if (d.work) {
    launch_edges_t<RC, EMF, true>(d, seg, st);
    return;
  }
  const int bs = 128;
  for (int e = 0; e < 3; ++e) {
    const int a = (e + 1) % 3;
    const int sg = edge_sweep_seg(d, a, seg);
    k_edge_lr<RC, EMF><<<(unsigned)((sweep_threads(d, a, sg) + bs - 1) / bs), bs, 0, st>>>(d, e, sg);
  }
}
template <int RC>
static void launch_b25_t(const Dev& d, int seg, cudaStream_t st) {
  const int bs = 128;
  for (int e = 0; e < 3; ++e)
    for (int to_a = 0; to_a < 2; ++to_a) {
      const int dir = to_a ? (e + 1) % 3 : (e + 2) % 3;
      const int sg = edge_sweep_seg(d, dir, seg);
      const long long th = sweep_threads(d, dir, sg);
      k_b25_cell_to_face<RC><<<(unsigned)((th + bs - 1) / bs), bs, 0, st>>>(d, e, to_a, sg);
    }
}

template <int RC>
static void edges_bt_r(const Dev& d, int seg, cudaStream_t st) {
  switch (d.emf) {
    case EMF_Q26: launch_bt_t<RC, EMF_Q26>(d, seg, st); break;
    case EMF_FS18: launch_bt_t<RC, EMF_FS18>(d, seg, st); break;
    default: launch_b25_t<RC>(d, seg, st); launch_bt_t<RC, EMF_B25A>(d, seg, st); break;
  }
}
template <int RC>
static void edges_lr_r(const Dev& d, int seg, cudaStream_t st) {
  switch (d.emf) {
    case EMF_Q26: launch_lr_t<RC, EMF_Q26>(d, seg, st); break;
    case EMF_FS18: launch_lr_t<RC, EMF_FS18>(d, seg, st); break;
    default: launch_lr_t<RC, EMF_B25A>(d, seg, st); break;
  }
}

// edge sweeps along c (for B25a preceded by the cell-to-face EMF sweeps)
void launch_edges_bt(const Dev& d, int recon, int seg, cudaStream_t st) {
  switch (recon) {
    case REC_PC: edges_bt_r<REC_PC>(d, seg, st); break;
    case REC_PLM_MC: edges_bt_r<REC_PLM_MC>(d, seg, st); break;
    case REC_PLM_MINMOD: edges_bt_r<REC_PLM_MINMOD>(d, seg, st); break;
    case REC_PPM: edges_bt_r<REC_PPM>(d, seg, st); break;
    default: edges_bt_r<REC_PPM_EP>(d, seg, st); break;
  }
}
void launch_edges_lr(const Dev& d, int recon, int seg, cudaStream_t st) {
  switch (recon) {
    case REC_PC: edges_lr_r<REC_PC>(d, seg, st); break;
    case REC_PLM_MC: edges_lr_r<REC_PLM_MC>(d, seg, st); break;
    case REC_PLM_MINMOD: edges_lr_r<REC_PLM_MINMOD>(d, seg, st); break;
    case REC_PPM: edges_lr_r<REC_PPM>(d, seg, st); break;
    default: edges_lr_r<REC_PPM_EP>(d, seg, st); break;
  }
}

}  // namespace mhd
