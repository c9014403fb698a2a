// mhd_batch.cuh -- device side of the batched step (many uneven periodic patches advanced
// together): the per-stage parameters, the grid barrier, the phases of a stage and the stage
// kernels. The kernels are instantiated per reconstruction in mhd_batch_<recon>.cu (five
// translation units that compile in parallel); mhd_batch.cu holds the other kernels and the host
// side.
#pragma once
#include "../../include/mhd.h"
#include "mhd_cell.cuh"
#include "mhd_edge.cuh"
#include "mhd_face.cuh"

namespace mhd {

struct BatchDev {
  const Dev* patches;             // per-patch parameters of this stage, [npatch]
  const int* order;               // patch visited at schedule position k, [npatch]
  const long long* cell_pref;     // [npatch + 1] cells before schedule position k
  const long long* sweep_pref;    // [4][npatch + 1] sweep segments along dir (row 3: the edge sweeps'
                                  // segments along x) before position k
  int npatch;
  int seg;
  int stage;
  int fofc;
  int emf;                        // EMF compute scheme of every patch (EMF_Q26, EMF_FS18, EMF_B25A)
  unsigned* barrier;              // [0] arrivals, [1] generation
  unsigned long long* counters;   // [0] stage-1 flags, [1] stage-2 flags, [2] max speed, [7] error
  long long spin_limit;           // bounded wait per barrier (iterations of ~100 ns)
  int barrier_extra;              // test hook: wait for this many blocks more than launched
  unsigned long long* ptime;      // [2][8] global-timer stamps at the phase boundaries of each stage
  unsigned long long* cursor;     // [5] work-list cursors of the face, edge_bt, edge_lr and B25a's two
                                  // cell-EMF phases
  unsigned* patch_flags;          // [2][npatch] flagged cells per stage and schedule position
};

// position k with pref[k] <= i < pref[k + 1]
__device__ __forceinline__ int find_pos(const long long* pref, int n, long long i) {
  int lo = 0, hi = n;  // invariant pref[lo] <= i < pref[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pref[mid] <= i) lo = mid; else hi = mid;
  }
  return lo;
}

// schedule position of item i at or after k (a thread's items only grow, by less than a patch)
__device__ __forceinline__ int advance_pos(const long long* pref, int k, long long i) {
  while (pref[k + 1] <= i) ++k;
  return k;
}

// block 0 stamps the global timer (ns) when it passes phase boundary j of this stage
__device__ __forceinline__ void stamp(const BatchDev& B, int j) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    B.ptime[8 * B.stage + j] = t;
  }
}

// Grid-wide barrier with a bounded wait: false (and the error flag set) if the other blocks did
// not all arrive within the limit; the caller then leaves the kernel.
__device__ inline bool grid_sync(const BatchDev& B) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned expected = gridDim.x + (unsigned)B.barrier_extra;
    volatile unsigned* vgen = B.barrier + 1;
    const unsigned gen = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(B.barrier, 1u);
    int ok = 1;
    if (arrived == expected - 1) {
      atomicExch(B.barrier, 0u);
      __threadfence();
      atomicAdd(B.barrier + 1, 1u);
    } else {
      long long spins = 0;
      while (*vgen == gen) {
        if (++spins > B.spin_limit || *(volatile unsigned long long*)(B.counters + 7)) {
          ok = 0;
          atomicExch(B.counters + 7, 1ull);
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// One sweep phase: the sweeps along dirs[0..2] of every patch form one work list (sweep j's
// segments after those of sweeps 0 .. j-1, patches in schedule order), taken 32 segments at a
// time per warp from `cursor`; fn(D, j, line, m0, m1) runs each segment. In the edge phases
// (EDGE) the lines along x are cut as the single-box edge sweeps cut them: short segments
// numbered along the line, so that a warp walks whole lines (one thread per x-line would stream
// a separate cache line per thread and array).
template <bool EDGE = false, class Fn>
__device__ __forceinline__ void sweep_phase(const BatchDev& B, unsigned long long* cursor, const int* dirs, Fn fn) {
  const long long* pref[3];
  long long tot[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    pref[j] = B.sweep_pref + ((EDGE && dirs[j] == 0) ? 3 : dirs[j]) * (B.npatch + 1);
    tot[j] = pref[j][B.npatch];
  }
  for_each_segment(cursor, tot[0] + tot[1] + tot[2], [&](long long t) {
    int j = 0;
    if (t >= tot[0]) {
      t -= tot[0];
      j = 1;
      if (t >= tot[1]) {
        t -= tot[1];
        j = 2;
      }
    }
    const int k = find_pos(pref[j], B.npatch, t);
    const Dev& D = B.patches[B.order[k]];
    const bool xl = EDGE && dirs[j] == 0;
    Line ln;
    int m0, m1;
    // (warps on 8 x 4 patches of lines, as in the single-box sweeps)
    if (sweep_line_at(D, dirs[j], xl ? edge_sweep_seg(D, 0, B.seg) : B.seg, t - pref[j][k], ln, m0, m1, xl, !xl))
      fn(D, j, ln, m0, m1);
  });
}

// cells per thread per pass of the per-cell phases: the face launch has few warps per SM to hide
// memory latency, the other launch twice as many
constexpr int kCellIlp = 4;
constexpr int kRestIlp = 2;
// CTAs of 128 threads per SM that the second launch of a stage is compiled to fit (one fewer for
// FS18, whose bottom/top sweep carries five reconstruction windows)
constexpr int kRestMinBlocks = 4;

// The phases of a stage, as device functions that the stage's launches run: false when a grid
// barrier gave up (the block then leaves the kernel).
//
// Stage 2's primitives (where flux correction changed stage 1's result) and the face sweeps.
template <int RC, int RS>
__device__ __forceinline__ bool face_part(const BatchDev& B) {
  // a barrier of an earlier launch gave up (the flag stays set until the host reads it): the
  // step is abandoned and the caller's state left as it was
  if (*(volatile unsigned long long*)(B.counters + 7)) return false;
  const long long nth = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long ncell = B.cell_pref[B.npatch];
  const int k0 = t0 < ncell ? find_pos(B.cell_pref, B.npatch, t0) : 0;
  stamp(B, 0);
  // the sweep phases' cursors start at zero: the face phase's is taken only after the grid
  // barrier below, which block 0 passes only after this, the edge phases' after later barriers or
  // in the next launch
  if (blockIdx.x == 0 && threadIdx.x < 5) atomicExch(B.cursor + threadIdx.x, 0ull);
  // per-patch flag counts of this stage start at zero (written and read after later barriers)
  unsigned* const pflags = B.patch_flags + (long long)B.stage * B.npatch;
  for (long long i = t0; i < B.npatch; i += nth) pflags[i] = 0u;
  // cons -> prim, kCellIlp cells per thread at a time, loads of all of them before any store.
  // Stage 1's primitives come from the CFL reduction, stage 2's from stage 1's flag phase unless
  // flux correction changed its state (per patch: only patches where stage 1 flagged a cell are
  // redone).
  const bool prim_given = B.stage == 0 || *(volatile unsigned long long*)(B.counters + 0) == 0;
  for (long long i0 = t0, k = k0; i0 < ncell && !prim_given; i0 += kCellIlp * nth) {
    double w[kCellIlp][8];
    const Dev* Dp[kCellIlp];
    long long X[kCellIlp];
#pragma unroll
    for (int g = 0; g < kCellIlp; ++g) {
      const long long i = i0 + g * nth;
      Dp[g] = nullptr;
      if (i < ncell) {
        k = advance_pos(B.cell_pref, (int)k, i);
        if (B.stage == 1 && B.patch_flags[k] == 0u) continue;  // stage 1 left this patch's primitives
        Dp[g] = &B.patches[B.order[k]];
        X[g] = i - B.cell_pref[k];
        prim_of(*Dp[g], Dp[g]->Uin, Dp[g]->Bin, X[g], w[g]);
      }
    }
#pragma unroll
    for (int g = 0; g < kCellIlp; ++g)
      if (Dp[g])
        for (int v = 0; v < 8; ++v) Dp[g]->P[v * Dp[g]->N + X[g]] = w[g][v];
  }
  if (!grid_sync(B)) return false;
  stamp(B, 1);
  // face sweeps along each direction
  const int dirs[3] = {0, 1, 2};
  sweep_phase(B, B.cursor + 0, dirs, [&](const Dev& D, int j, const Line& ln, int m0, int m1) {
    face_seg<RC, RS>(D, j, ln, m0, m1);
  });
  return true;
}

// The edge sweeps (for B25a after its cell-EMF sweeps), the update and the validity flags of the
// stage, for the EMF compute scheme EMF, ILP cells per thread at a time in the per-cell phases.
template <int RC, int EMF, int ILP>
__device__ __forceinline__ bool rest_part(const BatchDev& B) {
  if (*(volatile unsigned long long*)(B.counters + 7)) return false;  // an earlier launch gave up
  const long long nth = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long ncell = B.cell_pref[B.npatch];
  const int k0 = t0 < ncell ? find_pos(B.cell_pref, B.npatch, t0) : 0;
  unsigned* const pflags = B.patch_flags + (long long)B.stage * B.npatch;
  stamp(B, 2);
  if (EMF == EMF_B25A) {
    // the cell-centred EMF reconstructed to the a-faces (lines along a = e + 1) and to the c-faces
    // (lines along c = e + 2): two independent work lists, no barrier between them
    const int dirs_a[3] = {1, 2, 0}, dirs_c[3] = {2, 0, 1};
    sweep_phase<true>(B, B.cursor + 3, dirs_a, [&](const Dev& D, int e, const Line& ln, int m0, int m1) {
      b25_seg<RC>(D, e, 1, ln, m0, m1);
    });
    sweep_phase<true>(B, B.cursor + 4, dirs_c, [&](const Dev& D, int e, const Line& ln, int m0, int m1) {
      b25_seg<RC>(D, e, 0, ln, m0, m1);
    });
    if (!grid_sync(B)) return false;
  }
  // a-face quantities to e-edges (lines along c = e + 2)
  {
    const int dirs[3] = {2, 0, 1};
    sweep_phase<true>(B, B.cursor + 1, dirs, [&](const Dev& D, int e, const Line& ln, int m0, int m1) {
      edge_bt_seg<RC, EMF>(D, e, ln, m0, m1);
    });
  }
  if (!grid_sync(B)) return false;
  stamp(B, 3);
  // c-face quantities to e-edges (lines along a = e + 1) and the edge EMFs
  {
    const int dirs[3] = {1, 2, 0};
    sweep_phase<true>(B, B.cursor + 2, dirs, [&](const Dev& D, int e, const Line& ln, int m0, int m1) {
      edge_lr_seg<RC, EMF>(D, e, ln, m0, m1);
    });
  }
  if (!grid_sync(B)) return false;
  stamp(B, 4);
  // update, then (after a grid barrier) the validity flags of the new state, which the flag pass
  // reads back instead of recomputing each cell's upper faces
  {
    int ku = k0;
    for (long long base = t0; base < ncell; base += ILP * nth) {
      double w[ILP][8];
      const Dev* Dp[ILP];
      long long X[ILP];
#pragma unroll
      for (int g = 0; g < ILP; ++g) {
        const long long i = base + g * nth;
        Dp[g] = nullptr;
        if (i < ncell) {
          ku = advance_pos(B.cell_pref, ku, i);
          Dp[g] = &B.patches[B.order[ku]];
          X[g] = i - B.cell_pref[ku];
          update_vals(*Dp[g], X[g], w[g]);
        }
      }
#pragma unroll
      for (int g = 0; g < ILP; ++g)
        if (Dp[g]) store_update(*Dp[g], X[g], w[g]);
    }
  }
  if (!grid_sync(B)) return false;
  // (every lane of a warp runs the same number of passes for the ballot)
  int kf = k0;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < ncell; base += ILP * nth) {
    double u[ILP][5], lo[ILP][3], hi[ILP][3], pw[ILP][8];
    int K[ILP];
    bool f[ILP];
    const Dev* Dp[ILP];
    long long X[ILP];
#pragma unroll
    for (int g = 0; g < ILP; ++g) {
      const long long i = base + g * nth + threadIdx.x;
      Dp[g] = nullptr;
      if (i < ncell) {
        kf = advance_pos(B.cell_pref, kf, i);
        Dp[g] = &B.patches[B.order[kf]];
        X[g] = i - B.cell_pref[kf];
        K[g] = kf;
        load_cell(*Dp[g], Dp[g]->Uout, Dp[g]->Bout, X[g], u[g], lo[g], hi[g]);
      }
    }
    unsigned cnt = 0;
#pragma unroll
    for (int g = 0; g < ILP; ++g) {
      f[g] = false;
      if (Dp[g]) {
        // stage 1 also forms the primitives of its result (stage 2's input), and reads the
        // pressure of the validity test from them
        f[g] = B.stage == 0 ? prim_invalid(*Dp[g], u[g], lo[g], hi[g], pw[g])
                            : invalid_vals(*Dp[g], u[g], lo[g], hi[g]);
        Dp[g]->flag[X[g]] = f[g] ? 1 : 0;
        if (f[g]) atomicAdd(&pflags[K[g]], 1u);
        if (B.stage == 0)  // the primitives of S^{n+1/2}, stage 2's input
          for (int v = 0; v < 8; ++v) Dp[g]->P[v * Dp[g]->N + X[g]] = pw[g][v];
      }
      cnt += __popc(__ballot_sync(0xffffffffu, f[g]));
    }
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&B.counters[B.stage], (unsigned long long)cnt);
  }
  return true;
}

// First-order correction of the flagged patches' faces and edges and recompute of their touched
// cells (it returns at once when the stage flagged nothing; the flag counts are complete: a grid
// barrier or a launch boundary lies between the flag phase and this).
__device__ __forceinline__ void fofc_part(const BatchDev& B) {
  if (*(volatile unsigned long long*)(B.counters + 7)) return;  // an earlier launch gave up
  stamp(B, 5);
  if (*(volatile unsigned long long*)(B.counters + B.stage) == 0) return;  // uniform over the grid
  const long long nth = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long ncell = B.cell_pref[B.npatch];
  const int k0 = t0 < ncell ? find_pos(B.cell_pref, B.npatch, t0) : 0;
  const unsigned* const pflags = B.patch_flags + (long long)B.stage * B.npatch;
  // patches are independent boxes: only those with a flagged cell have anything to correct
  for (long long i = t0, k = k0; i < ncell; i += nth) {
    k = advance_pos(B.cell_pref, (int)k, i);
    if (pflags[k] == 0u) continue;
    const Dev& D = B.patches[B.order[k]];
    fo_faces_cell(D, i - B.cell_pref[k]);
    fo_edges_cell(D, i - B.cell_pref[k]);
  }
  if (!grid_sync(B)) return;
  stamp(B, 6);
  for (long long i = t0, k = k0; i < ncell; i += nth) {
    k = advance_pos(B.cell_pref, (int)k, i);
    if (pflags[k] == 0u) continue;
    fo_recompute_cell(B.patches[B.order[k]], i - B.cell_pref[k]);
  }
}

// The stage's launches. One launch per stage runs every phase at the face sweep's register
// budget; three launches per stage run the edge, update and flag phases at half that budget (twice
// the warps per SM) and the first-order correction apart.
template <int RC, int RS, int EMF>
__device__ __forceinline__ void stage_all(const BatchDev& B) {
  if (!face_part<RC, RS>(B)) return;
  if (!grid_sync(B)) return;
  if (!rest_part<RC, EMF, kCellIlp>(B)) return;
  if (!B.fofc) return;
  if (!grid_sync(B)) return;
  fofc_part(B);
}
template <int RC, int RS>
__global__ void __launch_bounds__(128) k_batch_stage(BatchDev B) {
  switch (B.emf) {  // uniform over the grid
    case EMF_FS18: stage_all<RC, RS, EMF_FS18>(B); break;
    case EMF_B25A: stage_all<RC, RS, EMF_B25A>(B); break;
    default: stage_all<RC, RS, EMF_Q26>(B); break;
  }
}
template <int RC, int RS>
__global__ void __launch_bounds__(128) k_batch_face(BatchDev B) {
  face_part<RC, RS>(B);
}
template <int RC, int EMF>
__global__ void __launch_bounds__(128, EMF == EMF_FS18 ? kRestMinBlocks - 1 : kRestMinBlocks) k_batch_rest(BatchDev B) {
  rest_part<RC, EMF, kRestIlp>(B);
}

typedef void (*StageKernel)(BatchDev);

// The stage kernels of reconstruction RC. which: 0 the one launch per stage (for rs), 1 the face
// launch of three (for rs), 2 the edge / update / flag launch (for emf).
template <int RC>
StageKernel batch_kernel_impl(int which, int rs, int emf) {
  if (which == 2) {
    switch (emf) {
      case EMF_FS18: return k_batch_rest<RC, EMF_FS18>;
      case EMF_B25A: return k_batch_rest<RC, EMF_B25A>;
      default: return k_batch_rest<RC, EMF_Q26>;
    }
  }
  switch (rs) {
    case RS_HLL: return which == 0 ? k_batch_stage<RC, RS_HLL> : k_batch_face<RC, RS_HLL>;
    case RS_HLLD: return which == 0 ? k_batch_stage<RC, RS_HLLD> : k_batch_face<RC, RS_HLLD>;
    default: return which == 0 ? k_batch_stage<RC, RS_LLF> : k_batch_face<RC, RS_LLF>;
  }
}
// defined, one reconstruction each, in mhd_batch_<recon>.cu
template <int RC>
StageKernel batch_kernel(int which, int rs, int emf);
template <> StageKernel batch_kernel<REC_PC>(int which, int rs, int emf);
template <> StageKernel batch_kernel<REC_PLM_MC>(int which, int rs, int emf);
template <> StageKernel batch_kernel<REC_PLM_MINMOD>(int which, int rs, int emf);
template <> StageKernel batch_kernel<REC_PPM>(int which, int rs, int emf);
template <> StageKernel batch_kernel<REC_PPM_EP>(int which, int rs, int emf);

}  // namespace mhd
