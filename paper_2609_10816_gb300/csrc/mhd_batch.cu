// mhd_batch.cu -- many uneven periodic patches advanced together (the batched form of the step):
// the CFL reduction, dt and copy-back kernels, the first-order correction launch and the host side.
//
// Each RK stage runs as one persistent cooperative launch, or as three (face phase; edge, update
// and flag phases at half the face phase's register budget; first-order correction), whose blocks
// walk, phase after phase, work lists that span every patch (cells for the per-cell phases, line
// segments of the sweeps for the face and edge phases), separated by a grid-wide barrier of the
// library's own with a bounded wait (mhd_batch.cuh). The CFL reduction and the time step stay on
// the device, so one step (reduction, dt, stage 1, stage 2, copy back) is captured once as a CUDA
// graph and replayed. Launch form, patch order, sweep segment length and the first launch's CTAs
// per SM form the schedule that mhd_batch_tune picks by timing candidates.
#include <algorithm>
#include <cstring>
#include <tuple>
#include <array>
#include <mutex>
#include <map>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/mhd.h"
#include "mhd_batch.cuh"

namespace mhd {

// the correction at the face sweep's register budget (it solves several face problems per cell)
__global__ void __launch_bounds__(128) k_batch_fofc(BatchDev B) { fofc_part(B); }

// max over all cells of all patches of the CFL signal speed (Sec. 2.4, cfl_speed_max), with the
// running maximum shared across each warp after every pass
__global__ void __launch_bounds__(256) k_batch_maxspeed(BatchDev B) {
  const long long nth = (long long)gridDim.x * blockDim.x;
  const long long ncell = B.cell_pref[B.npatch];
  const int lane = threadIdx.x & 31;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int k = t0 < ncell ? find_pos(B.cell_pref, B.npatch, t0) : 0;
  double s = 0.0;
  for (long long base = t0 - lane; base < ncell; base += nth) {  // uniform over the warp
    const long long i = base + lane;
    if (i < ncell) {
      k = advance_pos(B.cell_pref, k, i);
      const Dev& D = B.patches[B.order[k]];
      s = cfl_speed_max(D, D.U0, D.B0, i - B.cell_pref[k], s, D.P);  // and stage 1's primitives
    }
    unsigned long long b = (unsigned long long)dbits(s);
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long t = __shfl_xor_sync(0xffffffffu, b, o);
      b = t > b ? t : b;
    }
    s = __longlong_as_double((long long)b);
  }
  // block max then one atomic
  unsigned long long bits = (unsigned long long)dbits(s);
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, bits, o);
    bits = t > bits ? t : bits;
  }
  __shared__ unsigned long long sm[32];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = bits;
  __syncthreads();
  if (threadIdx.x < 32) {
    bits = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long t = __shfl_xor_sync(0xffffffffu, bits, o);
      bits = t > bits ? t : bits;
    }
    if (threadIdx.x == 0) atomicMax(B.counters + 2, bits);
  }
}

// dt = cfl hmin / max(smax, 2 eta / hmin), written into both stages' patch parameters and out
__global__ void k_batch_set_dt(Dev* p0, Dev* p1, int npatch, const unsigned long long* smax_bits, double cfl,
                               double eta, double hmin, double* dt_out, unsigned long long* err) {
  double smax = __longlong_as_double((long long)*smax_bits);
  smax = fmax(smax, 2.0 * eta / hmin);
  double dt = cfl * hmin / smax;
  if (!(dt > 0.0) || !finite_d(dt)) {  // non-finite speed: keep the step well defined, flag it
    dt = 0.0;
    if (threadIdx.x == 0 && blockIdx.x == 0) atomicExch(err, 1ull);
  }
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < npatch; k += gridDim.x * blockDim.x) {
    p0[k].dt = dt;
    p1[k].dt = dt;
    for (int d = 0; d < 3; ++d) {
      p0[k].dth[d] = dt * p0[k].hinv[d];
      p1[k].dth[d] = dt * p1[k].hinv[d];
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *dt_out = dt;
}

// S^{n+1} from the batch's scratch state into the caller's arrays, unless a grid barrier of this
// step (or of an unread earlier one) gave up; then the caller's state keeps S^n.
__global__ void __launch_bounds__(256) k_batch_copy_back(const double* __restrict__ U1, double* __restrict__ cons,
                                                        const double* __restrict__ B1, double* __restrict__ b,
                                                        long long ncell, const unsigned long long* timeout) {
  if (*(volatile const unsigned long long*)timeout) return;
  const long long nth = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nc = 5 * ncell, nb = 3 * ncell;
  for (long long i = t0; i < nc; i += nth) cons[i] = U1[i];
  for (long long i = t0; i < nb; i += nth) b[i] = B1[i];
}

static StageKernel batch_kernel_of(int recon, int which, int rs, int emf) {
  switch (recon) {
    case REC_PC: return batch_kernel<REC_PC>(which, rs, emf);
    case REC_PLM_MC: return batch_kernel<REC_PLM_MC>(which, rs, emf);
    case REC_PLM_MINMOD: return batch_kernel<REC_PLM_MINMOD>(which, rs, emf);
    case REC_PPM: return batch_kernel<REC_PPM>(which, rs, emf);
    default: return batch_kernel<REC_PPM_EP>(which, rs, emf);
  }
}
// the first launch of a stage: the one launch per stage (one) or the face launch of three
static StageKernel stage_kernel(int recon, int rs, bool one) { return batch_kernel_of(recon, one ? 0 : 1, rs, 0); }
// the second launch of three (edge, update and flag phases)
static StageKernel rest_kernel(int recon, int emf) { return batch_kernel_of(recon, 2, 0, emf); }

}  // namespace mhd

// ------------------------------------------------------------------------------------------
// Host side
// ------------------------------------------------------------------------------------------
struct mhd_batch {
  int npatch;
  std::vector<int> dims;          // 3 per patch
  std::vector<long long> off;     // cell offsets, npatch + 1
  long long ncell;
  double h, gamma;
  cudaStream_t stream;
  cudaStream_t cap;               // private stream the step graph is captured on
  int nsm;
  std::string err;
  // device memory (one allocation)
  void* mem;
  double* U1;                     // [patch][5][N_p]
  double* B1;                     // [patch][3][N_p]
  double* scratch;                // [patch][47][N_p]: P 8, F 15, Ap/Am/Us 9, Epart 12, E 3
  double* extra;                  // [patch][54][N_p] for FS18 / B25a: VL 9, VR 9, Xpart 24, EfL 6, EfB 6
                                  // (allocated by the first step that needs it)
  unsigned char* flag;
  unsigned long long* counters;   // 8
  unsigned* barrier;              // 2
  unsigned long long* ptime;      // [2][8] phase stamps of the last step
  unsigned long long* cursor;     // [3] sweep-phase work cursors
  unsigned* patch_flags;          // [2][npatch]
  double* dt_dev;
  mhd::Dev* pdev[2];              // per-patch parameters per stage
  int* order_dev;
  long long* cell_pref_dev;
  long long* sweep_pref_dev;      // 4 * (npatch + 1)
  // schedule
  int seg, order_kind, blocks_per_sm, use_graph;
  int launches_per_stage;         // 1: one persistent launch per stage; 3: face / rest / correction
  long long spin_limit;
  int barrier_extra;
  // what the current parameters / graph were built for
  const double* built_cons;
  const double* built_b;
  int built_scheme;
  double built_eta, built_cfl;
  bool params_ok;
  cudaGraphExec_t graph;
  bool graph_ok;
};

// schedules chosen by mhd_batch_tune, keyed by device, scheme and patch-size histogram
std::mutex g_tune_mu;
std::map<std::string, std::array<int, 4>> g_tune_cache;

namespace {

thread_local std::string g_batch_create_err;

mhd_status bfail(mhd_batch* b, mhd_status s, const std::string& m) {
  if (b) b->err = m;
  return s;
}
mhd_status bcuda(mhd_batch* b, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return MHD_OK;
  return bfail(b, MHD_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void drop_graph(mhd_batch* b) {
  if (b->graph_ok) cudaGraphExecDestroy(b->graph);
  b->graph_ok = false;
}

// schedule order of patches and the prefix tables of cells and sweep segments
mhd_status upload_schedule(mhd_batch* b) {
  const int np = b->npatch;
  std::vector<int> order(np);
  std::iota(order.begin(), order.end(), 0);
  if (b->order_kind == 1) {  // largest patches first
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
      return b->off[x + 1] - b->off[x] > b->off[y + 1] - b->off[y];
    });
  }
  std::vector<long long> cp(np + 1, 0), sp(4 * (np + 1), 0);
  for (int k = 0; k < np; ++k) {
    const int p = order[k];
    const int* n = &b->dims[3 * p];
    cp[k + 1] = cp[k] + (long long)n[0] * n[1] * n[2];
    for (int d = 0; d < 3; ++d) {
      const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
      const long long segs = (n[d] + b->seg - 1) / b->seg;
      sp[d * (np + 1) + k + 1] = sp[d * (np + 1) + k] + (long long)n[t1] * n[t2] * segs;
    }
    // the edge phases' segments along x: edge_sweep_seg's length, about nx / 32 points (4 to 16)
    const int sx = std::min(16, std::max(4, (n[0] + 31) / 32));
    sp[3 * (np + 1) + k + 1] = sp[3 * (np + 1) + k] + (long long)n[1] * n[2] * ((n[0] + sx - 1) / sx);
  }
  cudaError_t e = cudaMemcpyAsync(b->order_dev, order.data(), np * sizeof(int), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->cell_pref_dev, cp.data(), (np + 1) * sizeof(long long), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->sweep_pref_dev, sp.data(), 4 * (np + 1) * sizeof(long long), cudaMemcpyHostToDevice,
                        b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return bcuda(b, e, "schedule upload");
}

// per-patch stage parameters for a state, scheme and eta
mhd_status upload_params(mhd_batch* b, const mhd_batch_state* s, int scheme, double eta) {
  const int np = b->npatch;
  std::vector<mhd::Dev> d0(np), d1(np);
  const int recon = scheme & 0xf;
  (void)recon;
  for (int p = 0; p < np; ++p) {
    mhd::Dev D;
    std::memset(&D, 0, sizeof(D));
    const int* n = &b->dims[3 * p];
    const long long N = (long long)n[0] * n[1] * n[2];
    const long long o = b->off[p];
    D.n[0] = n[0]; D.n[1] = n[1]; D.n[2] = n[2];
    D.N = N;
    D.stride[0] = 1; D.stride[1] = n[0]; D.stride[2] = (long long)n[0] * n[1];
    for (int d = 0; d < 3; ++d) { D.h[d] = b->h; D.hinv[d] = 1.0 / b->h; }
    D.gam = b->gamma;
    D.gm1inv = 1.0 / (b->gamma - 1.0);
    D.eta = eta;
    D.resistive = eta != 0.0;
    D.fofc_criteria = (scheme & MHD_FOFC_OFF) ? 0 : 3;
    D.emf = (scheme >> 8) & 0xf;
    if (D.emf != mhd::EMF_Q26) {
      double* x = b->extra + 54 * o;
      D.VL = x; x += 9 * N;
      D.VR = x; x += 9 * N;
      D.Xpart = x; x += 24 * N;
      D.EfL = x; x += 6 * N;
      D.EfB = x;
    }
    D.U0 = s->cons + 5 * o;
    for (int d = 0; d < 3; ++d) D.B0[d] = s->b + 3 * o + d * N;
    double* q = b->scratch + 47 * o;
    D.P = q; q += 8 * N;
    D.F = q; q += 15 * N;
    D.Ap = q; q += 3 * N;
    D.Am = q; q += 3 * N;
    D.Us = q; q += 3 * N;
    D.Epart = q; q += 12 * N;
    D.E = q;
    D.flag = b->flag + o;
    D.counters = b->counters;
    double* U1 = b->U1 + 5 * o;
    double* B1 = b->B1 + 3 * o;
    D.Uout = U1;
    for (int d = 0; d < 3; ++d) D.Bout[d] = B1 + d * N;
    // stage 1 reads S^n, stage 2 reads S^{n+1/2}; both write the scratch state
    mhd::Dev A = D;
    A.Uin = A.U0;
    for (int d = 0; d < 3; ++d) A.Bin[d] = A.B0[d];
    A.combine = 0;
    A.stage = 0;
    mhd::Dev C = D;
    C.Uin = U1;
    for (int d = 0; d < 3; ++d) C.Bin[d] = B1 + d * N;
    C.combine = 1;
    C.stage = 1;
    d0[p] = A;
    d1[p] = C;
  }
  cudaError_t e = cudaMemcpyAsync(b->pdev[0], d0.data(), np * sizeof(mhd::Dev), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->pdev[1], d1.data(), np * sizeof(mhd::Dev), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return bcuda(b, e, "parameter upload");
}

mhd::BatchDev batch_dev(mhd_batch* b, int stage, bool fofc, int emf) {
  mhd::BatchDev B;
  B.patches = b->pdev[stage];
  B.order = b->order_dev;
  B.cell_pref = b->cell_pref_dev;
  B.sweep_pref = b->sweep_pref_dev;
  B.npatch = b->npatch;
  B.seg = b->seg;
  B.stage = stage;
  B.fofc = fofc ? 1 : 0;
  B.emf = emf;
  B.barrier = b->barrier;
  B.counters = b->counters;
  B.spin_limit = b->spin_limit;
  B.barrier_extra = b->barrier_extra;
  B.ptime = b->ptime;
  B.cursor = b->cursor;
  B.patch_flags = b->patch_flags;
  return B;
}

// A barrier gave up in a step since the last report: clear the sticky flag (steps run again from
// the next call) and return the error.
mhd_status report_timeout(mhd_batch* b) {
  cudaError_t e = cudaMemsetAsync(b->counters + 7, 0, sizeof(unsigned long long), b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "clear the barrier flag");
  return bfail(b, MHD_ERR_TIMEOUT,
               "a grid barrier of the batched stage gave up waiting; the steps since the last check left the "
               "state unchanged");
}

// enqueue one whole step on the stream (also used for graph capture)
mhd_status enqueue_step(mhd_batch* b, const mhd_batch_state* s, double cfl, int scheme, double eta,
                        cudaStream_t st) {
  const bool fofc = !(scheme & MHD_FOFC_OFF);
  const int recon = scheme & 0xf, rs = (scheme >> 4) & 0xf, emf = (scheme >> 8) & 0xf;
  const bool one = b->launches_per_stage == 1;
  mhd::StageKernel kf = mhd::stage_kernel(recon, rs, one), kr = mhd::rest_kernel(recon, emf);
  int per_sm = 0, per_sm_rest = 0;
  int per_sm_fofc = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kf, 128, 0);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_rest, kr, 128, 0);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_fofc, (const void*)mhd::k_batch_fofc, 128, 0);
  if (e != cudaSuccess) return bcuda(b, e, "occupancy query");
  if (per_sm < 1 || per_sm_rest < 1 || per_sm_fofc < 1)
    return bfail(b, MHD_ERR_CUDA, "stage kernel cannot be resident");
  const int bps = b->blocks_per_sm > 0 ? std::min(b->blocks_per_sm, per_sm) : per_sm;
  const unsigned grid_face = (unsigned)(b->nsm * bps), grid_rest = (unsigned)(b->nsm * per_sm_rest);
  const unsigned grid_fofc = (unsigned)(b->nsm * per_sm_fofc);
  // counters 0..6 start each step at zero; counter 7 (a barrier gave up) is cleared only when
  // mhd_batch_last_dt or mhd_batch_stats reports it
  e = cudaMemsetAsync(b->counters, 0, 7 * sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->barrier, 0, 2 * sizeof(unsigned), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->ptime, 0, 16 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return bcuda(b, e, "cudaMemsetAsync");
  mhd::BatchDev B0 = batch_dev(b, 0, fofc, emf);
  mhd::k_batch_maxspeed<<<b->nsm * 8, 256, 0, st>>>(B0);
  mhd::k_batch_set_dt<<<(b->npatch + 255) / 256, 256, 0, st>>>(
      b->pdev[0], b->pdev[1], b->npatch, b->counters + 2, cfl, eta, b->h, b->dt_dev, b->counters + 6);
  for (int stage = 0; stage < 2; ++stage) {
    mhd::BatchDev B = batch_dev(b, stage, fofc, emf);
    void* args[] = {&B};
    for (int part = 0; part < (one ? 1 : (fofc ? 3 : 2)); ++part) {
      cudaLaunchConfig_t lc;
      std::memset(&lc, 0, sizeof(lc));
      lc.gridDim = dim3(part == 1 ? grid_rest : (part == 0 ? grid_face : grid_fofc));
      lc.blockDim = dim3(128);
      lc.stream = st;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeCooperative;
      at[0].val.cooperative = 1;
      lc.attrs = at;
      lc.numAttrs = 1;
      const void* k = part == 0 ? (const void*)kf : (part == 1 ? (const void*)kr : (const void*)mhd::k_batch_fofc);
      e = cudaLaunchKernelExC(&lc, k, args);
      if (e != cudaSuccess) return bcuda(b, e, "cooperative stage launch");
    }
  }
  mhd::k_batch_copy_back<<<b->nsm * 8, 256, 0, st>>>(b->U1, s->cons, b->B1, s->b, b->ncell, b->counters + 7);
  e = cudaGetLastError();
  return bcuda(b, e, "batch step enqueue");
}

}  // namespace

extern "C" {

const char* mhd_batch_last_error(const mhd_batch* b) { return b ? b->err.c_str() : g_batch_create_err.c_str(); }

mhd_status mhd_batch_create(const int* dims, int npatch, double h, double gamma, void* cuda_stream, mhd_batch** out) {
  g_batch_create_err.clear();
  if (!out) return MHD_ERR_ARG;
  *out = nullptr;
  if (!dims || npatch < 1 || !(h > 0) || !(gamma > 1.0)) {
    g_batch_create_err = "need dims, npatch >= 1, h > 0, gamma > 1";
    return MHD_ERR_ARG;
  }
  mhd_batch* b = new mhd_batch();
  b->npatch = npatch;
  b->dims.assign(dims, dims + 3 * npatch);
  b->off.assign(npatch + 1, 0);
  for (int p = 0; p < npatch; ++p) {
    const int* n = &dims[3 * p];
    if (n[0] < 1 || n[1] < 1 || n[2] < 1 || (long long)n[0] * n[1] * n[2] > (1LL << 31) - 1) {
      g_batch_create_err = "every patch needs n >= 1 cells per direction and fewer than 2^31 cells";
      delete b;
      return MHD_ERR_ARG;
    }
    b->off[p + 1] = b->off[p] + (long long)n[0] * n[1] * n[2];
  }
  b->ncell = b->off[npatch];
  if (b->ncell > (1LL << 34)) {
    g_batch_create_err = "batch too large";
    delete b;
    return MHD_ERR_ARG;
  }
  b->h = h;
  b->gamma = gamma;
  b->stream = (cudaStream_t)cuda_stream;
  if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
    g_batch_create_err = "cudaStreamCreateWithFlags failed";
    delete b;
    return MHD_ERR_CUDA;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
  b->seg = 64;
  b->order_kind = 1;
  b->blocks_per_sm = 0;
  b->use_graph = 1;
  b->launches_per_stage = 1;
  b->spin_limit = 1LL << 25;  // ~3 s of waiting before a barrier gives up
  b->barrier_extra = 0;
  b->graph_ok = false;
  b->params_ok = false;
  b->extra = nullptr;
  const long long C = b->ncell;
  size_t bytes = (size_t)C * (5 + 3 + 47) * sizeof(double) + (size_t)C + 24 * 256 +
                 2 * npatch * sizeof(mhd::Dev) + 3 * npatch * sizeof(int) + 5 * (npatch + 1) * sizeof(long long);
  cudaError_t e = cudaMalloc(&b->mem, bytes);
  if (e != cudaSuccess) {
    g_batch_create_err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    cudaStreamDestroy(b->cap);
    delete b;
    return MHD_ERR_CUDA;
  }
  char* q = (char*)b->mem;
  auto take = [&](size_t n) { char* r = q; q += (n + 255) / 256 * 256; return r; };
  b->U1 = (double*)take(C * 5 * sizeof(double));
  b->B1 = (double*)take(C * 3 * sizeof(double));
  b->scratch = (double*)take(C * 47 * sizeof(double));
  b->counters = (unsigned long long*)take(8 * sizeof(unsigned long long));
  b->barrier = (unsigned*)take(2 * sizeof(unsigned));
  b->ptime = (unsigned long long*)take(16 * sizeof(unsigned long long));
  b->cursor = (unsigned long long*)take(8 * sizeof(unsigned long long));
  b->patch_flags = (unsigned*)take(2 * npatch * sizeof(unsigned));
  b->dt_dev = (double*)take(sizeof(double));
  b->pdev[0] = (mhd::Dev*)take(npatch * sizeof(mhd::Dev));
  b->pdev[1] = (mhd::Dev*)take(npatch * sizeof(mhd::Dev));
  b->order_dev = (int*)take(npatch * sizeof(int));
  b->cell_pref_dev = (long long*)take((npatch + 1) * sizeof(long long));
  b->sweep_pref_dev = (long long*)take(4 * (npatch + 1) * sizeof(long long));
  b->flag = (unsigned char*)q;
  if ((size_t)(q - (char*)b->mem) + C > bytes) {  // layout check (padding consumed the slack)
    cudaFree(b->mem);
    cudaStreamDestroy(b->cap);
    g_batch_create_err = "internal layout error";
    delete b;
    return MHD_ERR_CUDA;
  }
  e = cudaMemsetAsync(b->mem, 0, bytes, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    cudaFree(b->mem);
    cudaStreamDestroy(b->cap);
    g_batch_create_err = std::string("init: ") + cudaGetErrorString(e);
    delete b;
    return MHD_ERR_CUDA;
  }
  mhd_status s = upload_schedule(b);
  if (s != MHD_OK) {
    g_batch_create_err = b->err;
    cudaFree(b->mem);
    cudaStreamDestroy(b->cap);
    delete b;
    return s;
  }
  *out = b;
  return MHD_OK;
}

void mhd_batch_destroy(mhd_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  drop_graph(b);
  cudaStreamDestroy(b->cap);
  cudaFree(b->mem);
  if (b->extra) cudaFree(b->extra);
  delete b;
}

mhd_status mhd_batch_offsets(const mhd_batch* b, long long* cell_offsets) {
  if (!b || !cell_offsets) return MHD_ERR_ARG;
  for (int p = 0; p <= b->npatch; ++p) cell_offsets[p] = b->off[p];
  return MHD_OK;
}

mhd_status mhd_batch_set_schedule(mhd_batch* b, int seg, int order, int blocks_per_sm, int use_graph) {
  if (!b) return MHD_ERR_ARG;
  if (seg < 1 || seg > 4096 || order < 0 || order > 1 || blocks_per_sm < 0)
    return bfail(b, MHD_ERR_ARG, "need 1 <= seg <= 4096, order 0/1, blocks_per_sm >= 0");
  mhd_status s = bcuda(b, cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
  if (s != MHD_OK) return s;
  b->seg = seg;
  b->order_kind = order;
  b->blocks_per_sm = blocks_per_sm;
  b->use_graph = use_graph ? 1 : 0;
  drop_graph(b);
  return upload_schedule(b);
}

mhd_status mhd_batch_step(mhd_batch* b, const mhd_batch_state* s, double cfl, int scheme, double eta) {
  if (!b) return MHD_ERR_ARG;
  b->err.clear();
  if (!s || !s->cons || !s->b) return bfail(b, MHD_ERR_ARG, "state has a NULL array");
  if (!(cfl > 0) || !(cfl < 1e300)) return bfail(b, MHD_ERR_ARG, "cfl must be finite and > 0");
  if (!(eta >= 0) || !(eta < 1e300)) return bfail(b, MHD_ERR_ARG, "eta must be finite and >= 0");
  if (scheme & ~(0xffff | MHD_FOFC_OFF)) return bfail(b, MHD_ERR_ARG, "unknown scheme bits");
  const int recon = scheme & 0xf, rs = (scheme >> 4) & 0xf, emf = (scheme >> 8) & 0xf, avg = (scheme >> 12) & 0xf;
  if (avg == 1) return bfail(b, MHD_ERR_UNSUPPORTED, "B25b averaging is cited but not defined in the paper");
  if (recon > 4 || rs > 2 || emf > 2 || avg > 1) return bfail(b, MHD_ERR_ARG, "scheme field out of range");
  if (emf != mhd::EMF_Q26 && !b->extra) {  // FS18 / B25a arrays, on the first step that needs them
    mhd_status st = bcuda(b, cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
    if (st != MHD_OK) return st;
    st = bcuda(b, cudaMalloc(&b->extra, (size_t)b->ncell * 54 * sizeof(double)), "cudaMalloc of FS18/B25a arrays");
    if (st != MHD_OK) {
      b->extra = nullptr;
      return st;
    }
  }
  const bool same = b->params_ok && b->built_cons == s->cons && b->built_b == s->b && b->built_scheme == scheme &&
                    b->built_eta == eta && b->built_cfl == cfl;
  if (!same) {
    drop_graph(b);
    mhd_status st = upload_params(b, s, scheme, eta);
    if (st != MHD_OK) return st;
    b->built_cons = s->cons;
    b->built_b = s->b;
    b->built_scheme = scheme;
    b->built_eta = eta;
    b->built_cfl = cfl;
    b->params_ok = true;
  }
  if (!b->use_graph) return enqueue_step(b, s, cfl, scheme, eta, b->stream);
  if (!b->graph_ok) {
    // capture on the private stream (capture is not allowed on the legacy default stream); the
    // graph is then launched on the caller's stream
    mhd_status st = bcuda(b, cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
    if (st != MHD_OK) return st;
    cudaGraph_t g;
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bcuda(b, e, "cudaStreamBeginCapture");
    st = enqueue_step(b, s, cfl, scheme, eta, b->cap);
    e = cudaStreamEndCapture(b->cap, &g);
    if (st != MHD_OK) {
      if (e == cudaSuccess) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return bcuda(b, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bcuda(b, e, "cudaGraphInstantiate");
    b->graph_ok = true;
  }
  return bcuda(b, cudaGraphLaunch(b->graph, b->stream), "cudaGraphLaunch");
}

mhd_status mhd_batch_last_dt(mhd_batch* b, double* dt) {
  if (!b || !dt) return MHD_ERR_ARG;
  unsigned long long h[8];
  cudaError_t e = cudaMemcpyAsync(dt, b->dt_dev, sizeof(double), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, b->counters, sizeof(h), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  mhd_status s = bcuda(b, e, "read dt");
  if (s != MHD_OK) return s;
  if (h[7]) return report_timeout(b);
  if (h[6]) return bfail(b, MHD_ERR_NONFINITE, "signal speed not finite: no step taken");
  return MHD_OK;
}

mhd_status mhd_batch_stats(mhd_batch* b, long long* s1, long long* s2) {
  if (!b) return MHD_ERR_ARG;
  unsigned long long h[8];
  cudaError_t e = cudaMemcpyAsync(h, b->counters, sizeof(h), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  mhd_status s = bcuda(b, e, "read counters");
  if (s != MHD_OK) return s;
  if (s1) *s1 = (long long)h[0];
  if (s2) *s2 = (long long)h[1];
  if (h[7]) return report_timeout(b);
  return MHD_OK;
}

mhd_status mhd_batch_phase_ms(mhd_batch* b, double* ms) {
  if (!b || !ms) return MHD_ERR_ARG;
  unsigned long long t[16];
  cudaError_t e = cudaMemcpyAsync(t, b->ptime, sizeof(t), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  mhd_status s = bcuda(b, e, "read phase stamps");
  if (s != MHD_OK) return s;
  for (int st = 0; st < 2; ++st)
    for (int j = 0; j < 6; ++j) {
      const unsigned long long a = t[8 * st + j], z = t[8 * st + j + 1];
      ms[6 * st + j] = (a && z && z >= a) ? (double)(z - a) * 1e-6 : 0.0;
    }
  return MHD_OK;
}

mhd_status mhd_batch_set_launches(mhd_batch* b, int launches_per_stage) {
  if (!b) return MHD_ERR_ARG;
  if (launches_per_stage != 1 && launches_per_stage != 3) return bfail(b, MHD_ERR_ARG, "launches per stage: 1 or 3");
  mhd_status s = bcuda(b, cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
  if (s != MHD_OK) return s;
  b->launches_per_stage = launches_per_stage;
  drop_graph(b);
  return MHD_OK;
}

mhd_status mhd_batch_tune(mhd_batch* b, const mhd_batch_state* s, double cfl, int scheme, double eta, int* seg_out,
                          int* order_out, int* bps_out, int* launches_out) {
  if (!b || !s || !s->cons || !s->b) return MHD_ERR_ARG;
  // the choice depends on the device, the scheme and the patches' sizes (not on their order or
  // state): a batch with the same histogram of patch sizes reuses an earlier choice untimed
  std::string key;
  {
    int dev = 0;
    cudaGetDevice(&dev);
    std::map<std::tuple<int, int, int>, int> hist;
    for (int p = 0; p < b->npatch; ++p) ++hist[std::make_tuple(b->dims[3 * p], b->dims[3 * p + 1], b->dims[3 * p + 2])];
    key = std::to_string(dev) + ":" + std::to_string(b->nsm) + ":" + std::to_string(scheme) + ":" +
          std::to_string(eta != 0.0 ? 1 : 0);
    for (const auto& kv : hist)
      key += ":" + std::to_string(std::get<0>(kv.first)) + "x" + std::to_string(std::get<1>(kv.first)) + "x" +
             std::to_string(std::get<2>(kv.first)) + "*" + std::to_string(kv.second);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      const int c_seg = it->second[0], c_order = it->second[1], c_bps = it->second[2], c_l = it->second[3];
      mhd_status st = mhd_batch_set_schedule(b, c_seg, c_order, c_bps, b->use_graph);
      if (st == MHD_OK) st = mhd_batch_set_launches(b, c_l);
      if (seg_out) *seg_out = c_seg;
      if (order_out) *order_out = c_order;
      if (bps_out) *bps_out = c_bps;
      if (launches_out) *launches_out = c_l;
      return st;
    }
  }
  // time one step per candidate on a scratch copy of the state (the caller's state is unchanged)
  double* cpy = nullptr;
  cudaError_t e = cudaMalloc(&cpy, 8 * b->ncell * sizeof(double));
  if (e != cudaSuccess) return bcuda(b, e, "cudaMalloc");
  mhd_batch_state t = {cpy, cpy + 5 * b->ncell};
  int per_sm[2] = {0, 0};  // CTAs per SM of the first launch: one launch per stage, three
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[0], mhd::stage_kernel(scheme & 0xf, (scheme >> 4) & 0xf, true),
                                                128, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[1], mhd::stage_kernel(scheme & 0xf, (scheme >> 4) & 0xf, false),
                                                128, 0);
  const int segs[] = {16, 32, 64, 128};
  float best = 1e30f;
  int bs = 64, bo = 1, bb = 0, bl = 3;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  mhd_status st = MHD_OK;
  const int saved_graph = b->use_graph;
  for (int form = 0; form < 2 && st == MHD_OK; ++form)
  for (int seg : segs)
    for (int order = 0; order < 2 && st == MHD_OK; ++order)
      for (int bps = 1; bps <= std::max(1, per_sm[form]) && st == MHD_OK; ++bps) {
        st = mhd_batch_set_schedule(b, seg, order, bps, 0);
        if (st == MHD_OK) st = mhd_batch_set_launches(b, form == 0 ? 1 : 3);
        if (st != MHD_OK) break;
        float ms = 0.f;
        for (int rep = 0; rep < 2 && st == MHD_OK; ++rep) {  // first run warms up
          cudaMemcpyAsync(cpy, s->cons, 5 * b->ncell * sizeof(double), cudaMemcpyDeviceToDevice, b->stream);
          cudaMemcpyAsync(cpy + 5 * b->ncell, s->b, 3 * b->ncell * sizeof(double), cudaMemcpyDeviceToDevice, b->stream);
          cudaEventRecord(e0, b->stream);
          st = mhd_batch_step(b, &t, cfl, scheme, eta);
          cudaEventRecord(e1, b->stream);
          cudaEventSynchronize(e1);
          cudaEventElapsedTime(&ms, e0, e1);
        }
        if (st == MHD_OK) {
          double dt;
          st = mhd_batch_last_dt(b, &dt);
        }
        if (st == MHD_OK && ms < best) {
          best = ms;
          bs = seg;
          bo = order;
          bb = bps;
          bl = form == 0 ? 1 : 3;
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->params_ok = false;  // parameters pointed at the copy
  cudaFree(cpy);
  if (st != MHD_OK) return st;
  st = mhd_batch_set_schedule(b, bs, bo, bb, saved_graph);
  if (st == MHD_OK) st = mhd_batch_set_launches(b, bl);
  if (st == MHD_OK) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = {bs, bo, bb, bl};
  }
  if (seg_out) *seg_out = bs;
  if (order_out) *order_out = bo;
  if (bps_out) *bps_out = bb;
  if (launches_out) *launches_out = bl;
  return st;
}

mhd_status mhd_batch_test_barrier(mhd_batch* b, int extra_blocks, long long spin_limit) {
  if (!b || extra_blocks < 0 || spin_limit < 1) return MHD_ERR_ARG;
  b->barrier_extra = extra_blocks;
  b->spin_limit = spin_limit;
  drop_graph(b);
  b->params_ok = false;
  return MHD_OK;
}

}  // extern "C"
