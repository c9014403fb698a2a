// mhd_api.cu -- host side of the C ABI declared in include/mhd.h: context and scratch
// management, argument checks, and the launch sequence of one RK2 + FOFC step (Sec. 2.5).
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/mhd.h"
#include "mhd_device.cuh"
#include "mhd_internal.cuh"

struct mhd_ctx {
  mhd::Dev base;
  cudaStream_t stream;
  void* scratch;
  size_t scratch_bytes;
  double* U1;
  double* B1[3];
  double* dtbuf;  // device: dt, dt / h_d and an error flag of the last mhd_step_cfl
  int seg;
  std::string err;
  // profiling: launch counts per kernel class, and (when enabled) event pairs per launch
  long long launches[MHD_K_COUNT];
  bool prof;
  std::vector<cudaEvent_t> ev_pool;
  struct Rec { int cls; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  size_t ev_next;
  // adjoint scratch (allocated on the first mhd_step_adjoint call)
  double* adj;
  // mhd_step_cfl on small boxes: the launch sequence of a step recorded once as a CUDA graph (on
  // the private stream `cap`) and replayed while the arguments repeat
  struct StepKey {
    const double *cons, *b0, *b1, *b2;
    int scheme;
    double cfl, eta;
    bool operator==(const StepKey& o) const {
      return cons == o.cons && b0 == o.b0 && b1 == o.b1 && b2 == o.b2 && scheme == o.scheme && cfl == o.cfl &&
             eta == o.eta;
    }
  };
  cudaStream_t cap;
  cudaGraphExec_t graph;
  bool graph_ok;
  StepKey graph_key, prev_key;
  bool prev_ok;
  long long graph_launches[MHD_K_COUNT];
};

namespace {

thread_local std::string g_create_err;

mhd_status fail(mhd_ctx* c, mhd_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

mhd_status cuda_check(mhd_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return MHD_OK;
  return fail(c, MHD_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

struct Decoded {
  int recon, rs, emf, avg;
  bool fofc;
};

mhd_status decode(mhd_ctx* c, int scheme, Decoded& d) {
  d.recon = scheme & 0xf;
  d.rs = (scheme >> 4) & 0xf;
  d.emf = (scheme >> 8) & 0xf;
  d.avg = (scheme >> 12) & 0xf;
  d.fofc = !(scheme & MHD_FOFC_OFF);
  if (scheme & ~(0xffff | MHD_FOFC_OFF)) return fail(c, MHD_ERR_ARG, "unknown scheme bits");
  if (d.avg == 1) return fail(c, MHD_ERR_UNSUPPORTED, "B25b averaging is cited but not defined in the paper");
  if (d.recon > 4 || d.rs > 2 || d.emf > 2 || d.avg > 1) return fail(c, MHD_ERR_ARG, "scheme field out of range");
  return MHD_OK;
}

bool state_ok(const mhd_state* s) { return s && s->cons && s->b0 && s->b1 && s->b2; }

cudaEvent_t next_event(mhd_ctx* c) {
  if (c->ev_next == c->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    c->ev_pool.push_back(e);
  }
  return c->ev_pool[c->ev_next++];
}

// Brackets the launches of one kernel class with events when profiling is on.
struct Timed {
  mhd_ctx* c;
  int cls;
  cudaEvent_t a = nullptr;
  Timed(mhd_ctx* c_, int cls_, int nlaunch) : c(c_), cls(cls_) {
    c->launches[cls] += nlaunch;
    if (c->prof && (a = next_event(c))) cudaEventRecord(a, c->stream);
  }
  ~Timed() {
    if (!a) return;
    cudaEvent_t b = next_event(c);
    if (!b) return;
    cudaEventRecord(b, c->stream);
    c->recs.push_back({cls, a, b});
  }
};

// one RK stage: prim -> faces -> edges -> update -> flags -> flux correction. prim_given: the
// previous stage's flag pass wrote this stage's primitives (redo them only if it flagged cells).
// where the stage input's primitives come from: its own pass, the previous stage's flag pass
// (redone only for cells flux correction changed), or already in place (the CFL reduction)
enum PrimSource { PRIM_COMPUTE, PRIM_IF_FLAGGED, PRIM_READY };

void run_stage(mhd_ctx* c, const mhd::Dev& D, const Decoded& sc, PrimSource prim = PRIM_COMPUTE) {
  cudaStream_t st = c->stream;
  if (prim == PRIM_IF_FLAGGED) {
    Timed t(c, MHD_K_PRIM, 1);
    mhd::launch_prim_if_flagged(D, D.stage - 1, st);
  } else if (prim == PRIM_COMPUTE) {
    Timed t(c, MHD_K_PRIM, 1);
    mhd::launch_prim(D, st);
  }
  { Timed t(c, MHD_K_FACE, D.work ? 1 : 3); mhd::launch_faces(D, sc.recon, sc.rs, c->seg, st); }
  {
    // one launch per edge phase with work cursors (three without), B25a's six cell-to-face sweeps
    const int n = D.work ? 1 : 3;
    Timed t(c, MHD_K_EDGE_BT, sc.emf == mhd::EMF_B25A ? n + 6 : n);
    mhd::launch_edges_bt(D, sc.recon, c->seg, st);
  }
  { Timed t(c, MHD_K_EDGE_LR, D.work ? 1 : 3); mhd::launch_edges_lr(D, sc.recon, c->seg, st); }
  { Timed t(c, MHD_K_UPDATE, 1); mhd::launch_update(D, st); }
  { Timed t(c, MHD_K_FLAG, 1); mhd::launch_flag(D, st); }
  if (sc.fofc) { Timed t(c, MHD_K_FOFC, 3); mhd::launch_fofc(D, st); }
}

}  // namespace

void mhd::set_call_error(const char* msg) { g_create_err = msg; }

int mhd::resident_blocks(const void* fn, int threads) {
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, int>, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  const auto key = std::make_tuple(fn, threads, dev);
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int per_sm = 0, nsm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) nsm = 1;
  cache[key] = per_sm * nsm;
  return per_sm * nsm;
}

extern "C" {

const char* mhd_create_error(void) { return g_create_err.c_str(); }

const char* mhd_last_error(const mhd_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

mhd_status mhd_create(const mhd_config* cfg, void* cuda_stream, mhd_ctx** out) {
  g_create_err.clear();
  if (!out) { g_create_err = "out is NULL"; return MHD_ERR_ARG; }
  *out = nullptr;
  if (!cfg) { g_create_err = "cfg is NULL"; return MHD_ERR_ARG; }
  if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1 || !(cfg->dx > 0) || !(cfg->dy > 0) ||
      !(cfg->dz > 0) || !(cfg->gamma > 1.0)) {
    g_create_err = "invalid box: need n >= 1, dx > 0, gamma > 1";
    return MHD_ERR_ARG;
  }
  const long long N = (long long)cfg->nx * cfg->ny * cfg->nz;
  if (N > (1LL << 31) - 1) {
    g_create_err = "box larger than 2^31 - 1 cells";
    return MHD_ERR_ARG;
  }
  mhd_ctx* c = new mhd_ctx();
  c->stream = (cudaStream_t)cuda_stream;
  c->cap = nullptr;
  c->graph_ok = false;
  c->prev_ok = false;
  c->seg = 64;
  for (int k = 0; k < MHD_K_COUNT; ++k) c->launches[k] = 0;
  c->prof = false;
  c->ev_next = 0;
  c->adj = nullptr;
  mhd::Dev& D = c->base;
  std::memset(&D, 0, sizeof(D));
  D.n[0] = cfg->nx; D.n[1] = cfg->ny; D.n[2] = cfg->nz;
  D.N = N;
  D.stride[0] = 1; D.stride[1] = cfg->nx; D.stride[2] = (long long)cfg->nx * cfg->ny;
  D.h[0] = cfg->dx; D.h[1] = cfg->dy; D.h[2] = cfg->dz;
  for (int d = 0; d < 3; ++d) D.hinv[d] = 1.0 / D.h[d];
  D.gam = cfg->gamma;
  D.gm1inv = 1.0 / (cfg->gamma - 1.0);
  D.fofc_criteria = cfg->fofc_criteria ? cfg->fofc_criteria : 3;
  // scratch, in doubles per cell: U1 5, B1 3, P 8, F 15, Ap/Am/Us 9, Epart 12, E 3,
  // VL/VR 18, Xpart 24, EfL 6, EfB 6  -> 109; + flags (1 byte) + counters
  const size_t nd = 109;
  const size_t bytes = nd * sizeof(double) * (size_t)N + (size_t)N + 256 + 64 + 128;
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    g_create_err = std::string("cudaMalloc of scratch failed: ") + cudaGetErrorString(e);
    delete c;
    return MHD_ERR_CUDA;
  }
  c->scratch = p;
  c->scratch_bytes = bytes;
  double* q = (double*)p;
  auto take = [&](size_t k) { double* r = q; q += k * (size_t)N; return r; };
  c->U1 = take(5);
  for (int d = 0; d < 3; ++d) c->B1[d] = take(1);
  D.P = take(8);
  D.F = take(15);
  D.Ap = take(3);
  D.Am = take(3);
  D.Us = take(3);
  D.Epart = take(12);
  D.E = take(3);
  D.VL = take(9);
  D.VR = take(9);
  D.Xpart = take(24);
  D.EfL = take(6);
  D.EfB = take(6);
  D.counters = (unsigned long long*)q;  // 8 counters, then the sweeps' work cursors
  D.work = D.counters + 8;
  c->dtbuf = q + 8 + 16;                  // dt, dt / h_d and an error flag of mhd_step_cfl
  D.flag = (unsigned char*)(q + 8 + 16 + 8);
  e = cudaMemsetAsync(p, 0, bytes, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    g_create_err = std::string("scratch initialisation failed: ") + cudaGetErrorString(e);
    cudaFree(p);
    delete c;
    return MHD_ERR_CUDA;
  }
  *out = c;
  return MHD_OK;
}

void mhd_destroy(mhd_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  if (ctx->adj) cudaFree(ctx->adj);
  if (ctx->graph_ok) cudaGraphExecDestroy(ctx->graph);
  if (ctx->cap) cudaStreamDestroy(ctx->cap);
  cudaFree(ctx->scratch);
  delete ctx;
}

mhd_status mhd_profile(mhd_ctx* ctx, int enable) {
  if (!ctx) return MHD_ERR_ARG;
  mhd_status s = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
  if (s != MHD_OK) return s;
  ctx->prof = enable != 0;
  ctx->recs.clear();
  ctx->ev_next = 0;
  return MHD_OK;
}

mhd_status mhd_profile_read(mhd_ctx* ctx, double* total_ms, long long* launches, int reset) {
  if (!ctx) return MHD_ERR_ARG;
  mhd_status s = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
  if (s != MHD_OK) return s;
  if (total_ms) {
    for (int k = 0; k < MHD_K_COUNT; ++k) total_ms[k] = 0.0;
    for (const auto& r : ctx->recs) {
      float ms = 0.f;
      s = cuda_check(ctx, cudaEventElapsedTime(&ms, r.a, r.b), "cudaEventElapsedTime");
      if (s != MHD_OK) return s;
      total_ms[r.cls] += ms;
    }
  }
  if (launches)
    for (int k = 0; k < MHD_K_COUNT; ++k) launches[k] = ctx->launches[k];
  if (reset)
    for (int k = 0; k < MHD_K_COUNT; ++k) ctx->launches[k] = 0;
  return MHD_OK;
}

// The two stages and the copy-back of one step; D carries dt / h_d (by value or in device memory).
static mhd_status advance(mhd_ctx* ctx, const mhd_state* state, mhd::Dev D, const Decoded& sc, double eta,
                          bool prim_ready = false) {
  const long long N = D.N;
  mhd_status s;
  D.eta = eta;
  D.resistive = eta != 0.0;
  D.emf = sc.emf;
  if (!sc.fofc) D.fofc_criteria = 0;  // flags then count only non-finite cells
  D.U0 = state->cons;
  D.B0[0] = state->b0; D.B0[1] = state->b1; D.B0[2] = state->b2;
  cudaStream_t st = ctx->stream;
  s = cuda_check(ctx, cudaMemsetAsync(D.counters, 0, 4 * sizeof(unsigned long long), st), "cudaMemsetAsync");
  if (s != MHD_OK) return s;

  // stage 1: S^{n+1/2} = S^n + D^n  (Eq. rk1:update), written to scratch
  D.Uin = D.U0;
  for (int d = 0; d < 3; ++d) D.Bin[d] = D.B0[d];
  D.Uout = ctx->U1;
  for (int d = 0; d < 3; ++d) D.Bout[d] = ctx->B1[d];
  D.combine = 0;
  D.stage = 0;
  D.Pnext = D.P;  // stage 1's flag pass leaves the primitives of S^{n+1/2} for stage 2
  run_stage(ctx, D, sc, prim_ready ? PRIM_READY : PRIM_COMPUTE);

  // stage 2: S^{n+1} = S^n + D(F_rk), F_rk = (F^n + F^{n+1/2}) / 2  (Eq. rk2:update); the
  // update reads only S^n and the fluxes, so it may overwrite the stage-1 scratch in place.
  D.Uin = ctx->U1;
  for (int d = 0; d < 3; ++d) D.Bin[d] = ctx->B1[d];
  D.combine = 1;
  D.stage = 1;
  D.Pnext = nullptr;
  run_stage(ctx, D, sc, PRIM_IF_FLAGGED);

  s = cuda_check(ctx, cudaGetLastError(), "kernel launch");
  if (s != MHD_OK) return s;
  s = cuda_check(ctx, cudaMemcpyAsync(state->cons, ctx->U1, 5 * N * sizeof(double), cudaMemcpyDeviceToDevice, st),
                 "cudaMemcpyAsync");
  if (s != MHD_OK) return s;
  double* bout[3] = {state->b0, state->b1, state->b2};
  for (int d = 0; d < 3; ++d) {
    s = cuda_check(ctx, cudaMemcpyAsync(bout[d], ctx->B1[d], N * sizeof(double), cudaMemcpyDeviceToDevice, st),
                   "cudaMemcpyAsync");
    if (s != MHD_OK) return s;
  }
  return MHD_OK;
}

mhd_status mhd_step(mhd_ctx* ctx, const mhd_state* state, double dt, int scheme, double eta) {
  if (!ctx) return MHD_ERR_ARG;
  ctx->err.clear();
  if (!state_ok(state)) return fail(ctx, MHD_ERR_ARG, "state has a NULL array");
  if (!(dt > 0) || !(dt < 1e300)) return fail(ctx, MHD_ERR_ARG, "dt must be finite and > 0");
  if (!(eta >= 0) || !(eta < 1e300)) return fail(ctx, MHD_ERR_ARG, "eta must be finite and >= 0");
  Decoded sc;
  mhd_status s = decode(ctx, scheme, sc);
  if (s != MHD_OK) return s;
  mhd::Dev D = ctx->base;
  D.dt = dt;
  for (int d = 0; d < 3; ++d) D.dth[d] = dt * D.hinv[d];
  return advance(ctx, state, D, sc, eta);
}

}  // extern "C"

namespace {

// the launches of one mhd_step_cfl on ctx->stream: CFL reduction, dt, both stages
mhd_status enqueue_step_cfl(mhd_ctx* ctx, const mhd_state* state, double cfl, const Decoded& sc, double eta) {
  mhd::Dev D = ctx->base;
  cudaStream_t st = ctx->stream;
  mhd_status s = cuda_check(ctx, cudaMemsetAsync(D.counters + 2, 0, sizeof(unsigned long long), st),
                            "cudaMemsetAsync");
  if (s != MHD_OK) return s;
  mhd::Ptr3 B = {{state->b0, state->b1, state->b2}};
  const double hmin = std::fmin(D.h[0], std::fmin(D.h[1], D.h[2]));
  {
    Timed t(ctx, MHD_K_MAXSPEED, 2);  // the reduction (which also leaves S^n's primitives) and dt
    mhd::launch_maxspeed(D, state->cons, B, D.counters + 2, st, D.P);
    mhd::launch_set_dt(D.counters + 2, cfl, eta, hmin, D.hinv, ctx->dtbuf, st);
  }
  s = cuda_check(ctx, cudaGetLastError(), "kernel launch");
  if (s != MHD_OK) return s;
  D.dt = 0.0;
  D.dthp = ctx->dtbuf + 1;
  return advance(ctx, state, D, sc, eta, true);
}

void drop_step_graph(mhd_ctx* ctx) {
  if (ctx->graph_ok) cudaGraphExecDestroy(ctx->graph);
  ctx->graph_ok = false;
}

// Record one step's launches on the private stream as a graph (false, and nothing recorded, if
// any part of it fails: the caller then runs the step eagerly).
bool build_step_graph(mhd_ctx* ctx, const mhd_state* state, double cfl, const Decoded& sc, double eta,
                      const mhd_ctx::StepKey& key) {
  drop_step_graph(ctx);
  if (!ctx->cap && cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking) != cudaSuccess) {
    ctx->cap = nullptr;
    return false;
  }
  long long before[MHD_K_COUNT];
  std::memcpy(before, ctx->launches, sizeof(before));
  cudaStream_t user = ctx->stream;
  ctx->stream = ctx->cap;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal);
  mhd_status s = e == cudaSuccess ? enqueue_step_cfl(ctx, state, cfl, sc, eta) : MHD_ERR_CUDA;
  if (e == cudaSuccess) {
    const cudaError_t e2 = cudaStreamEndCapture(ctx->cap, &g);
    if (e2 != cudaSuccess) s = MHD_ERR_CUDA;
  }
  ctx->stream = user;
  // the launches one replay stands for; the recording itself launched nothing
  for (int k = 0; k < MHD_K_COUNT; ++k) ctx->graph_launches[k] = ctx->launches[k] - before[k];
  std::memcpy(ctx->launches, before, sizeof(before));
  bool ok = s == MHD_OK && g && cudaGraphInstantiate(&ctx->graph, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();  // a failed capture leaves nothing behind for the next launch to report
  ctx->err.clear();
  if (!ok) return false;
  ctx->graph_ok = true;
  ctx->graph_key = key;
  return true;
}

}  // namespace

extern "C" {

// Boxes of at most kGraphCells cells: the host's launch cost is a visible share of a step, so
// when mhd_step_cfl is called again with the same arguments (state arrays, scheme, cfl, eta), not
// while profiling or while the stream is being captured, the step's launch sequence is recorded
// once as a CUDA graph and replayed by one launch per call (the same kernels, parameters and
// results).
constexpr long long kGraphCells = 128LL * 128 * 128;

mhd_status mhd_step_cfl(mhd_ctx* ctx, const mhd_state* state, double cfl, int scheme, double eta) {
  if (!ctx) return MHD_ERR_ARG;
  ctx->err.clear();
  if (!state_ok(state)) return fail(ctx, MHD_ERR_ARG, "state has a NULL array");
  if (!(cfl > 0) || !(cfl < 1e300)) return fail(ctx, MHD_ERR_ARG, "cfl must be finite and > 0");
  if (!(eta >= 0) || !(eta < 1e300)) return fail(ctx, MHD_ERR_ARG, "eta must be finite and >= 0");
  Decoded sc;
  mhd_status s = decode(ctx, scheme, sc);
  if (s != MHD_OK) return s;
  const mhd_ctx::StepKey key = {state->cons, state->b0, state->b1, state->b2, scheme, cfl, eta};
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const bool capturing = cudaStreamIsCapturing(ctx->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone;
  if (ctx->base.N <= kGraphCells && !ctx->prof && !capturing) {
    const bool repeat = (ctx->graph_ok && ctx->graph_key == key) || (ctx->prev_ok && ctx->prev_key == key);
    ctx->prev_key = key;
    ctx->prev_ok = true;
    if (repeat && ((ctx->graph_ok && ctx->graph_key == key) || build_step_graph(ctx, state, cfl, sc, eta, key))) {
      for (int k = 0; k < MHD_K_COUNT; ++k) ctx->launches[k] += ctx->graph_launches[k];
      return cuda_check(ctx, cudaGraphLaunch(ctx->graph, ctx->stream), "cudaGraphLaunch");
    }
  }
  return enqueue_step_cfl(ctx, state, cfl, sc, eta);
}

mhd_status mhd_last_dt(mhd_ctx* ctx, double* dt_out) {
  if (!ctx) return MHD_ERR_ARG;
  ctx->err.clear();
  if (!dt_out) return fail(ctx, MHD_ERR_ARG, "NULL argument");
  double h[5] = {0, 0, 0, 0, 0};
  mhd_status s = cuda_check(ctx, cudaMemcpyAsync(h, ctx->dtbuf, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream),
                            "cudaMemcpyAsync");
  if (s != MHD_OK) return s;
  s = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
  if (s != MHD_OK) return s;
  *dt_out = h[0];
  if (h[4] != 0.0) return fail(ctx, MHD_ERR_NONFINITE, "signal speed is zero or not finite");
  return MHD_OK;
}

mhd_status mhd_stats(mhd_ctx* ctx, long long* s1, long long* s2) {
  if (!ctx) return MHD_ERR_ARG;
  unsigned long long h[2] = {0, 0};
  mhd_status s = cuda_check(ctx, cudaMemcpyAsync(h, ctx->base.counters, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream),
                            "cudaMemcpyAsync");
  if (s != MHD_OK) return s;
  s = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
  if (s != MHD_OK) return s;
  if (s1) *s1 = (long long)h[0];
  if (s2) *s2 = (long long)h[1];
  return MHD_OK;
}

static mhd_status read_counters(mhd_ctx* ctx, unsigned long long* h, int n) {
  mhd_status s = cuda_check(ctx, cudaMemcpyAsync(h, ctx->base.counters + 2, n * sizeof(unsigned long long),
                                                 cudaMemcpyDeviceToHost, ctx->stream), "cudaMemcpyAsync");
  if (s != MHD_OK) return s;
  return cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
}

mhd_status mhd_max_dt(mhd_ctx* ctx, const mhd_state* state, double cfl, double eta, double* dt_out) {
  if (!ctx) return MHD_ERR_ARG;
  ctx->err.clear();
  if (!state_ok(state) || !dt_out) return fail(ctx, MHD_ERR_ARG, "NULL argument");
  if (!(cfl > 0) || !(eta >= 0)) return fail(ctx, MHD_ERR_ARG, "need cfl > 0 and eta >= 0");
  const mhd::Dev& D = ctx->base;
  mhd_status s = cuda_check(ctx, cudaMemsetAsync(D.counters + 2, 0, sizeof(unsigned long long), ctx->stream),
                            "cudaMemsetAsync");
  if (s != MHD_OK) return s;
  mhd::Ptr3 B = {{state->b0, state->b1, state->b2}};
  {
    Timed t(ctx, MHD_K_MAXSPEED, 1);
    mhd::launch_maxspeed(D, state->cons, B, D.counters + 2, ctx->stream);
  }
  s = cuda_check(ctx, cudaGetLastError(), "kernel launch");
  if (s != MHD_OK) return s;
  unsigned long long h = 0;
  s = read_counters(ctx, &h, 1);
  if (s != MHD_OK) return s;
  double smax;
  std::memcpy(&smax, &h, sizeof(double));
  const double hmin = std::fmin(D.h[0], std::fmin(D.h[1], D.h[2]));
  const double sres = 2.0 * eta / hmin;
  if (sres > smax) smax = sres;
  if (!(smax > 0) || !(smax < 1e300)) return fail(ctx, MHD_ERR_NONFINITE, "signal speed is zero or not finite");
  *dt_out = cfl * hmin / smax;
  return MHD_OK;
}

mhd_status mhd_divb(mhd_ctx* ctx, const mhd_state* state, double* max_abs_divb, double* max_abs_b) {
  if (!ctx) return MHD_ERR_ARG;
  ctx->err.clear();
  if (!state_ok(state) || !max_abs_divb || !max_abs_b) return fail(ctx, MHD_ERR_ARG, "NULL argument");
  const mhd::Dev& D = ctx->base;
  mhd_status s = cuda_check(ctx, cudaMemsetAsync(D.counters + 2, 0, 2 * sizeof(unsigned long long), ctx->stream),
                            "cudaMemsetAsync");
  if (s != MHD_OK) return s;
  mhd::Ptr3 B = {{state->b0, state->b1, state->b2}};
  {
    Timed t(ctx, MHD_K_DIVB, 1);
    mhd::launch_divb(D, B, D.counters + 2, ctx->stream);
  }
  s = cuda_check(ctx, cudaGetLastError(), "kernel launch");
  if (s != MHD_OK) return s;
  unsigned long long h[2] = {0, 0};
  s = read_counters(ctx, h, 2);
  if (s != MHD_OK) return s;
  std::memcpy(max_abs_divb, &h[0], sizeof(double));
  std::memcpy(max_abs_b, &h[1], sizeof(double));
  return MHD_OK;
}

mhd_status mhd_step_adjoint(mhd_ctx* ctx, const mhd_state* state, const mhd_state* lam, double dt, int scheme,
                            double eta, double* dL_deta) {
  if (!ctx) return MHD_ERR_ARG;
  ctx->err.clear();
  if (!state_ok(state) || !state_ok(lam)) return fail(ctx, MHD_ERR_ARG, "state or adjoint has a NULL array");
  if (!(dt > 0) || !(dt < 1e300)) return fail(ctx, MHD_ERR_ARG, "dt must be finite and > 0");
  if (!(eta >= 0) || !(eta < 1e300)) return fail(ctx, MHD_ERR_ARG, "eta must be finite and >= 0");
  Decoded sc;
  mhd_status s = decode(ctx, scheme, sc);
  if (s != MHD_OK) return s;
  const long long N = ctx->base.N;
  cudaStream_t st = ctx->stream;
  // adjoint scratch: lF 15, lE 3, lAp/lAm/lUs 9, lEdge 24, lLR 42, lP 8, lU1 5, lB1 3, lU0 5,
  // lB0 3, lam2 8, the stage-1 input's P 8 and alpha+- / u* 9, the forward face states of both
  // stage inputs 2 x 42, and their reconstructed edge values 12 + 2 x 30 + 24, B25a's face EMF
  // values of the stage-1 input 12; for flux correction D^T lam and the stage-1 flux adjoint
  // 2 x 18, the stage-2 proposal 8 and the stage-1 flags (doubles per cell) + eta
  const size_t nd = 414;
  if (!ctx->adj) {
    s = cuda_check(ctx, cudaMalloc(&ctx->adj, (nd * N + (N + 7) / 8 + 8) * sizeof(double)),
                   "cudaMalloc of adjoint scratch");
    if (s != MHD_OK) { ctx->adj = nullptr; return s; }
  }
  double* q = ctx->adj;
  auto take = [&](long long k) { double* r = q; q += k * N; return r; };
  double* lF = take(15);
  double* lE = take(3);
  double* lAp = take(3);
  double* lAm = take(3);
  double* lUs = take(3);
  double* lEdge = take(60);  // Q26 uses 24, FS18 60, B25a 36 (+ 18 for its face and cell EMF adjoints)
  double* lLR = take(42);
  double* lP = take(8);
  double* lU1 = take(5);
  double* lB1 = take(3);
  double* lU0 = take(5);
  double* lB0 = take(3);
  double* lamU = take(5);
  double* lamB = take(3);
  double* P0 = take(8);
  double* Apm0 = take(9);
  double* LR0 = take(42);
  double* LR1 = take(42);
  double* Epart0 = take(12);
  double* EdgeC0 = take(30);  // Q26 uses 12, FS18 30
  double* EdgeC1 = take(30);
  double* Xpart0 = take(24);  // FS18 / B25a: stage 1's a-then-c corner partials
  double* Ef0 = take(12);     // B25a: stage 1's face EMF values (EfL, then EfB)
  double* gF = take(15);  // g = D^T lam
  double* gE = take(3);
  double* kF = take(15);  // k: the adjoint of the stage-1 fluxes and EMFs
  double* kE = take(3);
  double* U2 = take(8);   // the stage-2 proposal S^n + D((F1 + HO(S^{n+1/2})) / 2), for its flags
  double* lEta = q;
  unsigned char* flag1 = (unsigned char*)(q + 8);  // the flags after stage 1

  mhd::Dev D = ctx->base;
  D.dt = dt;
  for (int d = 0; d < 3; ++d) D.dth[d] = dt * D.hinv[d];
  D.eta = eta;
  // the resistive terms are linear in eta: their derivative in eta is needed even at eta = 0,
  // where they add exact zeros to the forward values
  D.resistive = 1;
  D.emf = sc.emf;
  if (!sc.fofc) D.fofc_criteria = 0;
  D.U0 = state->cons;
  D.B0[0] = state->b0; D.B0[1] = state->b1; D.B0[2] = state->b2;
  D.Uout = ctx->U1;
  for (int d = 0; d < 3; ++d) D.Bout[d] = ctx->B1[d];
  D.combine = 0;
  D.stage = 0;
  const double* lamb[3] = {lam->b0, lam->b1, lam->b2};
  cudaError_t e = cudaMemsetAsync(D.counters, 0, 4 * sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(lamU, lam->cons, 5 * N * sizeof(double), cudaMemcpyDeviceToDevice, st);
  for (int d = 0; d < 3 && e == cudaSuccess; ++d)
    e = cudaMemcpyAsync(lamB + d * N, lamb[d], N * sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(lEta, 0, sizeof(double), st);
  if ((s = cuda_check(ctx, e, "adjoint set-up")) != MHD_OK) return s;

  // forward stage 1 again: S^{n+1/2} into the context's stage scratch; its input's primitives,
  // alpha+- and u* go to buffers of their own, where the stage-1 adjoint reads them
  D.Uin = D.U0;
  for (int d = 0; d < 3; ++d) D.Bin[d] = D.B0[d];
  mhd::Dev D0 = D;
  D0.P = P0;
  D0.Ap = Apm0;
  D0.Am = Apm0 + 3 * N;
  D0.Us = Apm0 + 6 * N;
  D0.LR = LR0;  // the forward face and edge values, which the stage-1 adjoint reads
  D0.Epart = Epart0;
  D0.Xpart = Xpart0;
  D0.EfL = Ef0;
  D0.EfB = Ef0 + 6 * N;
  D0.EdgeC = EdgeC0;
  run_stage(ctx, D0, sc);
  // the stage-1 flags (none without flux correction: the flag pass then marks only cells that are
  // not finite, and the forward step corrects nothing)
  e = sc.fofc ? cudaMemcpyAsync(flag1, D.flag, N, cudaMemcpyDeviceToDevice, st) : cudaMemsetAsync(flag1, 0, N, st);
  if ((s = cuda_check(ctx, e, "flags")) != MHD_OK) return s;
  const unsigned char* flag2 = sc.fofc ? D.flag : flag1;

  auto adj_dev = [&](const mhd::Dev& Ds, double* lU, double* lB) {
    mhd::AdjDev A;
    A.D = Ds;
    A.lF = lF; A.lE = lE; A.lAp = lAp; A.lAm = lAm; A.lUs = lUs; A.lEdge = lEdge; A.lLR = lLR; A.lP = lP;
    A.lU = lU; A.lB = lB; A.lEta = lEta;
    // B25a: the face EMF adjoints, the cell EMF and its adjoint in lEdge's last 24 rows
    A.lEf = lEdge + 36 * N; A.eps = lEdge + 48 * N; A.leps = lEdge + 51 * N;
    return A;
  };
  auto recompute = [&](const mhd::Dev& Ds) {  // P, alpha+-, u*, face and edge values of the stage input
    mhd::launch_prim(Ds, st);
    mhd::launch_faces(Ds, sc.recon, sc.rs, ctx->seg, st);
    mhd::launch_edges_bt(Ds, sc.recon, ctx->seg, st);
    mhd::launch_edges_lr(Ds, sc.recon, ctx->seg, st);
  };
  auto zero = [&](double* p, long long k) { return cudaMemsetAsync(p, 0, k * N * sizeof(double), st); };

  // forward stage 2 again, up to its flags: P, alpha+-, u*, face and edge values of S^{n+1/2},
  // the fluxes (F1 + HO(S^{n+1/2})) / 2 and the proposal they give, whose invalid cells are the
  // stage-2 flags (the stage-1 fluxes F1 are still in the flux and EMF arrays)
  mhd::Dev D1 = D;
  D1.Uin = ctx->U1;
  for (int d = 0; d < 3; ++d) D1.Bin[d] = ctx->B1[d];
  D1.LR = LR1;
  D1.EdgeC = EdgeC1;
  {
    mhd::Dev D2 = D1;
    D2.combine = 1;
    D2.stage = 1;
    D2.Pnext = nullptr;
    D2.Uout = U2;
    for (int d = 0; d < 3; ++d) D2.Bout[d] = U2 + (5 + d) * N;
    recompute(D2);
    mhd::launch_update(D2, st);
    mhd::launch_flag(D2, st);
  }

  // stage 2 flux function at S^{n+1/2}: adjoint inputs (1 - M2) (D^T lam) / 2
  mhd::launch_adj_update(D, lamU, lamB, gF, gE, 1.0, 0.0, st);
  mhd::launch_adj_mask(D, flag2, gF, gE, lF, lE, 0.5, st);
  e = zero(lU1, 5);
  if (e == cudaSuccess) e = zero(lB1, 3);
  if (e == cudaSuccess) e = zero(lAp, 9);  // alpha+-, u* (accumulated)
  if (e == cudaSuccess) e = zero(lP, 8);   // primitives (accumulated)
  if ((s = cuda_check(ctx, e, "cudaMemsetAsync")) != MHD_OK) return s;
  mhd::launch_adj_flux(adj_dev(D1, lU1, lB1), sc.recon, sc.rs, st);

  // the stage-1 fluxes F1: k = (1 - M2) (D^T lam) / 2 + D^T lam_{n+1/2}; the high-order flux
  // function at S^n gets (1 - M1) k
  mhd::launch_adj_mask(D, flag2, gF, gE, kF, kE, 0.5, st);
  mhd::launch_adj_update(D, lU1, lB1, kF, kE, 1.0, 1.0, st);
  mhd::launch_adj_mask(D, flag1, kF, kE, lF, lE, 1.0, st);
  e = zero(lU0, 5);
  if (e == cudaSuccess) e = zero(lB0, 3);
  if (e == cudaSuccess) e = zero(lAp, 9);  // alpha+-, u* (accumulated)
  if (e == cudaSuccess) e = zero(lP, 8);   // primitives (accumulated)
  if ((s = cuda_check(ctx, e, "cudaMemsetAsync")) != MHD_OK) return s;
  mhd::launch_adj_flux(adj_dev(D0, lU0, lB0), sc.recon, sc.rs, st);
  // the first-order fluxes and EMFs of S^n on masked faces and edges get M2 (D^T lam) + M1 k
  // (the kernel returns at once when neither stage flagged a cell)
  if (sc.fofc) mhd::launch_adj_fo(adj_dev(D0, lU0, lB0), flag1, flag2, gF, gE, kF, kE, st);

  // lam_n = lam_{n+1} + lam_{n+1/2} + (stage-1 part), back into the caller's arrays
  mhd::launch_axpy3(5 * N, lamU, lU1, lU0, st);
  mhd::launch_axpy3(3 * N, lamB, lB1, lB0, st);
  e = cudaMemcpyAsync(lam->cons, lamU, 5 * N * sizeof(double), cudaMemcpyDeviceToDevice, st);
  double* lamb_out[3] = {lam->b0, lam->b1, lam->b2};
  for (int d = 0; d < 3 && e == cudaSuccess; ++d)
    e = cudaMemcpyAsync(lamb_out[d], lamB + d * N, N * sizeof(double), cudaMemcpyDeviceToDevice, st);
  if ((s = cuda_check(ctx, e, "adjoint write-back")) != MHD_OK) return s;
  if ((s = cuda_check(ctx, cudaGetLastError(), "kernel launch")) != MHD_OK) return s;
  if (dL_deta) {
    double h = 0.0;
    e = cudaMemcpyAsync(&h, lEta, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if ((s = cuda_check(ctx, e, "read d/deta")) != MHD_OK) return s;
    *dL_deta += h;
  }
  return MHD_OK;
}

mhd_status mhd_adjoint_check(mhd_ctx* ctx, long long n, int scheme, unsigned long long seed, double* max_rel_err) {
  if (!ctx) return MHD_ERR_ARG;
  ctx->err.clear();
  if (!max_rel_err || n < 1 || n > (1LL << 34)) return fail(ctx, MHD_ERR_ARG, "need 1 <= n <= 2^34 and an output");
  Decoded sc;
  mhd_status s = decode(ctx, scheme, sc);
  if (s != MHD_OK) return s;
  const mhd::Dev& D = ctx->base;
  // 7 results: the scratch's work cursors serve (they are rezeroed before every sweep)
  unsigned long long* out = D.work;
  s = cuda_check(ctx, cudaMemsetAsync(out, 0, 7 * sizeof(unsigned long long), ctx->stream), "cudaMemsetAsync");
  if (s != MHD_OK) return s;
  mhd::launch_vjp_check(n, seed, D.gam, sc.rs, out, ctx->stream);
  s = cuda_check(ctx, cudaGetLastError(), "kernel launch");
  if (s != MHD_OK) return s;
  unsigned long long h[7];
  s = cuda_check(ctx, cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream), "cudaMemcpyAsync");
  if (s == MHD_OK) s = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
  if (s != MHD_OK) return s;
  std::memcpy(max_rel_err, h, sizeof(h));
  return MHD_OK;
}

mhd_status mhd_math_check(mhd_ctx* ctx, long long n, double* max_rel_err) {
  if (!ctx) return MHD_ERR_ARG;
  ctx->err.clear();
  if (!max_rel_err || n < 1 || n > (1LL << 40)) return fail(ctx, MHD_ERR_ARG, "need 1 <= n <= 2^40 and an output");
  const mhd::Dev& D = ctx->base;
  // 7 results: the scratch's work cursors serve (they are rezeroed before every sweep)
  unsigned long long* out = D.work;
  mhd_status s = cuda_check(ctx, cudaMemsetAsync(out, 0, 7 * sizeof(unsigned long long), ctx->stream),
                            "cudaMemsetAsync");
  if (s != MHD_OK) return s;
  mhd::launch_math_check(n, out, ctx->stream);
  s = cuda_check(ctx, cudaGetLastError(), "kernel launch");
  if (s != MHD_OK) return s;
  unsigned long long h[7] = {0, 0, 0, 0, 0, 0, 0};
  s = cuda_check(ctx, cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream), "cudaMemcpyAsync");
  if (s == MHD_OK) s = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
  if (s != MHD_OK) return s;
  for (int k = 0; k < 3; ++k) std::memcpy(&max_rel_err[k], &h[k], sizeof(double));
  for (int k = 3; k < 7; ++k) max_rel_err[k] = (double)h[k];
  return MHD_OK;
}

}  // extern "C"
