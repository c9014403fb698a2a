// mhd_noalloc.cu -- mhd_step_noalloc: one step of a small periodic box that allocates nothing.
//
// Some callers cannot let a library allocate device memory: applications whose own memory
// manager owns every byte of the device (a pool that cannot have a library allocate beside it),
// and tight loops that cannot afford cudaMalloc's implicit device synchronisation. For them this entry point runs the same kernels as mhd_step, with all of the
// step's scratch in one fixed device array defined below. The array has a fixed size, so the
// entry point takes boxes of at most MHD_NOALLOC_MAX_CELLS cells; it exists, and occupies
// device memory, on every GPU that loads the library, until the process exits.
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/mhd.h"
#include "mhd_device.cuh"
#include "mhd_internal.cuh"

namespace {

// scratch per cell, in doubles: stage-1 state 8, prim 8, fluxes 15, alpha+- and u* 9,
// edge partials 12, EMFs 3  -> 55; plus 8 counters and one flag byte per cell
constexpr long long kMaxCells = MHD_NOALLOC_MAX_CELLS;
constexpr long long kDoublesPerCell = 55;
constexpr long long kHeadDoubles = 8 + (kMaxCells + 7) / 8;  // counters, then flags
constexpr long long kScratchDoubles = kHeadDoubles + kDoublesPerCell * kMaxCells;

}  // namespace

// The fixed scratch of mhd_step_noalloc (one copy per device). Host code must not pass this
// symbol to a kernel: on the host it names a stand-in, not device memory. Its device address
// comes from cudaGetSymbolAddress, taken once per device below.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (looked up once per device).
mhd_status scratch_address(void** out, std::string& err) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return MHD_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    err = "device index beyond the supported range";
    return MHD_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      err = std::string("cudaGetSymbolAddress of the fixed scratch: ") + cudaGetErrorString(e);
      return MHD_ERR_CUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return MHD_OK;
}

mhd_status fail(mhd_status s, const std::string& msg) {
  mhd::set_call_error(msg.c_str());
  return s;
}

}  // namespace

extern "C" mhd_status mhd_step_noalloc(const mhd_config* cfg, const mhd_state* state, double dt,
                                       int scheme, double eta, void* cuda_stream) {
  mhd::set_call_error("");
  if (!cfg || !state || !state->cons || !state->b0 || !state->b1 || !state->b2)
    return fail(MHD_ERR_ARG, "NULL argument");
  if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1 || !(cfg->dx > 0) || !(cfg->dy > 0) || !(cfg->dz > 0) ||
      !(cfg->gamma > 1.0))
    return fail(MHD_ERR_ARG, "invalid box: need n >= 1, dx > 0, gamma > 1");
  const long long N = (long long)cfg->nx * cfg->ny * cfg->nz;
  if (N > kMaxCells)
    return fail(MHD_ERR_ARG, "box of " + std::to_string(N) + " cells exceeds the fixed scratch of " +
                                 std::to_string(kMaxCells) + " cells (MHD_NOALLOC_MAX_CELLS); use mhd_step");
  if (!(dt > 0) || !(dt < 1e300)) return fail(MHD_ERR_ARG, "dt must be finite and > 0");
  if (!(eta >= 0) || !(eta < 1e300)) return fail(MHD_ERR_ARG, "eta must be finite and >= 0");
  if (scheme & ~(0xffff | MHD_FOFC_OFF)) return fail(MHD_ERR_ARG, "unknown scheme bits");
  const int recon = scheme & 0xf, rs = (scheme >> 4) & 0xf, emf = (scheme >> 8) & 0xf, avg = (scheme >> 12) & 0xf;
  const bool fofc = !(scheme & MHD_FOFC_OFF);
  if (avg == 1) return fail(MHD_ERR_UNSUPPORTED, "B25b averaging is cited but not defined in the paper");
  if (recon > 4 || rs > 2 || emf > 2 || avg > 1) return fail(MHD_ERR_ARG, "scheme field out of range");
  if (emf != mhd::EMF_Q26) return fail(MHD_ERR_UNSUPPORTED, "only the Q26 EMF compute runs without allocation");

  std::string err;
  void* base = nullptr;
  mhd_status s = scratch_address(&base, err);
  if (s != MHD_OK) return fail(s, err);
  cudaStream_t st = (cudaStream_t)cuda_stream;

  mhd::Dev D;
  std::memset(&D, 0, sizeof(D));
  D.n[0] = cfg->nx; D.n[1] = cfg->ny; D.n[2] = cfg->nz;
  D.N = N;
  D.stride[0] = 1; D.stride[1] = cfg->nx; D.stride[2] = (long long)cfg->nx * cfg->ny;
  D.h[0] = cfg->dx; D.h[1] = cfg->dy; D.h[2] = cfg->dz;
  for (int d = 0; d < 3; ++d) D.hinv[d] = 1.0 / D.h[d];
  D.gam = cfg->gamma;
  D.gm1inv = 1.0 / (cfg->gamma - 1.0);
  D.fofc_criteria = fofc ? (cfg->fofc_criteria ? cfg->fofc_criteria : 3) : 0;
  D.dt = dt;
  for (int d = 0; d < 3; ++d) D.dth[d] = dt * D.hinv[d];
  D.eta = eta;
  D.resistive = eta != 0.0;
  D.emf = emf;
  // carve the fixed array: counters, flags, then N-sized slices
  double* q = (double*)base;
  D.counters = (unsigned long long*)q;
  D.flag = (unsigned char*)(q + 8);
  q += kHeadDoubles;
  auto take = [&](long long k) { double* r = q; q += k * N; return r; };
  double* U1 = take(5);
  double* B1[3] = {take(1), take(1), take(1)};
  D.P = take(8);
  D.F = take(15);
  D.Ap = take(3);
  D.Am = take(3);
  D.Us = take(3);
  D.Epart = take(12);
  D.E = take(3);
  D.U0 = state->cons;
  D.B0[0] = state->b0; D.B0[1] = state->b1; D.B0[2] = state->b2;

  // the array keeps the previous call's contents: the flagged-cell counters must start at zero
  // (every other slice is fully written before it is read)
  cudaError_t e = cudaMemsetAsync(D.counters, 0, 4 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return fail(MHD_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));

  const int seg = 64;
  for (int stage = 0; stage < 2; ++stage) {
    if (stage == 0) {
      D.Uin = D.U0;
      for (int d = 0; d < 3; ++d) D.Bin[d] = D.B0[d];
    } else {
      D.Uin = U1;
      for (int d = 0; d < 3; ++d) D.Bin[d] = B1[d];
    }
    D.Uout = U1;
    for (int d = 0; d < 3; ++d) D.Bout[d] = B1[d];
    D.combine = stage;
    D.stage = stage;
    mhd::launch_prim(D, st);
    for (int dir = 0; dir < 3; ++dir) mhd::launch_face(D, dir, recon, rs, seg, st);
    mhd::launch_edges_bt(D, recon, seg, st);
    mhd::launch_edges_lr(D, recon, seg, st);
    mhd::launch_update(D, st);
    mhd::launch_flag(D, st);
    if (fofc) mhd::launch_fofc(D, st);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(MHD_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  e = cudaMemcpyAsync(state->cons, U1, 5 * N * sizeof(double), cudaMemcpyDeviceToDevice, st);
  double* bout[3] = {state->b0, state->b1, state->b2};
  for (int d = 0; d < 3 && e == cudaSuccess; ++d)
    e = cudaMemcpyAsync(bout[d], B1[d], N * sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return fail(MHD_ERR_CUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
  return MHD_OK;
}
