// mhd_probe.cu -- mhd_fp64_rate: the sustained rate of the FP64 instructions that bound the
// step's kernels, measured on the current GPU, and what a binary64 multiply on the integer pipe
// adds beside them.
//
// Every kernel of the step is bound by the FP64 pipe, so the roofline's denominator is that
// pipe's throughput. The probe runs independent chains of one instruction kind (eight chains per
// thread, enough to hide the pipe's latency) over a grid of 8 blocks of 256 threads per SM and
// times them with CUDA events on the context's stream. The chains stay bounded (x <- a x + b with
// 0 < a < 1), and their sum is stored so that nothing is optimised away. Kinds 4-6 run chains of
// the integer-pipe multiply (mhd_softmul.cuh), alone and mixed with DFMA chains, at the probe's
// occupancy and at the face sweep's (2 blocks of 128 threads per SM). Kinds 7 and 8 run the DFMA
// chains on 16 and 8 lanes of every warp (the others exit at once): whether the pipe's throughput
// in lane operations falls with the active lanes tells what a divergent branch of FP64 work costs.
#include <cstring>

#include "../../include/mhd.h"
#include "mhd_internal.cuh"
#include "mhd_softmul.cuh"

namespace mhd {

constexpr int kChains = 8;

// KIND 0-3: kChains chains of DFMA, DADD, DMUL or FP32 FFMA; KIND 4: NI chains of the
// integer-pipe multiply and NF chains of DFMA; KIND 5: kChains chains of DFMA on the first NF
// lanes of each warp
template <int KIND, int NF = 0, int NI = 0>
__global__ void __launch_bounds__(256) k_rate(long long iters, double a, double b, double* out) {
  if (KIND == 5 && (int)(threadIdx.x & 31) >= NF) return;
  double x[kChains], z[NI > 0 ? NI : 1];
  float y[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    y[c] = (float)x[c];
  }
#pragma unroll
  for (int c = 0; c < NI; ++c) z[c] = 1.0 + 1e-3 * (threadIdx.x + 3 * c);
  const float af = (float)a, bf = (float)b;
  for (long long i = 0; i < iters; ++i) {
    if constexpr (KIND == 4) {
#pragma unroll
      for (int c = 0; c < NF; ++c) x[c] = fma(x[c], a, b);
#pragma unroll
      for (int c = 0; c < NI; ++c) z[c] = mul_int(z[c], a);
    } else {
#pragma unroll
      for (int c = 0; c < kChains; ++c) {
        if (KIND == 0 || KIND == 5) x[c] = fma(x[c], a, b);  // DFMA
        else if (KIND == 1) x[c] = x[c] + b;          // DADD
        else if (KIND == 2) x[c] = x[c] * a;          // DMUL
        else y[c] = fmaf(y[c], af, bf);               // FFMA (FP32, for comparison)
      }
    }
  }
  double s = 0.0;
  if constexpr (KIND == 4) {
#pragma unroll
    for (int c = 0; c < NF; ++c) s += x[c];
#pragma unroll
    for (int c = 0; c < NI; ++c) s += z[c];
  } else {
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += KIND == 3 ? (double)y[c] : x[c];
  }
  if (s == 12345.678) out[0] = s;  // practically never true; keeps the chains live
}

}  // namespace mhd

extern "C" mhd_status mhd_fp64_rate(int kind, long long iters, void* cuda_stream, double* ops_per_s) {
  if (kind < 0 || kind > 8 || iters < 1 || iters > (1LL << 30) || !ops_per_s) return MHD_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess)
    return MHD_ERR_CUDA;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double)) != cudaSuccess) return MHD_ERR_CUDA;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // kind 6 runs at the face sweep's occupancy, the others at 8 blocks of 256 threads per SM
  const int threads = kind == 6 ? 128 : 256;
  const unsigned grid = (unsigned)((kind == 6 ? 2 : 8) * nsm);
  // chains per thread (every chain retires one operation per iteration)
  const int chains = mhd::kChains;
  // a < 1 keeps the multiply chains bounded; the add chains grow by b per step
  const double a = 0.9999999, b = 1e-9;
  auto launch = [&](long long n) {
    switch (kind) {
      case 0: mhd::k_rate<0><<<grid, threads, 0, st>>>(n, a, b, out); break;
      case 1: mhd::k_rate<1><<<grid, threads, 0, st>>>(n, a, b, out); break;
      case 2: mhd::k_rate<2><<<grid, threads, 0, st>>>(n, a, b, out); break;
      case 3: mhd::k_rate<3><<<grid, threads, 0, st>>>(n, a, b, out); break;
      case 4: mhd::k_rate<4, 0, 8><<<grid, threads, 0, st>>>(n, a, b, out); break;
      case 7: mhd::k_rate<5, 16><<<grid, threads, 0, st>>>(n, a, b, out); break;
      case 8: mhd::k_rate<5, 8><<<grid, threads, 0, st>>>(n, a, b, out); break;
      default: mhd::k_rate<4, 4, 4><<<grid, threads, 0, st>>>(n, a, b, out); break;
    }
  };
  launch(iters / 8 + 1);  // warm-up
  cudaEventRecord(e0, st);
  launch(iters);
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess || !(ms > 0.f)) return MHD_ERR_CUDA;
  // operations of the active lanes only
  const double lanes = kind == 7 ? 0.5 : (kind == 8 ? 0.25 : 1.0);
  *ops_per_s = (double)grid * (double)threads * lanes * (double)chains * (double)iters / (ms * 1e-3);
  return MHD_OK;
}
