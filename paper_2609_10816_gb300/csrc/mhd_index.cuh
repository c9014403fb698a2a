// mhd_index.cuh -- periodic index arithmetic for the box kernels (integer pipe only).
#pragma once
#include "mhd_device.cuh"
#include "mhd_internal.cuh"

namespace mhd {

// linear index of X shifted by s (|s| < n[d]) cells along d, periodic
__device__ __forceinline__ long long shift(const Dev& D, long long X, int d, int s) {
  const unsigned st = (unsigned)D.stride[d];
  const int nd = D.n[d];
  const int cd = (int)(((unsigned long long)X / st) % (unsigned)nd);
  int cn = cd + s;
  if (cn >= nd) cn -= nd;
  if (cn < 0) cn += nd;
  return X + (long long)(cn - cd) * (long long)st;
}

// X shifted by any s along d (true modulo, for lines shorter than |s|)
__device__ __forceinline__ long long shift2(const Dev& D, long long X, int d, int s) {
  const unsigned st = (unsigned)D.stride[d];
  const int nd = D.n[d];
  const int cd = (int)(((unsigned long long)X / st) % (unsigned)nd);
  int cn = (cd + s) % nd;
  if (cn < 0) cn += nd;
  return X + (long long)(cn - cd) * (long long)st;
}

// Sweeps along `dir`: lines are indexed by the two other axes, the faster one first so that
// neighbouring threads touch neighbouring addresses when dir != 0; each line is cut into
// segments of `seg` points, one per thread.
__host__ __device__ __forceinline__ void sweep_axes(int dir, int& t1, int& t2) {
  t1 = dir == 0 ? 1 : 0;
  t2 = dir == 2 ? 1 : 2;
}

__host__ __device__ inline long long sweep_threads(const Dev& D, int dir, int seg) {
  int t1, t2;
  sweep_axes(dir, t1, t2);
  const long long nseg = (D.n[dir] + seg - 1) / seg;
  return (long long)D.n[t1] * D.n[t2] * nseg;
}

// segment number `tid` of the sweeps along dir (false past the last one)
__device__ __forceinline__ bool sweep_line_at(const Dev& D, int dir, int seg, long long tid, Line& ln, int& m0,
                                              int& m1) {
  int t1, t2;
  sweep_axes(dir, t1, t2);
  const int n1 = D.n[t1], n2 = D.n[t2], nd = D.n[dir];
  const int nseg = (nd + seg - 1) / seg;
  if (tid >= (long long)n1 * n2 * nseg) return false;
  const int i1 = (int)(tid % n1);
  const long long r = tid / n1;
  const int i2 = (int)(r % n2);
  const int s = (int)(r / n2);
  ln.base = (long long)i1 * D.stride[t1] + (long long)i2 * D.stride[t2];
  ln.stride = D.stride[dir];
  ln.n = nd;
  m0 = s * seg;
  m1 = min(nd, m0 + seg);
  return true;
}

__device__ __forceinline__ bool sweep_line(const Dev& D, int dir, int seg, Line& ln, int& m0, int& m1) {
  return sweep_line_at(D, dir, seg, (long long)blockIdx.x * blockDim.x + threadIdx.x, ln, m0, m1);
}

}  // namespace mhd
