// mhd_index.cuh -- periodic index arithmetic for the box kernels (integer pipe only).
#pragma once
#include "mhd_device.cuh"
#include "mhd_internal.cuh"

namespace mhd {

// linear index of X shifted by s (|s| < n[d]) cells along d, periodic. A box holds fewer than
// 2^31 cells (checked when it is created), so the index arithmetic is 32-bit.
__device__ __forceinline__ long long shift(const Dev& D, long long X, int d, int s) {
  const unsigned st = (unsigned)D.stride[d];
  const int nd = D.n[d];
  const int cd = (int)(((unsigned)X / st) % (unsigned)nd);
  int cn = cd + s;
  if (cn >= nd) cn -= nd;
  if (cn < 0) cn += nd;
  return X + (long long)(cn - cd) * (long long)st;
}

// X shifted by any s along d (true modulo, for lines shorter than |s|)
__device__ __forceinline__ long long shift2(const Dev& D, long long X, int d, int s) {
  const unsigned st = (unsigned)D.stride[d];
  const int nd = D.n[d];
  const int cd = (int)(((unsigned)X / st) % (unsigned)nd);
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

// segment number `tid` of the sweeps along dir (false past the last one). Segments are numbered
// line by line, the faster line axis first, so that neighbouring threads walk neighbouring lines;
// with seg_fastest the segments of one line take consecutive numbers instead, so that
// neighbouring threads walk neighbouring stretches of the same line (for sweeps along x, whose
// neighbouring lines lie nx apart: one thread per line would stream a separate cache line per
// thread and array). With `tiled` (and the two line axes multiples of 8 and 4), each 32 threads
// from a multiple of 32 walk an 8 x 4 patch of lines instead of a row of 32: the faces a warp
// solves together then lie within 8 cells of each other, not 32, and fall more often in the
// same branch of the solver.
__device__ __forceinline__ bool sweep_line_at(const Dev& D, int dir, int seg, long long tid, Line& ln, int& m0,
                                              int& m1, bool seg_fastest = false, bool tiled = false) {
  int t1, t2;
  sweep_axes(dir, t1, t2);
  const int n1 = D.n[t1], n2 = D.n[t2], nd = D.n[dir];
  const int nseg = (nd + seg - 1) / seg;
  if (tid >= (long long)n1 * n2 * nseg) return false;
  int i1, i2, s;
  if (tiled && !seg_fastest && (n1 & 7) == 0 && (n2 & 3) == 0) {
    const long long per = (long long)n1 * n2;  // lines: a multiple of 32
    s = (int)(tid / per);
    const long long r = tid - (long long)s * per;
    const int w = (int)(r >> 5), l = (int)(r & 31), p1 = n1 >> 3;
    i1 = (w % p1) * 8 + (l & 7);
    i2 = (w / p1) * 4 + (l >> 3);
  } else if (seg_fastest) {
    s = (int)(tid % nseg);
    const long long r = tid / nseg;
    i1 = (int)(r % n1);
    i2 = (int)(r / n1);
  } else {
    i1 = (int)(tid % n1);
    const long long r = tid / n1;
    i2 = (int)(r % n2);
    s = (int)(r / n2);
  }
  ln.base = (long long)i1 * D.stride[t1] + (long long)i2 * D.stride[t2];
  ln.stride = D.stride[dir];
  ln.n = nd;
  m0 = s * seg;
  m1 = min(nd, m0 + seg);
  return true;
}

// cell of thread t of a per-cell kernel, with each 32 threads from a multiple of 32 on an 8 x 4
// patch of an x-y plane (when nx and ny are multiples of 8 and 4; else cell t), so that a warp's
// cells lie within 8 cells of each other
__device__ __forceinline__ long long tiled_cell(const Dev& D, long long t) {
  if ((D.n[0] & 7) || (D.n[1] & 3)) return t;
  const long long per = (long long)D.n[0] * D.n[1];
  const long long z = t / per;
  const long long r = t - z * per;
  const int w = (int)(r >> 5), l = (int)(r & 31), p = D.n[0] >> 3;
  const int x = (w % p) * 8 + (l & 7), y = (w / p) * 4 + (l >> 3);
  return z * per + (long long)y * D.n[0] + x;
}

__device__ __forceinline__ bool sweep_line(const Dev& D, int dir, int seg, Line& ln, int& m0, int& m1,
                                           bool seg_fastest = false) {
  return sweep_line_at(D, dir, seg, (long long)blockIdx.x * blockDim.x + threadIdx.x, ln, m0, m1, seg_fastest);
}

// Dynamic schedule of a sweep: a persistent grid whose warps each take the next 32 segments of the
// work list from a cursor in device memory until the list is exhausted, so that no SM idles while
// others finish a long tail (segments differ in cost through the Riemann-fan and limiter branches).
// Calls body(segment index) for every segment exactly once; lanes past the end skip the call.
template <class Body>
__device__ __forceinline__ void for_each_segment(unsigned long long* cursor, long long total, Body body) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    long long base = 0;
    if (lane == 0) base = (long long)atomicAdd(cursor, 32ull);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= total) return;
    if (base + lane < total) body(base + lane);
  }
}

// Segment length of a dynamically scheduled sweep: the requested length, halved (down to 4) until
// the sweep has at least two segments per resident thread, so that small boxes still fill the GPU
// (a shorter segment costs one more window start-up, about two points of reconstruction).
__host__ __device__ inline int fill_seg(const Dev& D, int dir, int seg, long long resident_threads) {
  while (seg > 4 && sweep_threads(D, dir, seg) < 2 * resident_threads) seg = (seg + 1) / 2;
  return seg;
}

// Segment length and numbering of the edge sweeps along dir: along x, a warp takes whole lines
// (segments of about nx/32 points, 4 to 16, numbered along the line); along y and z the given
// segment length with one line per thread.
__host__ __device__ inline int edge_sweep_seg(const Dev& D, int dir, int seg) {
  if (dir != 0) return seg;
  const int s = (D.n[0] + 31) / 32;
  return s < 4 ? 4 : (s > 16 ? 16 : s);
}

}  // namespace mhd
