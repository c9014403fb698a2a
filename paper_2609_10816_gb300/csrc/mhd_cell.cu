// mhd_cell.cu -- per-cell kernels: conserved -> primitive (Sec. 2.2), the update increments
// (Eqs. rk:increment-state, rk:increment-bfield), the validity flags and first-order flux
// correction (Sec. 2.5), and the CFL and divergence reductions (Sec. 2.4, Sec. 2.1).
#include <algorithm>

#include "mhd_cell.cuh"
#include "mhd_softmul.cuh"

namespace mhd {

__global__ void __launch_bounds__(256) k_prim(Dev D) {
  const long long X = cell_id();
  if (X < D.N) prim_cell(D, X);
}
// the primitives of a stage input that the previous stage's flag pass wrote, redone only when
// flux correction changed that state
__global__ void __launch_bounds__(256) k_prim_if_flagged(Dev D, int prev_stage) {
  if (D.counters[prev_stage] == 0) return;
  const long long X = cell_id();
  if (X < D.N) prim_cell(D, X);
}
__global__ void __launch_bounds__(256) k_update(Dev D) {
  const long long X = cell_id();
  if (X < D.N) update_cell(D, X);
}
__global__ void __launch_bounds__(256) k_flag(Dev D) {
  const long long X = cell_id();
  const bool f = X < D.N ? flag_cell(D, X) : false;
  count_flags(D, f);
}
// First-order fix-up passes: grid-stride loops over a grid of two waves, so that a stage with
// no flagged cell (the usual case) costs a few microseconds of early exits
__global__ void __launch_bounds__(128) k_fo_faces(Dev D) {
  if (D.counters[D.stage] == 0) return;
  for (long long X = cell_id(); X < D.N; X += (long long)gridDim.x * blockDim.x) fo_faces_cell(D, X);
}
__global__ void __launch_bounds__(128) k_fo_edges(Dev D) {
  if (D.counters[D.stage] == 0) return;
  for (long long X = cell_id(); X < D.N; X += (long long)gridDim.x * blockDim.x) fo_edges_cell(D, X);
}
__global__ void __launch_bounds__(128) k_fo_recompute(Dev D) {
  if (D.counters[D.stage] == 0) return;
  for (long long X = cell_id(); X < D.N; X += (long long)gridDim.x * blockDim.x) fo_recompute_cell(D, X);
}

// dt = cfl hmin / max(smax, 2 eta / hmin) (Eq. resistivity:cfl), the operations of mhd_max_dt
__global__ void k_set_dt(const unsigned long long* smax_bits, double cfl, double eta, double hmin, double hx,
                         double hy, double hz, double* out) {
  double smax = dfrom((long long)*smax_bits);
  const double sres = 2.0 * eta / hmin;
  if (sres > smax) smax = sres;
  double dt = 0.0, bad = 1.0;
  if (smax > 0.0 && smax < 1e300) {
    dt = cfl * hmin / smax;
    bad = 0.0;
  }
  out[0] = dt;
  out[1] = dt * hx;
  out[2] = dt * hy;
  out[3] = dt * hz;
  out[4] = bad;
}

// ---- reductions -----------------------------------------------------------------------------
__device__ __forceinline__ void block_max_atomic(double v, unsigned long long* out) {
  // v >= 0: the bit pattern orders like the value
  unsigned long long b = (unsigned long long)dbits(v);
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, b, o);
    b = t > b ? t : b;
  }
  __shared__ unsigned long long sm[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sm[wid] = b;
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    b = lane < nw ? sm[lane] : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long t = __shfl_xor_sync(0xffffffffu, b, o);
      b = t > b ? t : b;
    }
    if (lane == 0) atomicMax(out, b);
  }
  __syncthreads();  // sm[] may be reused by a following call
}

// max over cells of the CFL signal speed (cfl_speed_max): a grid-stride loop whose warps share
// their running maximum after every pass, so that most cells are settled by the bound check
__global__ void __launch_bounds__(256) k_maxspeed(Dev D, const double* U, Ptr3 Bp,
                                                  unsigned long long* out, double* Pout) {
  const long long nth = (long long)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (long long base = cell_id() - lane; base < D.N; base += nth) {  // uniform over the warp
    if (base + lane < D.N) s = cfl_speed_max(D, U, Bp.p, base + lane, s, Pout);
    unsigned long long b = (unsigned long long)dbits(s);
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long t = __shfl_xor_sync(0xffffffffu, b, o);
      b = t > b ? t : b;
    }
    s = __longlong_as_double((long long)b);
  }
  block_max_atomic(s, out);
}

// max over cells of |div b| and over faces of |b|
__global__ void __launch_bounds__(256) k_divb(Dev D, Ptr3 Bp, unsigned long long* out) {
  const long long X = cell_id();
  double dv = 0.0, mb = 0.0;
  if (X < D.N) {
    double acc = 0.0;
    for (int d = 0; d < 3; ++d) {
      const double lo = Bp.p[d][X], hi = Bp.p[d][shift(D, X, d, 1)];
      acc += (hi - lo) * D.hinv[d];
      mb = pmax(mb, vabs(lo));
    }
    dv = vabs(acc);
  }
  block_max_atomic(dv, out);
  block_max_atomic(mb, out + 1);
}

// relative error of rcp / rsqrt_ / sqrt_ against IEEE division and sqrt on hashed inputs
__global__ void __launch_bounds__(256) k_math_check(long long n, unsigned long long* out) {
  const long long i = cell_id();
  double er = 0.0, es = 0.0, eq = 0.0;
  if (i < n) {
    unsigned long long z = (unsigned long long)i * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    z ^= z >> 31;
    z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 29;
    const long long mant = (long long)(z & 0x000fffffffffffffull);
    const long long ex = 1023 - 40 + (long long)((z >> 52) % 81);
    const double x = dfrom((ex << 52) | mant);
    const double r0 = 1.0 / x, s0 = sqrt(x), q0 = 1.0 / s0;
    er = vabs(rcp(x) - r0) / r0;
    es = vabs(rsqrt_(x) - q0) / q0;
    eq = vabs(sqrt_(x) - s0) / s0;
  }
  block_max_atomic(er, out);
  block_max_atomic(es, out + 1);
  block_max_atomic(eq, out + 2);
  // exactness of the integer-pipe halving and quadrupling against the FP64 multiplies, on raw bit
  // patterns (every eighth with its exponent forced into the subnormal / smallest / largest
  // binades, where the integer paths branch)
  if (i < n) {
    unsigned long long z = (unsigned long long)(i + n) * 0xD1B54A32D192ED03ull + 0x8CB92BA72F3D8DD7ull;
    z ^= z >> 33;
    z *= 0xFF51AFD7ED558CCDull;
    z ^= z >> 29;
    long long b = (long long)z;
    if ((z & 7) == 0) {
      const long long exps[6] = {0, 1, 2, 2045, 2046, 2047};
      b = (b & (long long)0x800fffffffffffffULL) | (exps[(z >> 3) % 6] << 52);
    }
    const double x = dfrom(b);
    const double h0 = x * 0.5, h1 = halve(x);
    const bool hbad = (x == x) ? dbits(h0) != dbits(h1) : (h1 == h1);  // NaN must stay NaN
    const double m = vabs(x);
    const double f0 = m * 4.0, f1 = times4(m);
    const bool fbad = (m == m) ? dbits(f0) != dbits(f1) : false;
    if (hbad) atomicAdd(out + 3, 1ull);
    if (fbad) atomicAdd(out + 4, 1ull);
  }
  // the integer-pipe predicates, min/max and sign operations against IEEE comparisons and
  // operations on pairs of non-NaN doubles (zeros, subnormals, the extreme binades and infinities
  // forced in often)
  if (i < n) {
    auto draw = [](unsigned long long z) {
      z ^= z >> 31;
      z *= 0x94D049BB133111EBull;
      z ^= z >> 30;
      long long b = (long long)(z & 0x800fffffffffffffULL);
      const int k = (int)((z >> 52) & 7);
      long long ex = (long long)((z >> 20) % 2047);  // never 2047 here: no NaN
      if (k == 0) ex = 0;                             // subnormal (or zero)
      if (k == 1) { ex = 0; b &= (long long)0x8000000000000000ULL; }  // +-0
      if (k == 2) { ex = 2047; b &= (long long)0x8000000000000000ULL; }  // +-inf
      if (k == 3) ex = (long long)((z >> 40) & 1) ? 1 : 2046;
      return dfrom(b | (ex << 52));
    };
    const unsigned long long s0 = (unsigned long long)(i + 2 * n) * 0x9E3779B97F4A7C15ull;
    const double x = draw(s0 + 0x2545F4914F6CDD1Dull);
    const double y = (s0 & 0x300) == 0 ? x : draw(s0 ^ 0xDA942042E4DD58B5ull);  // ties now and then
    int bad = 0;
    bad |= gt0(x) != (x > 0.0);
    bad |= lt0(x) != (x < 0.0);
    bad |= ge0(x) != (x >= 0.0);
    bad |= le0(x) != (x <= 0.0);
    bad |= is_zero(x) != (x == 0.0);
    bad |= same_sign(x, y) != ((x > 0.0 && y > 0.0) || (x < 0.0 && y < 0.0));
    if (!(x == 0.0 && y == 0.0)) bad |= vgt(x, y) != (x > y);  // -0 orders just below +0
    bad |= vmax(x, y) != (x >= y ? x : y);
    bad |= vmin(x, y) != (x <= y ? x : y);
    const double ax = fabs(x), ay = fabs(y);
    bad |= dbits(vabs(x)) != dbits(ax);
    bad |= pmax(ax, ay) != (ax >= ay ? ax : ay);
    bad |= pmin(ax, ay) != (ax <= ay ? ax : ay);
    bad |= dbits(with_sign(x, y)) != dbits(copysign(x, y));
    bad |= dbits(neg_if(true, x)) != dbits(x * -1.0);
    bad |= dbits(neg_if(false, x)) != dbits(x);
    if (bad) atomicAdd(out + 5, 1ull);
  }
  // the integer-pipe multiply against the FP64 multiply, bit for bit (any two NaNs agree)
  if (i < n) {
    auto mix = [](unsigned long long z) {
      z += 0x9E3779B97F4A7C15ull;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      return z ^ (z >> 31);
    };
    auto draw = [&](unsigned long long z, int kind, double other) {
      const unsigned long long r = mix(z);
      const unsigned long long sign = r & 0x8000000000000000ull, frac = r & 0x000fffffffffffffull;
      unsigned long long ex;
      switch (kind) {
        case 0: ex = 1023 - 40 + (r >> 52) % 81; break;                       // nearby exponents
        case 1: return dfrom((long long)r);                                   // any pattern
        case 2:                                                               // few significand bits
          return dfrom((long long)(sign | ((1020 + (r >> 56) % 7) << 52) | (frac & 0xff0000000000full)));
        case 3: ex = (r >> 60) & 1 ? (r >> 52) % 60 : 2046 - (r >> 52) % 60; break;  // extreme binades
        case 4: {  // the product's exponent at the overflow or the underflow edge
          const long long edge = (r >> 59) & 1 ? 2046 : 1;
          ex = (unsigned long long)(edge + (long long)((r >> 52) % 5) - 2 - ((dbits(other) >> 52) & 0x7ff) + 1023) &
               0x7ff;
          break;
        }
        default: return (double)((long long)(r % 33) - 16) * ((r >> 40) & 1 ? 0.5 : 1.0);  // small, zeros
      }
      return dfrom((long long)(sign | (ex << 52) | frac));
    };
    const unsigned long long s0 = (unsigned long long)(i + 3 * n) * 0xD6E8FEB86659FD93ull;
    const int ka = (int)(mix(s0) % 6), kb = (int)(mix(s0 + 1) % 6);
    const double x = draw(s0 + 2, ka == 4 ? 0 : ka, 0.0);
    const double y = draw(s0 + 3, kb, x);
    const double p0 = __dmul_rn(x, y), p1 = mul_int(x, y);
    const bool mbad = (p0 == p0 || p1 == p1) && dbits(p0) != dbits(p1);
    if (mbad) atomicAdd(out + 6, 1ull);
  }
}

void launch_math_check(long long n, unsigned long long* out, cudaStream_t st) {
  k_math_check<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, out);
}

static unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

void launch_prim(const Dev& d, cudaStream_t st) { k_prim<<<blocks_for(d.N, 256), 256, 0, st>>>(d); }
void launch_update(const Dev& d, cudaStream_t st) { k_update<<<blocks_for(d.N, 256), 256, 0, st>>>(d); }
void launch_flag(const Dev& d, cudaStream_t st) { k_flag<<<blocks_for(d.N, 256), 256, 0, st>>>(d); }
void launch_prim_if_flagged(const Dev& d, int prev_stage, cudaStream_t st) {
  k_prim_if_flagged<<<blocks_for(d.N, 256), 256, 0, st>>>(d, prev_stage);
}
void launch_set_dt(const unsigned long long* smax_bits, double cfl, double eta, double hmin, const double* hinv,
                   double* out, cudaStream_t st) {
  k_set_dt<<<1, 1, 0, st>>>(smax_bits, cfl, eta, hmin, hinv[0], hinv[1], hinv[2], out);
}
void launch_fofc(const Dev& d, cudaStream_t st) {
  auto grid = [&](const void* k) {
    return (unsigned)std::min((long long)blocks_for(d.N, 128), 2LL * resident_blocks(k, 128));
  };
  k_fo_faces<<<grid((const void*)k_fo_faces), 128, 0, st>>>(d);
  k_fo_edges<<<grid((const void*)k_fo_edges), 128, 0, st>>>(d);
  k_fo_recompute<<<grid((const void*)k_fo_recompute), 128, 0, st>>>(d);
}
void launch_maxspeed(const Dev& d, const double* U, Ptr3 B, unsigned long long* out, cudaStream_t st,
                     double* Pout) {
  const long long cap = 2LL * resident_blocks((const void*)k_maxspeed, 256);  // two waves of blocks
  k_maxspeed<<<(unsigned)std::min((long long)blocks_for(d.N, 256), cap), 256, 0, st>>>(d, U, B, out, Pout);
}
void launch_divb(const Dev& d, Ptr3 B, unsigned long long* out, cudaStream_t st) {
  k_divb<<<blocks_for(d.N, 256), 256, 0, st>>>(d, B, out);
}

}  // namespace mhd
