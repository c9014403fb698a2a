// mhd_softmul.cuh -- binary64 multiply on the 32-bit integer pipe, for the FP64 rate probe and the
// arithmetic self-check only.
//
// Every kernel of the step is bound by the FP64 pipe (about 1.6 results per SM per clock) while the
// integer pipes stay mostly idle, so a product formed on the integer pipe would move work to the idle
// unit. A product of two doubles is a short integer computation: the two 53-bit significands
// multiply exactly in four 32 x 32 -> 64-bit multiply-adds, the 106-bit product is normalised by at
// most one bit, and IEEE 754's round-to-nearest-even needs only the first discarded bit and whether
// any later one is set. The step's kernels do not use it: measured (mhd_fp64_rate kinds 4-6) it adds
// throughput beside the FP64 pipe only with many warps per scheduler, and in the face sweep (two
// warps per scheduler at 255 registers) and the edge sweeps it made the kernels slower (about 50
// integer instructions per product, and a larger body that no longer fits the instruction cache).
#pragma once

namespace mhd {

// a b, bit for bit as the FP64 multiply rounds it (__dmul_rn) whenever both operands are normal
// and the product stays in the normal range; every other case (zero, subnormal, infinite or NaN
// operand, a product that underflows or may overflow) is handed to the FP64 multiply.
__device__ __forceinline__ double mul_int(double a, double b) {
  const unsigned ahi = (unsigned)__double2hiint(a), alo = (unsigned)__double2loint(a);
  const unsigned bhi = (unsigned)__double2hiint(b), blo = (unsigned)__double2loint(b);
  const unsigned ea = (ahi >> 20) & 0x7ffu, eb = (bhi >> 20) & 0x7ffu;
  // biased exponent of the product when the significand product lies in [2^104, 2^105)
  const int e = (int)(ea + eb) - 1023;
  if (!((ea - 1u < 0x7feu) & (eb - 1u < 0x7feu) & ((unsigned)(e - 1) < 0x7fdu))) return __dmul_rn(a, b);
  // significands with the implicit bit: high 21 bits and low 32 bits
  const unsigned ah = (ahi & 0xfffffu) | 0x100000u, bh = (bhi & 0xfffffu) | 0x100000u;
  const unsigned long long t0 = (unsigned long long)alo * blo;
  unsigned long long t1 = (unsigned long long)ah * blo + (t0 >> 32);
  t1 += (unsigned long long)alo * bh;
  const unsigned long long t2 = (unsigned long long)ah * bh + (t1 >> 32);
  // product P = t2 2^64 + w1 2^32 + w0; top: P >= 2^105 (one more in the exponent)
  const unsigned w0 = (unsigned)t0, w1 = (unsigned)t1;
  const unsigned top = (unsigned)(t2 >> 41);
  const unsigned long long n51 = (t2 << 13) | (w1 >> 19);  // P >> 51
  const unsigned long long sig = n51 >> (1 + top);         // the 53 kept bits
  const unsigned half = (unsigned)(n51 >> top) & 1u;       // the first discarded bit
  const unsigned rest = (((w1 & 0x7ffffu) | w0) != 0u) | (top & (unsigned)n51);  // any later one
  const unsigned up = half & (rest | (unsigned)sig);       // ties to even
  // exponent and significand add, so that a rounding carry moves into the exponent (to infinity
  // from the largest finite binade, as IEEE rounding does)
  unsigned long long r = ((unsigned long long)(unsigned)(e + (int)top - 1) << 52) + sig + up;
  r |= (unsigned long long)((ahi ^ bhi) & 0x80000000u) << 32;
  return __longlong_as_double((long long)r);
}

}  // namespace mhd
