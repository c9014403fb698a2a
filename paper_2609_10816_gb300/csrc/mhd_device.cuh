// mhd_device.cuh -- device numerics of the CT-MHD step (FP64, sm_103a).
//
// On GB300 the FP64 pipe retires about 2 DFMA per SM per clock (measured ~0.59 T DFMA/s over
// 152 SMs), 1/64 of the FP32 rate; a DMNMX or DSETP costs a full FP64 issue slot. Every
// comparison, min/max, |x| and sign test below therefore runs on the integer pipe, on the
// IEEE-754 bit pattern: for non-NaN doubles, the key  b ^ ((b >> 63) & 0x7fff...f)  of the bit
// pattern b orders like the value (with -0 just below +0), and for non-negative values the raw
// pattern already does. Only genuine arithmetic is issued to the FP64 pipe.
#pragma once
#include <cstdint>

namespace mhd {

enum { REC_PC = 0, REC_PLM_MC = 1, REC_PLM_MINMOD = 2, REC_PPM = 3 };
enum { RS_HLL = 0, RS_HLLD = 1, RS_LLF = 2 };
enum { EMF_Q26 = 0, EMF_FS18 = 1, EMF_B25A = 2 };

// ------------------------------------------------------------------------------------------
// Integer-pipe comparisons on doubles
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ double dfrom(long long b) { return __longlong_as_double(b); }
__device__ __forceinline__ long long okey(double x) {
  const long long b = dbits(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
// max/min return the first argument on ties (as in the method's tie rule).
__device__ __forceinline__ double vmax(double a, double b) { return okey(a) >= okey(b) ? a : b; }
__device__ __forceinline__ double vmin(double a, double b) { return okey(a) <= okey(b) ? a : b; }
// for a, b >= 0 (or +-0) the raw bit pattern orders like the value
__device__ __forceinline__ double pmax(double a, double b) { return dbits(a) >= dbits(b) ? a : b; }
__device__ __forceinline__ double pmin(double a, double b) { return dbits(a) <= dbits(b) ? a : b; }
__device__ __forceinline__ double vabs(double x) { return dfrom(dbits(x) & 0x7fffffffffffffffLL); }
__device__ __forceinline__ bool gt0(double x) { return okey(x) > 0; }    // x > 0
__device__ __forceinline__ bool lt0(double x) { return okey(x) < -1; }   // x < 0 (not -0)
__device__ __forceinline__ bool ge0(double x) { return okey(x) >= -1; }  // x >= 0 (either zero)
__device__ __forceinline__ bool le0(double x) { return !gt0(x); }
__device__ __forceinline__ bool vgt(double a, double b) { return okey(a) > okey(b); }
__device__ __forceinline__ bool is_zero(double x) { return (dbits(x) & 0x7fffffffffffffffLL) == 0; }
// strictly of the same sign, both non-zero
__device__ __forceinline__ bool same_sign(double a, double b) {
  return (gt0(a) && gt0(b)) || (lt0(a) && lt0(b));
}
// |m| carrying the sign of s
__device__ __forceinline__ double with_sign(double m, double s) {
  return dfrom((dbits(m) & 0x7fffffffffffffffLL) | (dbits(s) & (long long)0x8000000000000000ULL));
}
// sgn(x) in {-1, 0, +1} as a double (bit construction, no FP64 op)
__device__ __forceinline__ double sgnd(double x) {
  return gt0(x) ? 1.0 : (lt0(x) ? -1.0 : 0.0);
}
__device__ __forceinline__ bool finite_d(double x) {
  return ((dbits(x) >> 52) & 0x7ff) != 0x7ff;
}
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }

// ------------------------------------------------------------------------------------------
// Periodic line of points along one axis
// ------------------------------------------------------------------------------------------
struct Line {
  long long base;    // linear index of position 0 along the axis
  long long stride;  // linear-index step along the axis
  int n;             // points along the axis (periodic)
  __device__ __forceinline__ long long at(int p) const {
    p %= n;
    if (p < 0) p += n;
    return base + (long long)p * stride;
  }
};

// ------------------------------------------------------------------------------------------
// Sliding-window 1D reconstruction (Sec. 2.2). A Rec walks along a line of cell (or face)
// values. init() takes the LB + LA values at positions m0-LB .. m0+LA-1; each step() then
// takes the value at m + LA and returns the left/right states of the interface between
// points m-1 and m (left = upper value of point m-1, right = lower value of point m). Every
// point's slope, interface value and limiter run exactly once per sweep.
// ------------------------------------------------------------------------------------------
template <int R> struct Rec;

template <> struct Rec<REC_PC> {
  static constexpr int LB = 1, LA = 0;
  double prev;
  __device__ __forceinline__ void init(const double* q) { prev = q[0]; }
  __device__ __forceinline__ void step(double qn, double& L, double& R) {
    L = prev;
    R = qn;
    prev = qn;
  }
};

// half of the monotonised-central slope: sgn * min(|dl|, |dr|, |dl + dr| / 4)
__device__ __forceinline__ double half_slope_mc(double dl, double dr) {
  if (!same_sign(dl, dr)) return 0.0;
  double m = pmin(vabs(dl), vabs(dr));
  m = pmin(m, 0.25 * vabs(dl + dr));
  return with_sign(m, dl);
}
// half of the minmod slope: sgn * min(|dl|, |dr|) / 2
__device__ __forceinline__ double half_slope_minmod(double dl, double dr) {
  if (!same_sign(dl, dr)) return 0.0;
  return with_sign(0.5 * pmin(vabs(dl), vabs(dr)), dl);
}

template <int R> struct RecPLM {
  static constexpr int LB = 2, LA = 1;
  double qa, qb, aRprev;  // q[m-1], q[m], upper value of point m-1
  __device__ __forceinline__ double hs(double dl, double dr) const {
    return R == REC_PLM_MC ? half_slope_mc(dl, dr) : half_slope_minmod(dl, dr);
  }
  __device__ __forceinline__ void init(const double* q) {
    aRprev = q[1] + hs(q[1] - q[0], q[2] - q[1]);
    qa = q[1];
    qb = q[2];
  }
  __device__ __forceinline__ void step(double qn, double& L, double& Rt) {
    const double h = hs(qb - qa, qn - qb);
    L = aRprev;
    Rt = qb - h;
    aRprev = qb + h;
    qa = qb;
    qb = qn;
  }
};
template <> struct Rec<REC_PLM_MC> : RecPLM<REC_PLM_MC> {};
template <> struct Rec<REC_PLM_MINMOD> : RecPLM<REC_PLM_MINMOD> {};

// Colella & Woodward 1984: van Leer limited slope (their Eqs. 1.7-1.8), interface value
// (Eq. 1.6) and monotonicity constraints (Eq. 1.10).
__device__ __forceinline__ double vl_slope(double qm, double q0, double qp) {
  const double dl = q0 - qm, dr = qp - q0;
  if (!same_sign(dl, dr)) return 0.0;
  const double dc = 0.5 * (qp - qm);
  const double m = pmin(vabs(dc), 2.0 * pmin(vabs(dl), vabs(dr)));
  return with_sign(m, dc);
}
__device__ __forceinline__ double ppm_iface(double q0, double q1, double d0, double d1) {
  return fma(-(d1 - d0), 1.0 / 6.0, 0.5 * (q0 + q1));
}
__device__ __forceinline__ void ppm_mono(double a, double& aL, double& aR) {
  if (!same_sign(aR - a, a - aL)) {
    aL = a;
    aR = a;
    return;
  }
  const double da = aR - aL;
  const double a6 = 6.0 * fma(-0.5, aL + aR, a);
  const double p1 = da * a6, p2 = da * da;
  if (vgt(p1, p2)) {
    aL = fma(-2.0, aR, 3.0 * a);
  } else if (vgt(-p2, p1)) {
    aR = fma(-2.0, aL, 3.0 * a);
  }
}

template <> struct Rec<REC_PPM> {
  static constexpr int LB = 3, LA = 2;
  double q0, q1, q2;  // q[m-1], q[m], q[m+1]
  double d1;          // slope of point m
  double f1;          // interface value at m - 1/2
  double aRprev;      // upper value of point m-1
  __device__ __forceinline__ void init(const double* v) {  // v = q[m0-3 .. m0+1]
    const double da = vl_slope(v[0], v[1], v[2]);
    const double db = vl_slope(v[1], v[2], v[3]);
    const double dc = vl_slope(v[2], v[3], v[4]);
    const double fa = ppm_iface(v[1], v[2], da, db);
    const double fb = ppm_iface(v[2], v[3], db, dc);
    double aL = fa, aR = fb;
    ppm_mono(v[2], aL, aR);
    aRprev = aR;
    q0 = v[2];
    q1 = v[3];
    q2 = v[4];
    d1 = dc;
    f1 = fb;
  }
  __device__ __forceinline__ void step(double qn, double& L, double& R) {
    const double d2 = vl_slope(q1, q2, qn);
    const double f2 = ppm_iface(q1, q2, d1, d2);
    double aL = f1, aR = f2;
    ppm_mono(q1, aL, aR);
    L = aRprev;
    R = aL;
    aRprev = aR;
    q0 = q1;
    q1 = q2;
    q2 = qn;
    d1 = d2;
    f1 = f2;
  }
};

// ------------------------------------------------------------------------------------------
// Riemann problem on one face, in the face frame (n, t1, t2).
// W = {rho, u_n, u_t1, u_t2, p, b_t1, b_t2}; bn = stored face field.
// ------------------------------------------------------------------------------------------
struct FaceState {
  double rho, u, v, w, p, by, bz;
};

struct PhysFlux {
  double U[5], F[5];
  double pt, e, cf;
};

// Ideal-MHD flux of Eq. (mhd:conservation-laws) in the face frame, energy flux with e_tot,
// and the fast magnetosonic speed of Eq. (waves:fast-speed) along the normal.
__device__ __forceinline__ void phys(const FaceState& s, double bn, double gam, double gm1inv,
                                     PhysFlux& o) {
  const double bn2 = bn * bn;
  const double b2 = fma(s.by, s.by, fma(s.bz, s.bz, bn2));
  const double u2 = fma(s.u, s.u, fma(s.v, s.v, s.w * s.w));
  const double e = fma(s.p, gm1inv, 0.5 * fma(s.rho, u2, b2));
  const double pt = fma(0.5, b2, s.p);
  const double ub = fma(s.u, bn, fma(s.v, s.by, s.w * s.bz));
  const double mu = s.rho * s.u;
  o.U[0] = s.rho;
  o.U[1] = mu;
  o.U[2] = s.rho * s.v;
  o.U[3] = s.rho * s.w;
  o.U[4] = e;
  o.F[0] = mu;
  o.F[1] = fma(mu, s.u, pt - bn2);
  o.F[2] = fma(mu, s.v, -bn * s.by);
  o.F[3] = fma(mu, s.w, -bn * s.bz);
  o.F[4] = fma(e + pt, s.u, -ub * bn);
  o.pt = pt;
  o.e = e;
  const double rinv = rcp(s.rho);
  const double a2 = gam * s.p * rinv;
  const double sum = fma(b2, rinv, a2);
  double disc = fma(sum, sum, -4.0 * (a2 * bn2 * rinv));
  disc = pmax(disc, 0.0);
  o.cf = sqrt(0.5 * (sum + sqrt(disc)));
}

__device__ __forceinline__ void two_state(const PhysFlux& L, const PhysFlux& R, double ap,
                                          double am, double* F) {
  const double sum = ap + am;
  if (is_zero(sum)) {
    for (int v = 0; v < 5; ++v) F[v] = L.F[v];
    return;
  }
  const double inv = rcp(sum);
  const double apam = ap * am;
  for (int v = 0; v < 5; ++v)
    F[v] = (fma(ap, L.F[v], am * R.F[v]) - apam * (R.U[v] - L.U[v])) * inv;
}

// Miyoshi & Kusano (2005) HLLD without the Minoshima fixes.
__device__ __forceinline__ void hlld(const FaceState& sl, const FaceState& sr, double bn,
                                     const PhysFlux& L, const PhysFlux& R, double SL, double SR,
                                     double* F) {
  if (gt0(SL)) {
    for (int v = 0; v < 5; ++v) F[v] = L.F[v];
    return;
  }
  if (lt0(SR)) {
    for (int v = 0; v < 5; ++v) F[v] = R.F[v];
    return;
  }
  const double sluL = SL - sl.u, sruR = SR - sr.u;
  const double mL = sluL * sl.rho, mR = sruR * sr.rho;  // mass fluxes through the outer waves
  const double dinv = rcp(mR - mL);
  const double SM = ((mR * sr.u - mL * sl.u) + (L.pt - R.pt)) * dinv;
  const double ptS = (mR * L.pt - mL * R.pt + mL * mR * (sr.u - sl.u)) * dinv;
  const double bn2 = bn * bn;
  const FaceState* st[2] = {&sl, &sr};
  const PhysFlux* ph[2] = {&L, &R};
  const double S[2] = {SL, SR};
  double Us[2][5], rS[2], vS[2], wS[2], byS[2], bzS[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const FaceState& q = *st[s];
    const double su = S[s] - q.u;
    const double ssm = S[s] - SM;
    const double ssminv = rcp(ssm);
    const double rsu = q.rho * su;
    const double rs = rsu * ssminv;
    const double dd = fma(rsu, ssm, -bn2);
    const double scale = fma(rsu, su, bn2);
    double vs, ws, bys, bzs;
    if (!vgt(vabs(dd), 1e-12 * scale)) {
      vs = q.v;
      ws = q.w;
      bys = q.by;
      bzs = q.bz;
    } else {
      const double ddinv = rcp(dd);
      const double cv = bn * (SM - q.u) * ddinv;
      const double cb = fma(rsu, su, -bn2) * ddinv;
      vs = fma(-q.by, cv, q.v);
      ws = fma(-q.bz, cv, q.w);
      bys = q.by * cb;
      bzs = q.bz * cb;
    }
    const double vb = fma(q.u, bn, fma(q.v, q.by, q.w * q.bz));
    const double vbs = fma(SM, bn, fma(vs, bys, ws * bzs));
    const double es = (fma(su, ph[s]->e, -ph[s]->pt * q.u) + fma(ptS, SM, bn * (vb - vbs))) * ssminv;
    rS[s] = rs;
    vS[s] = vs;
    wS[s] = ws;
    byS[s] = bys;
    bzS[s] = bzs;
    Us[s][0] = rs;
    Us[s][1] = rs * SM;
    Us[s][2] = rs * vs;
    Us[s][3] = rs * ws;
    Us[s][4] = es;
  }
  const double sqL = sqrt(rS[0]), sqR = sqrt(rS[1]);
  const double abn = vabs(bn);
  const double SsL = SM - abn * rcp(sqL);
  const double SsR = SM + abn * rcp(sqR);
  const double sb = sgnd(bn);
  const double inv = rcp(sqL + sqR);
  const double vss = fma(sqL, vS[0], fma(sqR, vS[1], (byS[1] - byS[0]) * sb)) * inv;
  const double wss = fma(sqL, wS[0], fma(sqR, wS[1], (bzS[1] - bzS[0]) * sb)) * inv;
  const double sLR = sqL * sqR;
  const double byss = fma(sqL, byS[1], fma(sqR, byS[0], sLR * (vS[1] - vS[0]) * sb)) * inv;
  const double bzss = fma(sqL, bzS[1], fma(sqR, bzS[0], sLR * (wS[1] - wS[0]) * sb)) * inv;
  const double vbss = fma(SM, bn, fma(vss, byss, wss * bzss));
  // choose the region of the fan that contains the face (x/t = 0)
  int side;     // 0 left, 1 right
  bool dstar;   // double-star region
  if (ge0(SsL)) { side = 0; dstar = false; }
  else if (ge0(SM)) { side = 0; dstar = true; }
  else if (ge0(SsR)) { side = 1; dstar = true; }
  else { side = 1; dstar = false; }
  const PhysFlux& P = side ? R : L;
  const double Sx = side ? SR : SL;
  double Fs[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) Fs[v] = fma(Sx, Us[side][v] - P.U[v], P.F[v]);
  if (!dstar) {
    for (int v = 0; v < 5; ++v) F[v] = Fs[v];
    return;
  }
  const double sq = side ? sqR : sqL;
  const double sgn_side = side ? 1.0 : -1.0;
  const double vbs = fma(SM, bn, fma(vS[side], byS[side], wS[side] * bzS[side]));
  const double rs = rS[side];
  double Uss[5];
  Uss[0] = rs;
  Uss[1] = rs * SM;
  Uss[2] = rs * vss;
  Uss[3] = rs * wss;
  Uss[4] = fma(sgn_side * sq, (vbs - vbss) * sb, Us[side][4]);
  const double Ss = side ? SsR : SsL;
#pragma unroll
  for (int v = 0; v < 5; ++v) F[v] = fma(Ss, Uss[v] - Us[side][v], Fs[v]);
}

// Full face solve: flux of {rho, m_n, m_t1, m_t2, e}, alpha+/-, and the Q26 face velocity.
template <int RS>
__device__ __forceinline__ void riemann(const FaceState& sl, const FaceState& sr, double bn,
                                        double gam, double gm1inv, double* F, double& ap,
                                        double& am, double& ustar) {
  PhysFlux L, R;
  phys(sl, bn, gam, gm1inv, L);
  phys(sr, bn, gam, gm1inv, R);
  if (RS == RS_LLF) {
    const double a = pmax(vabs(sl.u) + L.cf, vabs(sr.u) + R.cf);
    ap = a;
    am = a;
    two_state(L, R, ap, am, F);
  } else {
    // Eq. (alpha-pm) = MK05 Eq. 67 speeds
    const double cmax = pmax(L.cf, R.cf);
    const double umax = vmax(sl.u, sr.u), umin = vmin(sl.u, sr.u);
    const double SR = umax + cmax;
    const double SL = umin - cmax;
    ap = vmax(0.0, SR);
    am = vmax(0.0, cmax - umin);
    if (RS == RS_HLL)
      two_state(L, R, ap, am, F);
    else
      hlld(sl, sr, bn, L, R, SL, SR, F);
  }
  // Eq. (q26-facevel)
  const double sum = ap + am;
  ustar = is_zero(sum) ? sl.u : fma(ap, sl.u, am * sr.u) * rcp(sum);
}

}  // namespace mhd
