// mhd_cell.cuh -- per-cell operations: conserved -> primitive (Sec. 2.2), the update increments
// (Eqs. rk:increment-state, rk:increment-bfield), the validity flags and first-order flux
// correction (Sec. 2.5).
#pragma once
#include "mhd_device.cuh"
#include "mhd_index.cuh"
#include "mhd_internal.cuh"

namespace mhd {

__device__ __forceinline__ long long cell_id() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }

// ---- cons -> prim (Eq. state:primitive), with the face-averaged cell field ----------------
// from a cell's 5 conserved values u and its lower / upper face fields
__device__ __forceinline__ void prim_from(const Dev& D, const double* u, const double* lo, const double* hi,
                                          double* w) {
  const double rho = u[0];
  const double rinv = rcp(rho);
  const double u0 = u[1] * rinv, u1 = u[2] * rinv, u2 = u[3] * rinv;
  const double b0 = halve(lo[0] + hi[0]);
  const double b1 = halve(lo[1] + hi[1]);
  const double b2 = halve(lo[2] + hi[2]);
  const double u2s = fma(u0, u0, fma(u1, u1, u2 * u2));
  const double b2s = fma(b0, b0, fma(b1, b1, b2 * b2));
  const double eint = u[4] - halve(fma(rho, u2s, b2s));
  w[0] = rho; w[1] = u0; w[2] = u1; w[3] = u2;
  w[4] = (D.gam - 1.0) * eint;
  w[5] = b0; w[6] = b1; w[7] = b2;
}
__device__ __forceinline__ void load_cell(const Dev& D, const double* U, const double* const* B, long long X,
                                          double* u, double* lo, double* hi) {
  const long long N = D.N;
#pragma unroll
  for (int v = 0; v < 5; ++v) u[v] = U[v * N + X];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    lo[d] = B[d][X];
    hi[d] = B[d][shift(D, X, d, 1)];
  }
}
__device__ __forceinline__ void prim_of(const Dev& D, const double* U, const double* const* B,
                                        long long X, double* w) {
  double u[5], lo[3], hi[3];
  load_cell(D, U, B, X, u, lo, hi);
  prim_from(D, u, lo, hi, w);
}

// ---- CFL signal speed (Sec. 2.4, Eq. waves:fast-speed) ----------------------------------------
// max(m, s) for the cell's speed s = max_d (|u_d| + c_f,d) hmin / h_d, given a running maximum m.
// With S = a^2 + b^2/rho, every fast speed lies between sqrt(max(a^2, b^2/rho)) and sqrt(S) (the
// discriminant (a^2 + b^2/rho)^2 - 4 a^2 b_d^2/rho is (a^2 - b^2/rho)^2 + 4 a^2 (b^2 - b_d^2)/rho),
// so the three fast speeds are evaluated only when the upper bound, widened by 1e-12 against
// rounding, reaches m: the running maximum is the same value, with no square root for most cells
// of a cubic grid (one otherwise) instead of six. A non-finite speed gives +inf.
__device__ __forceinline__ double cfl_speed_max(const Dev& D, const double* U, const double* const* B, long long X,
                                                double m, double* Pout = nullptr) {
  double w[8];
  prim_of(D, U, B, X, w);
  if (Pout) {  // the primitives of the state, for a stage that starts from it
#pragma unroll
    for (int v = 0; v < 8; ++v) Pout[v * D.N + X] = w[v];
  }
  // a cell with a value that is not finite gives +inf, which the callers report as an error
  bool ok = true;
#pragma unroll
  for (int v = 0; v < 8; ++v) ok = ok && finite_d(w[v]);
  if (!ok) return __longlong_as_double(0x7ff0000000000000LL);
  const double hmin = pmin(D.h[0], pmin(D.h[1], D.h[2]));  // h_d > 0: bit patterns order them
  const double rinv = rcp(w[0]);
  const double a2 = D.gam * w[4] * rinv;
  const double b2 = fma(w[5], w[5], fma(w[6], w[6], w[7] * w[7]));
  const double sum = fma(b2, rinv, a2);
  if (dbits(D.h[0]) == dbits(D.h[1]) && dbits(D.h[0]) == dbits(D.h[2])) {
    // cubic cells (hmin / h_d is 1 up to an ulp): every speed is at most umax + sqrt(S) when
    // p >= 0 and rho > 0, and umax + sqrt(S) < m (1 - 1e-12) is tested on squares, without the
    // square root, S widened by 1e-12 against the rounding of the squares and the scale
    const double umax = pmax(vabs(w[1]), pmax(vabs(w[2]), vabs(w[3])));
    const double t = fma(m, -1e-12, m) - umax;
    if (gt0(t) && gt0(w[0]) && ge0(w[4]) && finite_d(sum) && dbits(sum * (1.0 + 1e-12)) < dbits(t * t))
      return m;
  } else {
    const double cu = sqrt_(sum);
    double hi = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) hi = pmax(hi, (vabs(w[1 + d]) + cu) * (hmin * D.hinv[d]));
    hi *= 1.0 + 1e-12;
    if (finite_d(hi) && dbits(hi) < dbits(m)) return m;
  }
  double s = 0.0;
  for (int d = 0; d < 3; ++d) {
    const double bn2 = w[5 + d] * w[5 + d];
    const double disc = pmax(fma(sum, sum, -4.0 * (a2 * bn2 * rinv)), 0.0);
    const double cf = sqrt_(halve(sum + sqrt_(disc)));
    const double v = (vabs(w[1 + d]) + cf) * (hmin * D.hinv[d]);
    // a speed that is not a number (a state with p < 0 or rho <= 0 can give one) is passed over,
    // as an ordered comparison with the running maximum passes it over; +inf is kept
    if (mag_bits(v) <= 0x7ff0000000000000LL) s = pmax(s, v);
  }
  return pmax(m, s);
}

__device__ __forceinline__ void prim_cell(const Dev& D, long long X) {
  double w[8];
  prim_of(D, D.Uin, D.Bin, X, w);
#pragma unroll
  for (int v = 0; v < 8; ++v) D.P[v * D.N + X] = w[v];
}

// ---- update: S_out = S^n + D(F, E) --------------------------------------------------------
// dt / h_d: from device memory when the step's dt came from the device-side CFL reduction
__device__ __forceinline__ double dth_of(const Dev& D, int d) { return D.dthp ? __ldg(D.dthp + d) : D.dth[d]; }
// U_v^n + dt sum_d (F_d[X] - F_d[X + d]) / h_d (Eq. rk:increment-state), with dt / h_d folded
// into the FMAs
__device__ __forceinline__ double cell_new(const Dev& D, int v, long long X, const long long* Xp) {
  const long long N = D.N;
  const double* F0 = D.F + (0 * 5 + v) * N;
  const double* F1 = D.F + (1 * 5 + v) * N;
  const double* F2 = D.F + (2 * 5 + v) * N;
  return fma(F0[X] - F0[Xp[0]], dth_of(D, 0),
             fma(F1[X] - F1[Xp[1]], dth_of(D, 1), fma(F2[X] - F2[Xp[2]], dth_of(D, 2), D.U0[v * N + X])));
}
// the updated field on the d-face of cell X (its lower face), by the discrete Stokes theorem
// (Eq. rk:increment-bfield); Xp[a], Xp[c] = X + 1 along a, c
__device__ __forceinline__ double face_new(const Dev& D, int d, long long X, const long long* Xp) {
  const long long N = D.N;
  const int a = (d + 1) % 3, c = (d + 2) % 3;
  const double* Ec = D.E + c * N;
  const double* Ea = D.E + a * N;
  return fma(Ec[X] - Ec[Xp[a]], dth_of(D, a), fma(Ea[Xp[c]] - Ea[X], dth_of(D, c), D.B0[d][X]));
}
// the updated state of cell X (5 conserved values, then its 3 lower faces), not yet stored
__device__ __forceinline__ void update_vals(const Dev& D, long long X, const long long* Xp, double* out) {
#pragma unroll
  for (int v = 0; v < 5; ++v) out[v] = cell_new(D, v, X, Xp);
#pragma unroll
  for (int d = 0; d < 3; ++d) out[5 + d] = face_new(D, d, X, Xp);
}
__device__ __forceinline__ void update_vals(const Dev& D, long long X, double* out) {
  const long long Xp[3] = {shift(D, X, 0, 1), shift(D, X, 1, 1), shift(D, X, 2, 1)};
  update_vals(D, X, Xp, out);
}
__device__ __forceinline__ void store_update(const Dev& D, long long X, const double* out) {
  const long long N = D.N;
#pragma unroll
  for (int v = 0; v < 5; ++v) D.Uout[v * N + X] = out[v];
#pragma unroll
  for (int d = 0; d < 3; ++d) D.Bout[d][X] = out[5 + d];
}
__device__ __forceinline__ void update_cell(const Dev& D, long long X) {
  double out[8];
  update_vals(D, X, out);
  store_update(D, X, out);
}

// ---- validity flags (Sec. 2.5) --------------------------------------------------------------
// u: the cell's 5 conserved values; lo / hi: its lower / upper face fields
__device__ __forceinline__ bool invalid_vals(const Dev& D, const double* u, const double* lo, const double* hi) {
  bool fin = true;
#pragma unroll
  for (int v = 0; v < 5; ++v) fin = fin && finite_d(u[v]);
  double bc[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    fin = fin && finite_d(lo[d]) && finite_d(hi[d]);
    bc[d] = halve(lo[d] + hi[d]);
  }
  if (!fin) return true;
  const double rho = u[0];
  if ((D.fofc_criteria & 1) && le0(rho)) return true;
  if (D.fofc_criteria & 2) {
    const double rinv = rcp(rho);
    const double u0 = u[1] * rinv, u1 = u[2] * rinv, u2 = u[3] * rinv;
    const double u2s = fma(u0, u0, fma(u1, u1, u2 * u2));
    const double b2s = fma(bc[0], bc[0], fma(bc[1], bc[1], bc[2] * bc[2]));
    const double p = (D.gam - 1.0) * (u[4] - halve(fma(rho, u2s, b2s)));
    if (!gt0(p)) return true;  // p <= 0 or NaN
  }
  return false;
}
__device__ __forceinline__ bool invalid_cell(const Dev& D, const double* U, double* const* B, long long X) {
  const long long N = D.N;
  double u[5], lo[3], hi[3];
#pragma unroll
  for (int v = 0; v < 5; ++v) u[v] = U[v * N + X];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    lo[d] = B[d][X];
    hi[d] = B[d][shift(D, X, d, 1)];
  }
  return invalid_vals(D, u, lo, hi);
}


// invalid_vals and the primitives w of the same state in one pass: the pressure the test needs
// is w[4], formed by the same operations (so the flag is the same bit for bit)
__device__ __forceinline__ bool prim_invalid(const Dev& D, const double* u, const double* lo, const double* hi,
                                             double* w) {
  prim_from(D, u, lo, hi, w);
  bool fin = true;
#pragma unroll
  for (int v = 0; v < 5; ++v) fin = fin && finite_d(u[v]);
#pragma unroll
  for (int d = 0; d < 3; ++d) fin = fin && finite_d(lo[d]) && finite_d(hi[d]);
  if (!fin) return true;
  if ((D.fofc_criteria & 1) && le0(u[0])) return true;
  return (D.fofc_criteria & 2) && !gt0(w[4]);
}

// flag of cell X (written) and whether it is set; with D.Pnext also the cell's primitives
__device__ __forceinline__ bool flag_cell(const Dev& D, long long X) {
  double u[5], lo[3], hi[3];
  load_cell(D, D.Uout, D.Bout, X, u, lo, hi);
  if (!D.Pnext) {
    const unsigned char f = invalid_vals(D, u, lo, hi) ? 1 : 0;
    D.flag[X] = f;
    return f != 0;
  }
  double w[8];
  const unsigned char f = prim_invalid(D, u, lo, hi, w) ? 1 : 0;
  D.flag[X] = f;
#pragma unroll
  for (int v = 0; v < 8; ++v) D.Pnext[v * D.N + X] = w[v];
  return f != 0;
}

// warp-aggregated count of flagged cells into counters[stage] (every lane of the warp calls it)
__device__ __forceinline__ void count_flags(const Dev& D, bool f) {
  const unsigned bal = __ballot_sync(0xffffffffu, f);
  if ((threadIdx.x & 31) == 0 && bal) atomicAdd(&D.counters[D.stage], (unsigned long long)__popc(bal));
}

// ---- first-order flux correction (Sec. 2.5) -------------------------------------------------
// First-order (piecewise-constant + LLF) face problem between cells Xl and Xr of S^n.
__device__ __forceinline__ void fo_face(const Dev& D, int d, long long Xl, long long Xr, long long Xface,
                                        double* f, double& alpha, double& ustar) {
  const int a = (d + 1) % 3, c = (d + 2) % 3;
  double wl[8], wr[8];
  prim_of(D, D.U0, D.B0, Xl, wl);
  prim_of(D, D.U0, D.B0, Xr, wr);
  const FaceState sl = {wl[0], wl[1 + d], wl[1 + a], wl[1 + c], wl[4], wl[5 + a], wl[5 + c]};
  const FaceState sr = {wr[0], wr[1 + d], wr[1 + a], wr[1 + c], wr[4], wr[5 + a], wr[5 + c]};
  double ap, am;
  riemann<RS_LLF>(sl, sr, D.B0[d][Xface], D.gam, D.gm1inv, f, ap, am, ustar);
  alpha = ap;
}

__device__ __forceinline__ bool flagged(const Dev& D, long long X) { return D.flag[X] != 0; }

__device__ __forceinline__ void fo_faces_cell(const Dev& D, long long X) {
  const long long N = D.N;
  for (int d = 0; d < 3; ++d) {
    const long long Xl = shift(D, X, d, -1);
    if (!(flagged(D, X) || flagged(D, Xl))) continue;
    const int a = (d + 1) % 3, c = (d + 2) % 3;
    double f[5], al, us;
    fo_face(D, d, Xl, X, X, f, al, us);
    if (D.resistive) {
      // Joule flux from the S^n field (same reading as the high-order faces)
      auto jedge = [&](int e, long long Y) {
        const int ae = (e + 1) % 3, ce = (e + 2) % 3;
        return (D.B0[ce][Y] - D.B0[ce][shift(D, Y, ae, -1)]) * D.hinv[ae] -
               (D.B0[ae][Y] - D.B0[ae][shift(D, Y, ce, -1)]) * D.hinv[ce];
      };
      const long long Xc = shift(D, X, c, 1), Xa = shift(D, X, a, 1);
      const double ea = 0.5 * D.eta * (jedge(a, X) + jedge(a, Xc));
      const double ec = 0.5 * D.eta * (jedge(c, X) + jedge(c, Xa));
      const double* Ba = D.B0[a];
      const double* Bc = D.B0[c];
      const double bcbar = 0.25 * (Bc[Xl] + Bc[X] + Bc[shift(D, Xl, c, 1)] + Bc[Xc]);
      const double babar = 0.25 * (Ba[Xl] + Ba[X] + Ba[shift(D, Xl, a, 1)] + Ba[Xa]);
      f[4] += fma(ea, bcbar, -ec * babar);
    }
    double* F = D.F + 5LL * d * N;
    F[0 * N + X] = f[0];
    F[(1 + d) * N + X] = f[1];
    F[(1 + a) * N + X] = f[2];
    F[(1 + c) * N + X] = f[3];
    F[4 * N + X] = f[4];
  }
}

// First-order EMF on the e-edge of X: the four cells around it are X, X-a, X-c, X-a-c.
__device__ __forceinline__ void fo_edges_cell(const Dev& D, long long X) {
  const long long N = D.N;
  for (int e = 0; e < 3; ++e) {
    const int a = (e + 1) % 3, c = (e + 2) % 3;
    const long long Xa = shift(D, X, a, -1), Xc = shift(D, X, c, -1), Xac = shift(D, Xa, c, -1);
    if (!(flagged(D, X) || flagged(D, Xa) || flagged(D, Xc) || flagged(D, Xac))) continue;
    // a-faces at X - c (between Xac, Xc) and X (between Xa, X); c-faces at X - a (Xac, Xa) and X (Xc, X)
    double f[5], apaB, apaT, apcL, apcR, uaB, uaT, ucL, ucR;
    fo_face(D, a, Xac, Xc, Xc, f, apaB, uaB);
    fo_face(D, a, Xa, X, X, f, apaT, uaT);
    fo_face(D, c, Xac, Xa, Xa, f, apcL, ucL);
    fo_face(D, c, Xc, X, X, f, apcR, ucR);
    const double baB = D.B0[a][Xc], baT = D.B0[a][X];
    const double bcL = D.B0[c][Xa], bcR = D.B0[c][X];
    double eLB, eRB, eLT, eRT;
    if (D.emf == EMF_Q26) {
      eLB = fma(-uaB, bcL, ucL * baB);
      eRB = fma(-uaB, bcR, ucR * baB);
      eLT = fma(-uaT, bcL, ucL * baT);
      eRT = fma(-uaT, bcR, ucR * baT);
    } else {
      // piecewise-constant FS18 / B25a: each corner takes the cell in that corner
      // (LB = X-a-c, RB = X-c, LT = X-a, RT = X)
      const long long cellQ[4] = {Xac, Xc, Xa, X};
      double ec[4];
      for (int q = 0; q < 4; ++q) {
        double w[8];
        prim_of(D, D.U0, D.B0, cellQ[q], w);
        if (D.emf == EMF_FS18) {
          const double bcs = (q & 1) ? bcR : bcL;
          const double bas = (q >> 1) ? baT : baB;
          ec[q] = fma(-w[1 + a], bcs, w[1 + c] * bas);
        } else {
          ec[q] = fma(-w[1 + a], w[5 + c], w[1 + c] * w[5 + a]);
        }
      }
      eLB = ec[0]; eRB = ec[1]; eLT = ec[2]; eRT = ec[3];
    }
    const double apa = pmax(apaB, apaT), apc = pmax(apcL, apcR);
    const double ia = rcp(apa + apa), ic = rcp(apc + apc);
    const double up = fma(apc, fma(apa, eLB, apa * eRB), apc * fma(apa, eLT, apa * eRT)) * (ia * ic);
    double emf = fma(apa * apa * ia, bcR - bcL, fma(-apc * apc * ic, baT - baB, up));
    if (D.resistive) {
      const double j = (D.B0[c][X] - D.B0[c][Xa]) * D.hinv[a] - (D.B0[a][X] - D.B0[a][Xc]) * D.hinv[c];
      emf = fma(D.eta, j, emf);
    }
    D.E[e * N + X] = emf;
  }
}

// Recompute every cell with a masked face and every face with a masked edge.
__device__ __forceinline__ void fo_recompute_cell(const Dev& D, long long X) {
  const long long N = D.N;
  const long long Xp[3] = {shift(D, X, 0, 1), shift(D, X, 1, 1), shift(D, X, 2, 1)};
  const long long Xm[3] = {shift(D, X, 0, -1), shift(D, X, 1, -1), shift(D, X, 2, -1)};
  bool cell = flagged(D, X);
  for (int d = 0; d < 3; ++d) cell = cell || flagged(D, Xp[d]) || flagged(D, Xm[d]);
  if (cell)
    for (int v = 0; v < 5; ++v) D.Uout[v * N + X] = cell_new(D, v, X, Xp);
  // e-edge at Y is masked if one of Y, Y-a, Y-c, Y-a-c is flagged
  auto edge_masked = [&](int e, long long Y) {
    const int a = (e + 1) % 3, c = (e + 2) % 3;
    const long long Ya = shift(D, Y, a, -1), Yc = shift(D, Y, c, -1);
    return flagged(D, Y) || flagged(D, Ya) || flagged(D, Yc) || flagged(D, shift(D, Ya, c, -1));
  };
  for (int d = 0; d < 3; ++d) {
    const int a = (d + 1) % 3, c = (d + 2) % 3;
    // the d-face at X is bounded by c-edges at X and X+a, and a-edges at X and X+c
    if (edge_masked(c, X) || edge_masked(c, Xp[a]) || edge_masked(a, X) || edge_masked(a, Xp[c]))
      D.Bout[d][X] = face_new(D, d, X, Xp);
  }
}

}  // namespace mhd
