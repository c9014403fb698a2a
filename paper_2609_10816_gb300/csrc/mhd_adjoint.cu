// mhd_adjoint.cu -- hand-written adjoint (vector-Jacobian product) of one step.
//
// The step is S1 = S0 + D(F(S0)), S2 = S0 + D((F(S0) + F(S1)) / 2), where F(S) collects the face
// fluxes and edge EMFs of a state and D is the flux divergence / discrete curl (Eqs.
// rk:increment-state, rk:increment-bfield). Reverse mode runs backwards through this chain; the
// adjoint of F at a state is assembled from local Jacobians, each obtained with forward-mode
// dual numbers on the GPU (one tangent per local input), so every limiter, min/max and
// Riemann-fan branch is differentiated on the branch the forward pass took:
//   edges   : E = LD04(Q26 corners) from 8 reconstructed edge values and 4 edge speeds, + eta j
//   edge rec: face fields and face velocities reconstructed to edges (point-wise reconstruction)
//   faces   : Riemann solve from the 7 + 7 reconstructed states and the normal field
//   face rec: primitives reconstructed to faces
//   prim    : conserved variables and the face field to primitives
// plus the Joule flux and eta j terms, which are bilinear and differentiated by hand. Adjoint
// contributions that several threads add to the same face are accumulated with atomics.
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mhd.h"
#include "mhd_cell.cuh"
#include "mhd_edge.cuh"
#include "mhd_face.cuh"
#include "mhd_riemann_vjp.cuh"

namespace mhd {

__device__ __forceinline__ long long aid() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }

// adds v, summed over the warp, to *out with one atomic (every lane of the warp must call it)
__device__ __forceinline__ void warp_add(double v, double* out) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(out, v);
}

// Jacobian of a point's reconstructed lower / upper values (aL, aR) in its window q[0..4]
// (q[2] the point): every reconstruction is piecewise linear, so the rows follow from the branch
// decisions, taken on the same values and with the same tie rules as the forward sweep.
// d(slope) / d(dl, dr) of the limited slopes, on the branch taken
__device__ __forceinline__ void vl_slope2_jac(double dl, double dr, double& gl, double& gr) {
  gl = gr = 0.0;
  if (!same_sign(dl, dr)) return;
  const double a = vabs(dl + dr);
  const bool left_min = dbits(vabs(dl)) <= dbits(vabs(dr));
  const double m4 = times4(left_min ? vabs(dl) : vabs(dr));
  if (dbits(a) <= dbits(m4)) { gl = 1.0; gr = 1.0; }   // |dl + dr|
  else if (left_min) gl = 4.0;                         // 4 |dl|
  else gr = 4.0;                                       // 4 |dr|
}
template <int R>
__device__ __forceinline__ void half_slope_jac(double dl, double dr, double& gl, double& gr) {
  gl = gr = 0.0;
  if (!same_sign(dl, dr)) return;
  const bool left_min = dbits(vabs(dl)) <= dbits(vabs(dr));
  if (R == REC_PLM_MINMOD) {
    (left_min ? gl : gr) = 0.5;
    return;
  }
  const double m = left_min ? vabs(dl) : vabs(dr);
  if (dbits(m) <= dbits(0.25 * vabs(dl + dr))) (left_min ? gl : gr) = 1.0;
  else { gl = 0.25; gr = 0.25; }
}
template <int R>
__device__ __forceinline__ void recon_jac(const double* q, double* JL, double* JR) {
#pragma unroll
  for (int k = 0; k < 5; ++k) JL[k] = JR[k] = 0.0;
  if (R == REC_PC) {
    JL[2] = JR[2] = 1.0;
  } else if (R == REC_PLM_MC || R == REC_PLM_MINMOD) {
    double gl, gr;  // h = gl (q2 - q1) + gr (q3 - q2); aL = q2 - h, aR = q2 + h
    half_slope_jac<R>(q[2] - q[1], q[3] - q[2], gl, gr);
    const double h1 = -gl, h2 = gl - gr, h3 = gr;
    JL[1] = -h1; JL[2] = 1.0 - h2; JL[3] = -h3;
    JR[1] = h1;  JR[2] = 1.0 + h2; JR[3] = h3;
  } else if (R == REC_PPM_EP) {
    // the decisions of Rec<REC_PPM_EP> on the same window
    const double e0 = q[1] - q[0], e1 = q[2] - q[1], e2 = q[3] - q[2], e3 = q[4] - q[3];
    const int s0 = sgn_code(e0), s1 = sgn_code(e1), s2 = sgn_code(e2), s3 = sgn_code(e3);
    const int ka = sgn_code(e1 - e0), kb = sgn_code(e2 - e1), kc = sgn_code(e3 - e2);
    const bool xa = ext_code(s0, s1, s2), xb = ext_code(s1, s2, s3);
    int pa, pb;  // 0: fourth-order value, 1: the lower cell's value, 2: the upper cell's
    const double aL = ppm_ep_face(q[0], q[1], q[2], q[3], xa && same_code(ka, kb), pa);
    const double aR = ppm_ep_face(q[1], q[2], q[3], q[4], xb && same_code(kb, kc), pb);
    if (pa == 0) {
      JL[0] = -1.0 / 12.0; JL[1] = 7.0 / 12.0; JL[2] = 7.0 / 12.0; JL[3] = -1.0 / 12.0;
    } else {
      JL[pa == 1 ? 1 : 2] = 1.0;
    }
    if (pb == 0) {
      JR[1] = -1.0 / 12.0; JR[2] = 7.0 / 12.0; JR[3] = 7.0 / 12.0; JR[4] = -1.0 / 12.0;
    } else {
      JR[pb == 1 ? 2 : 3] = 1.0;
    }
    if (!((xa || xb) && same_code(ka, kb) && same_code(kb, kc))) {
      const int mc = ppm_mono_case(aR - q[2], q[2] - aL);
      if (mc == PPM_FLAT) {
#pragma unroll
        for (int k = 0; k < 5; ++k) JL[k] = JR[k] = 0.0;
        JL[2] = JR[2] = 1.0;
      } else if (mc == PPM_FIX_L) {
#pragma unroll
        for (int k = 0; k < 5; ++k) JL[k] = -2.0 * JR[k];
        JL[2] += 3.0;
      } else if (mc == PPM_FIX_R) {
#pragma unroll
        for (int k = 0; k < 5; ++k) JR[k] = -2.0 * JL[k];
        JR[2] += 3.0;
      }
    }
  } else {
    const double e0 = q[1] - q[0], e1 = q[2] - q[1], e2 = q[3] - q[2], e3 = q[4] - q[3];
    double a0, b0, a1, b1, a2, b2;  // d_k = a_k e_k + b_k e_(k+1)
    vl_slope2_jac(e0, e1, a0, b0);
    vl_slope2_jac(e1, e2, a1, b1);
    vl_slope2_jac(e2, e3, a2, b2);
    // coefficient rows of d0, d1, d2 in q (e_k = q_(k+1) - q_k)
    double D0[5] = {-a0, a0 - b0, b0, 0.0, 0.0};
    double D1[5] = {0.0, -a1, a1 - b1, b1, 0.0};
    double D2[5] = {0.0, 0.0, -a2, a2 - b2, b2};
    // aL = q1 + e1/2 - (d1 - d0)/12, aR = q2 + e2/2 - (d2 - d1)/12
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      JL[k] = -(D1[k] - D0[k]) * (1.0 / 12.0);
      JR[k] = -(D2[k] - D1[k]) * (1.0 / 12.0);
    }
    JL[1] += 0.5; JL[2] += 0.5;
    JR[2] += 0.5; JR[3] += 0.5;
    // monotonicity (ppm_mono on the values)
    const double d0 = vl_slope2(e0, e1), d1 = vl_slope2(e1, e2), d2 = vl_slope2(e2, e3);
    const double aL = ppm_iface(q[1], e1, d0, d1), aR = ppm_iface(q[2], e2, d1, d2);
    const int mc = ppm_mono_case(aR - q[2], q[2] - aL);
    if (mc == PPM_FLAT) {
#pragma unroll
      for (int k = 0; k < 5; ++k) JL[k] = JR[k] = 0.0;
      JL[2] = JR[2] = 1.0;
    } else if (mc == PPM_FIX_L) {  // aL = 3 a - 2 aR
#pragma unroll
      for (int k = 0; k < 5; ++k) JL[k] = -2.0 * JR[k];
      JL[2] += 3.0;
    } else if (mc == PPM_FIX_R) {  // aR = 3 a - 2 aL
#pragma unroll
      for (int k = 0; k < 5; ++k) JR[k] = -2.0 * JL[k];
      JR[2] += 3.0;
    }
  }
}

// adjoint of the reconstruction of `arr` along dir at point X: lam_lo / lam_hi are the adjoints of
// its lower / upper values; the contributions go to the window's points (atomics: every point
// gets them from the five windows it lies in, and more than once on lines shorter than five)
template <int RC>
__device__ __forceinline__ void rec_scatter(const Dev& D, const double* arr, long long X, int dir, double lam_lo,
                                            double lam_hi, double* out) {
  if (lam_lo == 0.0 && lam_hi == 0.0) return;
  long long Z[5];
  double q[5], JL[5], JR[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    Z[k] = shift2(D, X, dir, k - 2);
    q[k] = arr[Z[k]];
  }
  recon_jac<RC>(q, JL, JR);
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const double c = fma(JL[k], lam_lo, JR[k] * lam_hi);
    if (c != 0.0) atomicAdd(&out[Z[k]], c);
  }
}

// Reverse sweep of q26_edge_emf (the Q26 corner EMFs of Eq. q26 and the LD04 average of Eq. ld04):
// g[k] = lam dE/d in[k] for in = (baB, baT, uaB, uaT, bcL, bcR, ucL, ucR, apa, ama, apc, amc).
__device__ __forceinline__ void q26_edge_vjp(const double* in, double lam, double* g) {
  const double baB = in[0], baT = in[1], uaB = in[2], uaT = in[3], bcL = in[4], bcR = in[5], ucL = in[6],
               ucR = in[7], apa = in[8], ama = in[9], apc = in[10], amc = in[11];
  const double eLB = fma(-uaB, bcL, ucL * baB), eRB = fma(-uaB, bcR, ucR * baB);
  const double eLT = fma(-uaT, bcL, ucL * baT), eRT = fma(-uaT, bcR, ucR * baT);
  const double sa = apa + ama, sc = apc + amc;
  const double w = rcp(sa * sc);
  const double ia = sc * w, ic = sa * w;
  const double hB = fma(apa, eLB, ama * eRB), hT = fma(apa, eLT, ama * eRT);
  const double P = fma(apc, hB, amc * hT);
  const double D1 = bcR - bcL, D2 = baT - baB;
  // E = apa ama ia D1 - apc amc ic D2 + P w
  const double dP = lam * w;
  double dw = lam * P;
  double dapc = dP * hB, damc = dP * hT;
  const double dhB = dP * apc, dhT = dP * amc;
  double dapa = dhB * eLB + dhT * eLT, dama = dhB * eRB + dhT * eRT;
  const double deLB = dhB * apa, deRB = dhB * ama, deLT = dhT * apa, deRT = dhT * ama;
  const double g1 = apa * ama * ia, g2 = apc * amc * ic;
  dapa += lam * ama * ia * D1;
  dama += lam * apa * ia * D1;
  const double dia = lam * apa * ama * D1;
  dapc -= lam * amc * ic * D2;
  damc -= lam * apc * ic * D2;
  const double dic = -lam * apc * amc * D2;
  // ia = sc w, ic = sa w, w = 1 / (sa sc)
  double dsc = dia * w, dsa = dic * w;
  dw += dia * sc + dic * sa;
  const double dprod = -dw * w * w;
  dsa += dprod * sc;
  dsc += dprod * sa;
  dapa += dsa;
  dama += dsa;
  dapc += dsc;
  damc += dsc;
  // corners e = -u_a b_c + u_c b_a
  g[0] = lam * g2 + deLB * ucL + deRB * ucR;          // baB
  g[1] = -lam * g2 + deLT * ucL + deRT * ucR;         // baT
  g[2] = -(deLB * bcL + deRB * bcR);                  // uaB
  g[3] = -(deLT * bcL + deRT * bcR);                  // uaT
  g[4] = -lam * g1 - deLB * uaB - deLT * uaT;         // bcL
  g[5] = lam * g1 - deRB * uaB - deRT * uaT;          // bcR
  g[6] = deLB * baB + deLT * baT;                     // ucL
  g[7] = deRB * baB + deRT * baT;                     // ucR
  g[8] = dapa;
  g[9] = dama;
  g[10] = dapc;
  g[11] = damc;
}

// Reverse sweep of Eq. (ld04) for any four corner EMFs e = (LB, RB, LT, RT): with
// s_a = apa + ama, s_c = apc + amc, w = 1 / (s_a s_c), E = apa ama (bcR - bcL) / s_a
// - apc amc (baT - baB) / s_c + (apc (apa eLB + ama eRB) + amc (apa eLT + ama eRT)) w; lam times
// dE/de -> de, dE/d(baB, baT, bcL, bcR) -> db, dE/d(apa, ama, apc, amc) -> dal.
__device__ __forceinline__ void ld04_vjp(double apa, double ama, double apc, double amc, const double* e, double baB,
                                         double baT, double bcL, double bcR, double lam, double* de, double* db,
                                         double* dal) {
  const double sa = apa + ama, sc = apc + amc;
  const double w = rcp(sa * sc);
  const double isa = sc * w, isc = sa * w;
  const double hB = fma(apa, e[0], ama * e[1]), hT = fma(apa, e[2], ama * e[3]);
  const double up = fma(apc, hB, amc * hT) * w;
  const double D1 = bcR - bcL, D2 = baT - baB;
  const double lw = lam * w;
  de[0] = lw * apc * apa;
  de[1] = lw * apc * ama;
  de[2] = lw * amc * apa;
  de[3] = lw * amc * ama;
  const double c1 = lam * apa * ama * isa, c2 = lam * apc * amc * isc;
  db[0] = c2;   // baB
  db[1] = -c2;  // baT
  db[2] = -c1;  // bcL
  db[3] = c1;   // bcR
  dal[0] = lam * (D1 * ama * ama * isa * isa + fma(apc, e[0], amc * e[2]) * w - up * isa);
  dal[1] = lam * (D1 * apa * apa * isa * isa + fma(apc, e[1], amc * e[3]) * w - up * isa);
  dal[2] = lam * (-D2 * amc * amc * isc * isc + hB * w - up * isc);
  dal[3] = lam * (-D2 * apc * apc * isc * isc + hT * w - up * isc);
}

// Reverse sweep of the FS18 corners (Eqs. fs18-average, fs18) and their LD04 average. in: baB, baT,
// bcL, bcR, the a-then-c partials xp[0..7] (u_a L:B,T, u_a R:B,T, u_c L:B,T, u_c R:B,T), the
// c-then-a partials (u_a B:L,R, u_a T:L,R, u_c B:L,R, u_c T:L,R), then apa, ama, apc, amc (24
// values); g (24) receives lam times the derivative in each.
__device__ __forceinline__ void fs18_edge_vjp(const double* in, double lam, double* g) {
  const double baB = in[0], baT = in[1], bcL = in[2], bcR = in[3];
  const double* xp = in + 4;
  const double* lr = in + 12;
  double ua[4], uc[4], e[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {  // corner q = sI + 2 sII: LB, RB, LT, RT
    const int sI = q & 1, sII = q >> 1;
    ua[q] = halve(xp[2 * sI + sII] + lr[2 * sII + sI]);
    uc[q] = halve(xp[4 + 2 * sI + sII] + lr[4 + 2 * sII + sI]);
    e[q] = fma(-ua[q], sI ? bcR : bcL, uc[q] * (sII ? baT : baB));
  }
  double de[4], db[4];
  ld04_vjp(in[20], in[21], in[22], in[23], e, baB, baT, bcL, bcR, lam, de, db, g + 20);
#pragma unroll
  for (int k = 0; k < 20; ++k) g[k] = 0.0;
  g[0] = db[0];
  g[1] = db[1];
  g[2] = db[2];
  g[3] = db[3];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int sI = q & 1, sII = q >> 1;
    const double bc = sI ? bcR : bcL, ba = sII ? baT : baB;
    const double dua = -de[q] * bc, duc = de[q] * ba;
    g[sI ? 3 : 2] -= de[q] * ua[q];
    g[sII ? 1 : 0] += de[q] * uc[q];
    // each velocity is the mean of its two reconstruction orders
    g[4 + 2 * sI + sII] += 0.5 * dua;
    g[12 + 2 * sII + sI] += 0.5 * dua;
    g[8 + 2 * sI + sII] += 0.5 * duc;
    g[16 + 2 * sII + sI] += 0.5 * duc;
  }
}

// Reverse sweep of the B25a corners (Eq. b25a-average: the mean of the two reconstruction orders
// of the cell EMF) and their LD04 average. in: baB, baT, bcL, bcR, the a-then-c partials (eps
// L:B,T, eps R:B,T), the c-then-a partials (eps B:L,R, eps T:L,R), then apa, ama, apc, amc (16
// values); g (16) receives lam times the derivative in each.
__device__ __forceinline__ void b25a_edge_vjp(const double* in, double lam, double* g) {
  const double* xp = in + 4;
  const double* lr = in + 8;
  double e[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int sI = q & 1, sII = q >> 1;
    e[q] = halve(xp[2 * sI + sII] + lr[2 * sII + sI]);
  }
  double de[4];
  ld04_vjp(in[12], in[13], in[14], in[15], e, in[0], in[1], in[2], in[3], lam, de, g, g + 12);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int sI = q & 1, sII = q >> 1;
    g[4 + 2 * sI + sII] = 0.5 * de[q];
    g[8 + 2 * sII + sI] = 0.5 * de[q];
  }
}

// ---- edges: adjoint of E_e from the reconstructed edge values, the edge speeds, eta j ------
template <int RC, int EMF>
__global__ void __launch_bounds__(128) k_adj_edges(AdjDev A) {
  const Dev& D = A.D;
  const long long X = aid();
  const long long N = D.N;
  double etaacc = 0.0;
  for (int e = 0; e < 3 && X < N; ++e) {  // no early return: the whole warp sums d/d(eta) below
    const int a = (e + 1) % 3, c = (e + 2) % 3;
    constexpr int NE = EMF == EMF_FS18 ? 20 : (EMF == EMF_B25A ? 12 : 8);  // adjoint slots per edge
    const double lam = A.lE[e * N + X];
    if (lam == 0.0) {
      for (int k = 0; k < NE; ++k) A.lEdge[(NE * e + k) * N + X] = 0.0;
      continue;
    }
    const long long Xc = shift(D, X, c, -1), Xa = shift(D, X, a, -1);
    // the reconstructed edge values as the forward edge sweeps formed them. Q26: b_a, u_a* bottom
    // and top (Epart), b_c, u_c* left and right (EdgeC). FS18: b_a bottom and top (Epart), b_c
    // left and right, the a-then-c velocity partials (Xpart) and the c-then-a ones (EdgeC). B25a:
    // the same with the partials of the cell EMF.
    constexpr int NI = EMF == EMF_FS18 ? 24 : (EMF == EMF_B25A ? 16 : 12);
    double in[NI];
    const double* pa = D.Epart + 4LL * e * N;
    if (EMF == EMF_B25A) {  // b_a B/T, b_c L/R, the a-then-c EMF partials (Xpart), the c-then-a ones
      const double* pc = D.EdgeC + 10LL * e * N;
      const double* xp = D.Xpart + 8LL * e * N;
      in[0] = pa[X];
      in[1] = pa[N + X];
      in[2] = pc[X];
      in[3] = pc[N + X];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        in[4 + k] = xp[k * N + X];
        in[8 + k] = pc[(2 + k) * N + X];
      }
    } else if (EMF == EMF_FS18) {
      const double* pc = D.EdgeC + 10LL * e * N;
      const double* xp = D.Xpart + 8LL * e * N;
      in[0] = pa[X];
      in[1] = pa[N + X];
      in[2] = pc[X];
      in[3] = pc[N + X];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        in[4 + k] = xp[k * N + X];
        in[12 + k] = pc[(2 + k) * N + X];
      }
    } else {
      const double* pc = D.EdgeC + 4LL * e * N;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        in[k] = pa[k * N + X];
        in[4 + k] = pc[k * N + X];
      }
    }
    const double* Apa = D.Ap + a * N;
    const double* Ama = D.Am + a * N;
    const double* Apc = D.Ap + c * N;
    const double* Amc = D.Am + c * N;
    // Eq. (alpha-edge): the max keeps its first argument on ties (pmax)
    const bool wa_p = dbits(Apa[Xc]) >= dbits(Apa[X]), wa_m = dbits(Ama[Xc]) >= dbits(Ama[X]);
    const bool wc_p = dbits(Apc[Xa]) >= dbits(Apc[X]), wc_m = dbits(Amc[Xa]) >= dbits(Amc[X]);
    in[NI - 4] = wa_p ? Apa[Xc] : Apa[X];
    in[NI - 3] = wa_m ? Ama[Xc] : Ama[X];
    in[NI - 2] = wc_p ? Apc[Xa] : Apc[X];
    in[NI - 1] = wc_m ? Amc[Xa] : Amc[X];
    double g[NI];
    if (EMF == EMF_FS18) fs18_edge_vjp(in, lam, g);
    else if (EMF == EMF_B25A) b25a_edge_vjp(in, lam, g);
    else q26_edge_vjp(in, lam, g);
    for (int k = 0; k < NE; ++k) A.lEdge[(NE * e + k) * N + X] = g[k];
    atomicAdd(&A.lAp[a * N + (wa_p ? Xc : X)], g[NI - 4]);
    atomicAdd(&A.lAm[a * N + (wa_m ? Xc : X)], g[NI - 3]);
    atomicAdd(&A.lAp[c * N + (wc_p ? Xa : X)], g[NI - 2]);
    atomicAdd(&A.lAm[c * N + (wc_m ? Xa : X)], g[NI - 1]);
    if (D.resistive) {  // E += eta j, j = (b_c[X] - b_c[X-a]) / h_a - (b_a[X] - b_a[X-c]) / h_c
      const double* Ba = D.Bin[a];
      const double* Bc = D.Bin[c];
      const double j = (Bc[X] - Bc[Xa]) * D.hinv[a] - (Ba[X] - Ba[Xc]) * D.hinv[c];
      etaacc += lam * j;
      const double la = D.eta * lam * D.hinv[a], lc = D.eta * lam * D.hinv[c];
      atomicAdd(&A.lB[c * N + X], la);
      atomicAdd(&A.lB[c * N + Xa], -la);
      atomicAdd(&A.lB[a * N + X], -lc);
      atomicAdd(&A.lB[a * N + Xc], lc);
    }
  }
  warp_add(etaacc, A.lEta);
}

// ---- edge reconstructions: adjoint of the face arrays reconstructed to the edges -----------
// Face array of direction d is reconstructed along t1 = d + 1 as the "a" array of e-edges with
// e = d + 2 (Q26: bottom/top slots 0/1 for b, 2/3 for u*), and along t2 = d + 2 as the "c" array
// of e-edges with e = d + 1 (Q26: left/right slots 4/5 for b, 6/7 for u*; FS18 and B25a: the
// slots of the lEdge layouts in mhd_internal.cuh). Point m's lower value is the top/right value
// at edge m; its upper value is the bottom/left value at edge m + t.
// FS18's velocity sources on the d-faces, as rows of the face states (LR): reconstructed along c of
// the e-edges with d = a (u_a L, u_a R, u_c L, u_c R: the normal and the first tangential
// component) and along a of the e-edges with d = c (u_a B, u_a T, u_c B, u_c T: the second
// tangential and the normal component)
__device__ constexpr int kFs18RowBt[4] = {1, 8, 2, 9};
__device__ constexpr int kFs18RowLr[4] = {3, 10, 1, 8};

template <int RC, int EMF>
__global__ void __launch_bounds__(128) k_adj_edge_rec(AdjDev A) {
  const Dev& D = A.D;
  const long long X = aid();
  if (X >= D.N) return;
  const long long N = D.N;
  constexpr int NE = EMF == EMF_FS18 ? 20 : (EMF == EMF_B25A ? 12 : 8);
  for (int d = 0; d < 3; ++d) {
    const int t1 = (d + 1) % 3, e1 = (d + 2) % 3;  // d is "a" of e1, reconstructed along c(e1) = t1
    const int t2 = (d + 2) % 3, e2 = (d + 1) % 3;  // d is "c" of e2, reconstructed along a(e2) = t2
    const double* L1 = A.lEdge + (long long)NE * e1 * N;
    const double* L2 = A.lEdge + (long long)NE * e2 * N;
    const long long X1 = shift(D, X, t1, 1), X2 = shift(D, X, t2, 1);
    // point X's lower value is the top (right) value at edge X, its upper value the bottom (left)
    // value at edge X + t
    if (EMF == EMF_B25A) {  // b_d, and the e-EMF face values EfL (d = a of e1) and EfB (d = c of e2)
      rec_scatter<RC>(D, D.Bin[d], X, t1, L1[1 * N + X], L1[0 * N + X1], A.lB + d * N);
      rec_scatter<RC>(D, D.Bin[d], X, t2, L2[3 * N + X], L2[2 * N + X2], A.lB + d * N);
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const long long r1 = (2LL * e1 + k) * N, r2 = (2LL * e2 + k) * N;
        rec_scatter<RC>(D, D.EfL + r1, X, t1, L1[(5 + 2 * k) * N + X], L1[(4 + 2 * k) * N + X1], A.lEf + r1);
        rec_scatter<RC>(D, D.EfB + r2, X, t2, L2[(9 + 2 * k) * N + X], L2[(8 + 2 * k) * N + X2], A.lEf + 6 * N + r2);
      }
    } else if (EMF == EMF_FS18) {
      rec_scatter<RC>(D, D.Bin[d], X, t1, L1[1 * N + X], L1[0 * N + X1], A.lB + d * N);
      rec_scatter<RC>(D, D.Bin[d], X, t2, L2[3 * N + X], L2[2 * N + X2], A.lB + d * N);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const long long rb = (14LL * d + kFs18RowBt[k]) * N, rl = (14LL * d + kFs18RowLr[k]) * N;
        rec_scatter<RC>(D, D.LR + rb, X, t1, L1[(5 + 2 * k) * N + X], L1[(4 + 2 * k) * N + X1], A.lLR + rb);
        rec_scatter<RC>(D, D.LR + rl, X, t2, L2[(13 + 2 * k) * N + X], L2[(12 + 2 * k) * N + X2], A.lLR + rl);
      }
    } else {
      rec_scatter<RC>(D, D.Bin[d], X, t1, L1[1 * N + X], L1[0 * N + X1], A.lB + d * N);
      rec_scatter<RC>(D, D.Bin[d], X, t2, L2[5 * N + X], L2[4 * N + X2], A.lB + d * N);
      rec_scatter<RC>(D, D.Us + d * N, X, t1, L1[3 * N + X], L1[2 * N + X1], A.lUs + d * N);
      rec_scatter<RC>(D, D.Us + d * N, X, t2, L2[7 * N + X], L2[6 * N + X2], A.lUs + d * N);
    }
  }
}

// ---- reconstructions as reverse sweeps (PPM) ------------------------------------------------
// The adjoint of Rec<REC_PPM> walking a line: with e_k = q_{k+1} - q_k, the doubled slope
// d_k = vl_slope2(e_{k-1}, e_k) (linear on its branch, d_k = a_k e_{k-1} + b_k e_k), the interface
// value f_{k+1/2} = q_k + e_k / 2 - (d_{k+1} - d_k) / 12 and the monotonicity constraint of point k
// acting on (f_{k-1/2}, f_{k+1/2}), the adjoints flow back through these relations in the order
// they were formed. Step i takes the adjoints of point i's lower and upper values; the adjoint of
// q_{i-2} is then complete and is returned. A thread walks its segment [m0, m1) from m0 - 2 to
// m1 + 1 (the windows of every point whose window holds a point of the segment), with the
// forward values recomputed by the forward functions (the same values and branch decisions) and
// no atomics: each point's sum is formed by one thread.
struct RevPPM {
  double q0, q1, q2;          // q_i, q_{i+1}, q_{i+2}
  double e1;                  // e_{i+1}
  double d0, d1;              // d_i, d_{i+1}
  double am, bm, a0, b0, a1, b1;  // slope jacobians of d_{i-1}, d_i, d_{i+1}
  double fL, fR;              // f_{i-1/2}, f_{i+1/2}
  double lfp, ld, le, g2, g1;  // adjoints: upper value of point i-1, d_{i-1}, e_{i-2}, q_{i-2}, q_{i-1}

  // v = q_{i-2} .. q_{i+2} for the first step i
  __device__ __forceinline__ void init(const double* v) {
    const double e0 = v[1] - v[0], e1_ = v[2] - v[1], e2 = v[3] - v[2], e3 = v[4] - v[3];
    const double dm = vl_slope2(e0, e1_);
    vl_slope2_jac(e0, e1_, am, bm);
    d0 = vl_slope2(e1_, e2);
    vl_slope2_jac(e1_, e2, a0, b0);
    d1 = vl_slope2(e2, e3);
    vl_slope2_jac(e2, e3, a1, b1);
    fL = ppm_iface(v[1], e1_, dm, d0);
    fR = ppm_iface(v[2], e2, d0, d1);
    q0 = v[2]; q1 = v[3]; q2 = v[4];
    e1 = e3;
    lfp = ld = le = g2 = g1 = 0.0;
  }
  // lam_lo, lam_hi: adjoints of point i's lower / upper values; qn = q_{i+3}. Returns the adjoint of
  // q_{i-2}.
  __device__ __forceinline__ double step(double lam_lo, double lam_hi, double qn) {
    double lL = lam_lo, lR = lam_hi, gi = 0.0;
    const int mc = ppm_mono_case(fR - q0, q0 - fL);
    if (mc == PPM_FLAT) {  // aL = aR = q_i
      gi = lam_lo + lam_hi;
      lL = lR = 0.0;
    } else if (mc == PPM_FIX_L) {  // aL = 3 q_i - 2 aR
      gi = 3.0 * lam_lo;
      lR = fma(-2.0, lam_lo, lam_hi);
      lL = 0.0;
    } else if (mc == PPM_FIX_R) {  // aR = 3 q_i - 2 aL
      gi = 3.0 * lam_hi;
      lL = fma(-2.0, lam_hi, lam_lo);
      lR = 0.0;
    }
    const double lf = lfp + lL;           // f_{i-1/2}, complete
    g1 += lf;                             // its q_{i-1}
    double le1 = halve(lf);               // its e_{i-1}
    const double ldi = lf * (-1.0 / 12.0);  // its d_i
    ld = fma(lf, 1.0 / 12.0, ld);         // its d_{i-1}: complete
    le = fma(am, ld, le);                 // d_{i-1} -> e_{i-2} (complete), e_{i-1}
    le1 = fma(bm, ld, le1);
    g1 += le;                             // e_{i-2} = q_{i-1} - q_{i-2}
    const double out = g2 - le;
    g2 = g1; g1 = gi; le = le1; ld = ldi; lfp = lR;
    // forward values of the next step
    const double en = qn - q2;            // e_{i+2}
    const double dn = vl_slope2(e1, en);  // d_{i+2}
    double an, bn;
    vl_slope2_jac(e1, en, an, bn);
    const double fn = ppm_iface(q1, e1, d1, dn);  // f_{i+3/2}
    am = a0; bm = b0; a0 = a1; b0 = b1; a1 = an; b1 = bn;
    d0 = d1; d1 = dn;
    e1 = en;
    q0 = q1; q1 = q2; q2 = qn;
    fL = fR; fR = fn;
    return out;
  }
};

// One reconstruction source of the reverse sweeps along s: the reconstructed array, the adjoints
// of the lower value at X and of the upper value at X (stored at X + s), and where the result
// accumulates.
struct RecSrc {
  const double* q;
  const double* lam_lo;
  const double* lam_hi;
  double* out;
};
// face states (k_adj_face_rec): the 7 reconstructed primitives of the s-faces
__device__ __forceinline__ RecSrc face_src(const AdjDev& A, int s, int v) {
  const long long N = A.D.N;
  const int a = (s + 1) % 3, c = (s + 2) % 3;
  const int slot = v == 0 ? 0 : v == 1 ? 1 + s : v == 2 ? 1 + a : v == 3 ? 1 + c : v == 4 ? 4 : v == 5 ? 5 + a : 5 + c;
  const double* lLR = A.lLR + 14LL * s * N;
  return {A.D.P + slot * N, lLR + (7 + v) * N, lLR + v * N, A.lP + slot * N};
}
// edge values (k_adj_edge_rec): the arrays reconstructed along s, for the face arrays d = s - 1
// (s is their "c" direction, e-edges e = s + 1: bottom / top values) and d = s + 1 (s is their "a"
// direction, e-edges e = s + 2: left / right values). Q26: b_d and u_d^* of each (4 sources);
// FS18: b_d and the four velocity states of each (10 sources); B25a: b_d and the two face values
// of the cell EMF of each (6 sources).
template <int EMF>
__device__ __forceinline__ RecSrc edge_src(const AdjDev& A, int s, int v) {
  const long long N = A.D.N;
  if (EMF == EMF_B25A) {  // b_d and the e-EMF values EfL (bottom/top) or EfB (left/right)
    const bool bt = v < 3;
    const int d = bt ? (s + 2) % 3 : (s + 1) % 3;
    const int e = bt ? (s + 1) % 3 : (s + 2) % 3;
    const int k = bt ? v : v - 3;
    const double* L = A.lEdge + 12LL * e * N;
    if (k == 0) {
      const int lo = bt ? 1 : 3;
      return {A.D.Bin[d], L + lo * N, L + (lo - 1) * N, A.lB + d * N};
    }
    const long long row = (2LL * e + k - 1) * N;
    const int lo = (bt ? 5 : 9) + 2 * (k - 1);
    return {(bt ? A.D.EfL : A.D.EfB) + row, L + lo * N, L + (lo - 1) * N, A.lEf + (bt ? 0 : 6 * N) + row};
  }
  if (EMF == EMF_FS18) {
    const bool bt = v < 5;
    const int d = bt ? (s + 2) % 3 : (s + 1) % 3;
    const int e = bt ? (s + 1) % 3 : (s + 2) % 3;
    const int k = bt ? v : v - 5;  // 0: b_d; 1-4: the velocity states
    const double* L = A.lEdge + 20LL * e * N;
    if (k == 0) {
      const int lo = bt ? 1 : 3;
      return {A.D.Bin[d], L + lo * N, L + (lo - 1) * N, A.lB + d * N};
    }
    const long long row = (14LL * d + (bt ? kFs18RowBt[k - 1] : kFs18RowLr[k - 1])) * N;
    const int lo = (bt ? 5 : 13) + 2 * (k - 1);
    return {A.D.LR + row, L + lo * N, L + (lo - 1) * N, A.lLR + row};
  }
  const bool bt = v < 2;
  const int d = bt ? (s + 2) % 3 : (s + 1) % 3;
  const int e = bt ? (s + 1) % 3 : (s + 2) % 3;
  const bool vel = v & 1;
  const double* L = A.lEdge + 8LL * e * N;
  const int lo = bt ? (vel ? 3 : 1) : (vel ? 7 : 5), hi = lo - 1;
  return {vel ? A.D.Us + d * N : A.D.Bin[d], L + lo * N, L + hi * N, (vel ? A.lUs : A.lB) + d * N};
}

// B25a's cell EMF eps_e reconstructed along s to faces (Eqs. b25a-b-avg, b25a-emf-centre): along
// a for e = s - 1 (the EfL values, left / right), along c for e = s + 1 (the EfB values)
__device__ __forceinline__ RecSrc eps_src(const AdjDev& A, int s, int v) {
  const long long N = A.D.N;
  const int e = v == 0 ? (s + 2) % 3 : (s + 1) % 3;
  const double* lf = A.lEf + (v == 0 ? 0 : 6 * N) + 2LL * e * N;
  // point Y's lower value is the right value at face Y, its upper value the left value at Y + s
  return {A.eps + e * N, lf + N, lf, A.leps + e * N};
}

template <int KIND, int EMF>
__device__ __forceinline__ int rec_sources() {
  return KIND == 1 ? 7 : (KIND == 2 ? 2 : (EMF == EMF_FS18 ? 10 : (EMF == EMF_B25A ? 6 : 4)));
}

// Reverse PPM sweeps along s over all sources of one kind (0 edge values, 1 face states, 2 B25a's
// cell EMF): thread = (source, line segment).
template <int KIND, int EMF = EMF_Q26>
__global__ void __launch_bounds__(128) k_adj_rec_sweep(AdjDev A, int s, int seg) {
  const Dev& D = A.D;
  const long long nsw = sweep_threads(D, s, seg);
  const long long tid = aid();
  const int nsrc = rec_sources<KIND, EMF>();
  if (tid >= nsw * nsrc) return;
  const int v = (int)(tid / nsw);
  Line ln;
  int m0, m1;
  if (!sweep_line_at(D, s, seg, tid - v * nsw, ln, m0, m1, s == 0)) return;
  const RecSrc r = KIND == 1 ? face_src(A, s, v) : (KIND == 2 ? eps_src(A, s, v) : edge_src<EMF>(A, s, v));
  RevPPM w;
  double v5[5];
#pragma unroll
  for (int t = 0; t < 5; ++t) v5[t] = r.q[ln.at(m0 - 4 + t)];
  w.init(v5);
  for (int i = m0 - 2; i <= m1 + 1; ++i) {
    const long long X = ln.at(i);
    const double g = w.step(r.lam_lo[X], r.lam_hi[ln.at(i + 1)], r.q[ln.at(i + 3)]);
    if (i - 2 >= m0) {
      const long long Y = ln.at(i - 2);
      r.out[Y] += g;
    }
  }
}

// ---- faces: adjoint of the Riemann solve -------------------------------------------------
// gradient of the weighted face outputs in the 15 inputs by the dual numbers: one forward pass
// per input (the reference that the reverse sweep of mhd_riemann_vjp.cuh is checked against)
template <int RS>
__device__ void riemann_grad_dual(const double* WL, const double* WR, double bn, double gam, double gm1inv,
                                  const double* lf, double lap, double lam_, double lus, double* g) {
#pragma unroll 1
  for (int i = 0; i < 15; ++i) {
    FaceStateT<Dual> sl, sr;
    Dual* pl = &sl.rho;
    Dual* pr = &sr.rho;
    for (int v = 0; v < 7; ++v) {
      pl[v] = Dual(WL[v], i == v ? 1.0 : 0.0);
      pr[v] = Dual(WR[v], i == 7 + v ? 1.0 : 0.0);
    }
    const Dual b = Dual(bn, i == 14 ? 1.0 : 0.0);
    Dual F[5], ap, am, us;
    riemann<RS>(sl, sr, b, gam, gm1inv, F, ap, am, us);
    double acc = lap * ap.t + lam_ * am.t + lus * us.t;
#pragma unroll
    for (int v = 0; v < 5; ++v) acc = fma(lf[v], F[v].t, acc);
    g[i] = acc;
  }
}

// the same gradient by the reverse sweep
template <int RS>
__device__ __forceinline__ void riemann_grad_rev(const double* WL, const double* WR, double bn, double gam,
                                                 double gm1inv, const double* lf, double lap, double lam_,
                                                 double lus, double* g) {
  const FaceState sl = {WL[0], WL[1], WL[2], WL[3], WL[4], WL[5], WL[6]};
  const FaceState sr = {WR[0], WR[1], WR[2], WR[3], WR[4], WR[5], WR[6]};
  FaceState dl, dr;
  double dbn;
  riemann_vjp<RS>(sl, sr, bn, gam, gm1inv, lf, lap, lam_, lus, dl, dr, dbn);
  const double* pl = &dl.rho;
  const double* pr = &dr.rho;
  for (int v = 0; v < 7; ++v) {
    g[v] = pl[v];
    g[7 + v] = pr[v];
  }
  g[14] = dbn;
}

template <int RC, int RS>
__global__ void __launch_bounds__(128) k_adj_faces(AdjDev A, int dir) {
  const Dev& D = A.D;
  const long long t = aid();
  if (t >= D.N) return;
  const long long f = tiled_cell(D, t);  // a warp's faces on an 8 x 4 patch: fewer divergent fan branches
  const long long N = D.N;
  const int a = (dir + 1) % 3, c = (dir + 2) % 3;
  // the face states as the forward sweep reconstructed them (stored by its recompute)
  double WL[7], WR[7];
  const double* lr = D.LR + 14LL * dir * N;
#pragma unroll
  for (int v = 0; v < 7; ++v) {
    WL[v] = lr[v * N + f];
    WR[v] = lr[(7 + v) * N + f];
  }
  const double bn = D.Bin[dir][f];
  const double* lF = A.lF + 5LL * dir * N;
  const double lf[5] = {lF[0 * N + f], lF[(1 + dir) * N + f], lF[(1 + a) * N + f], lF[(1 + c) * N + f],
                        lF[4 * N + f]};
  double g[15];
  riemann_grad_rev<RS>(WL, WR, bn, D.gam, D.gm1inv, lf, A.lAp[dir * N + f], A.lAm[dir * N + f],
                       A.lUs[dir * N + f], g);
#pragma unroll
  for (int i = 0; i < 14; ++i) A.lLR[(14LL * dir + i) * N + f] += g[i];
  atomicAdd(&A.lB[dir * N + f], g[14]);
}

// Self-check of the reverse sweep: n hashed face problems (states from smooth to extreme, with
// repeated, zero and sign-flipped values to reach the degenerate branches) and weights; the
// largest |reverse - dual| / (|dual|_inf + 1e-300) over all problems goes to out[0] and, per
// kind of problem, to out[1 + kind] (as bits).
__device__ __forceinline__ double hash_unit(unsigned long long k) {  // splitmix64 -> [0, 1)
  k += 0x9e3779b97f4a7c15ull;
  k = (k ^ (k >> 30)) * 0xbf58476d1ce4e5b9ull;
  k = (k ^ (k >> 27)) * 0x94d049bb133111ebull;
  k ^= k >> 31;
  return (double)(k >> 11) * (1.0 / 9007199254740992.0);
}
// the kind of face problem number i of the check (0 equal states, 1 nearby states, 2 no normal
// field, 3 field along the normal, 4 near-vacuum pressure, 5 large velocities and fields)
__device__ __forceinline__ int mode_of(unsigned long long seed, long long i) {
  return (int)(hash_unit(seed * 0x100000001b3ull + (unsigned long long)i * 64) * 6.0);
}
template <int RS>
__global__ void __launch_bounds__(128) k_vjp_check(long long n, unsigned long long seed, double gam,
                                                   unsigned long long* out) {
  const long long i = aid();
  double err = 0.0;
  if (i < n) {
    unsigned long long k = seed * 0x100000001b3ull + (unsigned long long)i * 64;
    auto u = [&]() { return hash_unit(k++); };
    const int mode = (int)(u() * 6.0);
    double WL[7], WR[7];
    const double scale = mode == 5 ? 20.0 : 2.0;
    WL[0] = 0.05 + 2.0 * u();
    WL[4] = (mode == 4 ? 1e-4 : 0.02) + 2.0 * u();
    for (int v : {1, 2, 3, 5, 6}) WL[v] = scale * (2.0 * u() - 1.0);
    for (int v = 0; v < 7; ++v) WR[v] = WL[v];
    if (mode != 0) {  // mode 0: equal states
      WR[0] = 0.05 + 2.0 * u();
      WR[4] = (mode == 4 ? 1e-4 : 0.02) + 2.0 * u();
      for (int v : {1, 2, 3, 5, 6}) WR[v] = mode == 1 ? WL[v] + 0.01 * (2.0 * u() - 1.0) : scale * (2.0 * u() - 1.0);
    }
    double bn = 2.0 * (2.0 * u() - 1.0);
    if (mode == 2) bn = 0.0;               // no normal field
    if (mode == 3) { WL[1] = 0.0; WR[1] = 0.0; WL[5] = WR[5] = 0.0; WL[6] = WR[6] = 0.0; }  // field along n
    const double lf[5] = {2 * u() - 1, 2 * u() - 1, 2 * u() - 1, 2 * u() - 1, 2 * u() - 1};
    const double lap = 2 * u() - 1, lam_ = 2 * u() - 1, lus = 2 * u() - 1;
    const double gm1inv = 1.0 / (gam - 1.0);
    double gd[15], gr[15];
    riemann_grad_dual<RS>(WL, WR, bn, gam, gm1inv, lf, lap, lam_, lus, gd);
    riemann_grad_rev<RS>(WL, WR, bn, gam, gm1inv, lf, lap, lam_, lus, gr);
    double nrm = 0.0, dif = 0.0;
    for (int v = 0; v < 15; ++v) {
      nrm = pmax(nrm, vabs(gd[v]));
      dif = pmax(dif, vabs(gr[v] - gd[v]));
    }
    err = (finite_d(nrm) && finite_d(dif)) ? dif / (nrm + 1e-300) : 1e300;
  }
  if (i < n) atomicMax(out + 1 + mode_of(seed, i), (unsigned long long)dbits(err));
  unsigned long long b = (unsigned long long)dbits(err);
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, b, o);
    b = t > b ? t : b;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(out, b);
}

void launch_vjp_check(long long n, unsigned long long seed, double gam, int rs, unsigned long long* out,
                      cudaStream_t st) {
  const unsigned nb = (unsigned)((n + 127) / 128);
  if (rs == RS_HLL) k_vjp_check<RS_HLL><<<nb, 128, 0, st>>>(n, seed, gam, out);
  else if (rs == RS_HLLD) k_vjp_check<RS_HLLD><<<nb, 128, 0, st>>>(n, seed, gam, out);
  else k_vjp_check<RS_LLF><<<nb, 128, 0, st>>>(n, seed, gam, out);
}

// ---- Joule flux eta (j x b)_d (bilinear; by hand) ----------------------------------------
// the Joule flux's adjoint on the d-face of X (weight lam): scatters into lB, returns d/d(eta)
__device__ __forceinline__ double joule_adj(const AdjDev& A, int d, long long X, double lam) {
  const Dev& D = A.D;
  const long long N = D.N;
  const int a = (d + 1) % 3, c = (d + 2) % 3;
  const double* Ba = D.Bin[a];
  const double* Bc = D.Bin[c];
  auto jedge = [&](int e, long long Y) {
    const int ae = (e + 1) % 3, ce = (e + 2) % 3;
    return (D.Bin[ce][Y] - D.Bin[ce][shift(D, Y, ae, -1)]) * D.hinv[ae] -
           (D.Bin[ae][Y] - D.Bin[ae][shift(D, Y, ce, -1)]) * D.hinv[ce];
  };
  // d j_e(Y) += w  ->  dB scatter
  auto jadj = [&](int e, long long Y, double w) {
    const int ae = (e + 1) % 3, ce = (e + 2) % 3;
    atomicAdd(&A.lB[ce * N + Y], w * D.hinv[ae]);
    atomicAdd(&A.lB[ce * N + shift(D, Y, ae, -1)], -w * D.hinv[ae]);
    atomicAdd(&A.lB[ae * N + Y], -w * D.hinv[ce]);
    atomicAdd(&A.lB[ae * N + shift(D, Y, ce, -1)], w * D.hinv[ce]);
  };
  const long long Xc = shift(D, X, c, 1), Xa = shift(D, X, a, 1), Xmd = shift(D, X, d, -1);
  const long long Xmdc = shift(D, Xmd, c, 1), Xmda = shift(D, Xmd, a, 1);
  const double ja = 0.5 * (jedge(a, X) + jedge(a, Xc)), jc = 0.5 * (jedge(c, X) + jedge(c, Xa));
  const double bcbar = 0.25 * (Bc[Xmd] + Bc[X] + Bc[Xmdc] + Bc[Xc]);
  const double babar = 0.25 * (Ba[Xmd] + Ba[X] + Ba[Xmda] + Ba[Xa]);
  // flux = eta (ja bcbar - jc babar)
  const double deta = lam * (ja * bcbar - jc * babar);
  const double wja = 0.5 * D.eta * lam * bcbar, wjc = -0.5 * D.eta * lam * babar;
  jadj(a, X, wja);
  jadj(a, Xc, wja);
  jadj(c, X, wjc);
  jadj(c, Xa, wjc);
  const double wbc = 0.25 * D.eta * lam * ja, wba = -0.25 * D.eta * lam * jc;
  atomicAdd(&A.lB[c * N + Xmd], wbc);
  atomicAdd(&A.lB[c * N + X], wbc);
  atomicAdd(&A.lB[c * N + Xmdc], wbc);
  atomicAdd(&A.lB[c * N + Xc], wbc);
  atomicAdd(&A.lB[a * N + Xmd], wba);
  atomicAdd(&A.lB[a * N + X], wba);
  atomicAdd(&A.lB[a * N + Xmda], wba);
  atomicAdd(&A.lB[a * N + Xa], wba);
  return deta;
}


__global__ void __launch_bounds__(128) k_adj_joule(AdjDev A, int d) {
  const Dev& D = A.D;
  if (!D.resistive) return;
  const long long X = aid();
  const long long N = D.N;
  const double lam = X < N ? A.lF[(5LL * d + 4) * N + X] : 0.0;
  double deta = 0.0;
  if (lam != 0.0) deta = joule_adj(A, d, X, lam);
  warp_add(deta, A.lEta);
}
// ---- face reconstructions: adjoint of the primitives --------------------------------------
template <int RC>
__global__ void __launch_bounds__(128) k_adj_face_rec(AdjDev A) {
  const Dev& D = A.D;
  const long long X = aid();
  if (X >= D.N) return;
  const long long N = D.N;
  for (int dir = 0; dir < 3; ++dir) {
    const int a = (dir + 1) % 3, c = (dir + 2) % 3;
    const int slot[7] = {0, 1 + dir, 1 + a, 1 + c, 4, 5 + a, 5 + c};
    const double* lLR = A.lLR + 14LL * dir * N;
    const long long Xn = shift(D, X, dir, 1);
    // point X's lower value = right state of face X, upper value = left state of face X + dir
    for (int v = 0; v < 7; ++v)
      rec_scatter<RC>(D, D.P + slot[v] * N, X, dir, lLR[(7 + v) * N + X], lLR[v * N + Xn], A.lP + slot[v] * N);
  }
}

// ---- primitives: adjoint of cons -> prim ------------------------------------------------
// reverse of cons -> prim (prim_from) for cell X, given the adjoints lp of its 8 primitives: adds
// the adjoints of its conserved variables to lU and returns, per direction, the adjoint of its
// cell-centred field b_d = (b_d^lo + b_d^hi) / 2 (the faces get half of it each)
__device__ __forceinline__ void prim_rev(const AdjDev& A, long long X, double* lbc) {
  const Dev& D = A.D;
  const long long N = D.N;
  double lp[8], u[5], b[3];
#pragma unroll
  for (int v = 0; v < 8; ++v) lp[v] = A.lP[v * N + X];
#pragma unroll
  for (int v = 0; v < 5; ++v) u[v] = D.Uin[v * N + X];
#pragma unroll
  for (int d = 0; d < 3; ++d) b[d] = 0.5 * (D.Bin[d][X] + D.Bin[d][shift(D, X, d, 1)]);
  const double rho = u[0], rinv = rcp(rho);
  const double ui[3] = {u[1] * rinv, u[2] * rinv, u[3] * rinv};
  const double u2s = fma(ui[0], ui[0], fma(ui[1], ui[1], ui[2] * ui[2]));
  const double leint = (D.gam - 1.0) * lp[4];        // p = (gamma - 1) eint
  const double lq = -0.5 * leint;                     // eint = e - (rho u2s + b2s) / 2
  double lrinv = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double lu = fma(2.0 * ui[i], lq * rho, lp[1 + i]);  // u_i directly and through u2s
    A.lU[(1 + i) * N + X] += lu * rinv;                       // u_i = m_i / rho
    lrinv = fma(lu, u[1 + i], lrinv);
  }
  A.lU[4 * N + X] += leint;
  A.lU[0 * N + X] += fma(lq, u2s, lp[0]) - lrinv * rinv * rinv;  // rho directly, via u2s, via 1/rho
#pragma unroll
  for (int d = 0; d < 3; ++d) lbc[d] = fma(2.0 * b[d], lq, lp[5 + d]);
}

// adjoint of cons -> prim, by hand: each thread owns cell X's conserved adjoints and the lower
// d-face of X, which gets half of the cell-centred field adjoint of X and of X - d (no atomics)
__global__ void __launch_bounds__(128) k_adj_prim(AdjDev A) {
  const Dev& D = A.D;
  const long long X = aid();
  if (X >= D.N) return;
  const long long N = D.N;
  double lbc[3];
  prim_rev(A, X, lbc);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    // the same quantity for cell X - d (its upper d-face is X's lower one)
    const long long Xm = shift(D, X, d, -1);
    const double bm = 0.5 * (D.Bin[d][Xm] + D.Bin[d][X]);
    const double lqm = -0.5 * ((D.gam - 1.0) * A.lP[4 * N + Xm]);
    const double lbm = fma(2.0 * bm, lqm, A.lP[(5 + d) * N + Xm]);
    A.lB[d * N + X] += 0.5 * (lbc[d] + lbm);
  }
}

// ---- update: lF, lE = D^T lam (Eqs. rk:increment-state, rk:increment-bfield) ---------------
// lF = s_old * lF + scale * D^T(lU, lB) (and lE likewise): s_old = 0 overwrites.
__global__ void __launch_bounds__(256) k_adj_update(Dev D, const double* lU, const double* lB, double* lF,
                                                    double* lE, double scale, double s_old) {
  const long long X = aid();
  if (X >= D.N) return;
  const long long N = D.N;
  for (int d = 0; d < 3; ++d) {
    const long long Xm = shift(D, X, d, -1);
    const double k = scale * D.dt * D.hinv[d];
    for (int v = 0; v < 5; ++v) {
      const double g = k * (lU[v * N + X] - lU[v * N + Xm]);
      double* t = &lF[(5LL * d + v) * N + X];
      *t = s_old == 0.0 ? g : fma(s_old, *t, g);
    }
  }
  for (int e = 0; e < 3; ++e) {
    // E_e enters B_{e+1} as its "c" EMF and B_{e+2} as its "a" EMF (see face_new)
    const int d1 = (e + 1) % 3, a1 = (d1 + 1) % 3;  // B_d1[Y]: +dt/h_a1 E_e[Y] - dt/h_a1 E_e[Y + a1]
    const int d2 = (e + 2) % 3, c2 = (d2 + 2) % 3;  // B_d2[Y]: -dt/h_c2 E_e[Y] + dt/h_c2 E_e[Y + c2]
    const double g = scale * D.dt *
                     ((lB[d1 * N + X] - lB[d1 * N + shift(D, X, a1, -1)]) * D.hinv[a1] +
                      (lB[d2 * N + shift(D, X, c2, -1)] - lB[d2 * N + X]) * D.hinv[c2]);
    double* t = &lE[e * N + X];
    *t = s_old == 0.0 ? g : fma(s_old, *t, g);
  }
}

// ---- first-order flux correction (Sec. 2.5): masks and the adjoint of the first-order fluxes ---
// With the masks M1, M2 of the cells flagged after stage 1 and stage 2 frozen, the step is
//   F1 = M1 FO(S^n) + (1 - M1) HO(S^n),        S^{n+1/2} = S^n + D F1,
//   F2 = M2 FO(S^n) + (1 - M2) (F1 + HO(S^{n+1/2})) / 2,   S^{n+1} = S^n + D F2,
// for the face fluxes and edge EMFs alike (a face is masked when one of its two cells is flagged,
// an edge when one of its four cells is). Its transpose, for g = D^T lam: the stage-2 flux
// function gets (1 - M2) g / 2, F1 gets k = (1 - M2) g / 2 + D^T lam_{n+1/2}, HO(S^n) gets
// (1 - M1) k and FO(S^n) gets M2 g + M1 k.
__device__ __forceinline__ bool face_masked(const Dev& D, const unsigned char* fl, int d, long long X) {
  return fl[X] || fl[shift(D, X, d, -1)];
}
__device__ __forceinline__ bool edge_masked(const Dev& D, const unsigned char* fl, int e, long long X) {
  const int a = (e + 1) % 3, c = (e + 2) % 3;
  const long long Xa = shift(D, X, a, -1);
  return fl[X] || fl[Xa] || fl[shift(D, X, c, -1)] || fl[shift(D, Xa, c, -1)];
}
// lF, lE <- scale g on faces and edges outside the mask of `fl`, 0 inside
__global__ void __launch_bounds__(256) k_adj_mask(Dev D, const unsigned char* fl, const double* gF,
                                                  const double* gE, double* lF, double* lE, double scale) {
  const long long X = aid();
  if (X >= D.N) return;
  const long long N = D.N;
  for (int d = 0; d < 3; ++d) {
    const bool m = face_masked(D, fl, d, X);
    for (int v = 0; v < 5; ++v) lF[(5LL * d + v) * N + X] = m ? 0.0 : scale * gF[(5LL * d + v) * N + X];
    lE[d * N + X] = edge_masked(D, fl, d, X) ? 0.0 : scale * gE[d * N + X];
  }
}

// adds the adjoint of cons -> prim (prim_from) of cell Y of S^n, given its 8 primitives' adjoints
// lp, to lU (conserved variables) and lB (the cell's six faces): atomics, since several first-order
// faces share a cell
__device__ __forceinline__ void prim_vjp_atomic(const AdjDev& A, long long Y, const double* lp) {
  const Dev& D = A.D;
  const long long N = D.N;
  double u[5], lo[3], hi[3];
  load_cell(D, D.U0, D.B0, Y, u, lo, hi);
  const double rho = u[0], rinv = rcp(rho);
  const double ui[3] = {u[1] * rinv, u[2] * rinv, u[3] * rinv};
  const double u2s = fma(ui[0], ui[0], fma(ui[1], ui[1], ui[2] * ui[2]));
  const double leint = (D.gam - 1.0) * lp[4];  // p = (gamma - 1) eint
  const double lq = -0.5 * leint;               // eint = e - (rho u2s + b2s) / 2
  double lrinv = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double lu = fma(2.0 * ui[i], lq * rho, lp[1 + i]);
    atomicAdd(&A.lU[(1 + i) * N + Y], lu * rinv);
    lrinv = fma(lu, u[1 + i], lrinv);
  }
  atomicAdd(&A.lU[4 * N + Y], leint);
  atomicAdd(&A.lU[0 * N + Y], fma(lq, u2s, lp[0]) - lrinv * rinv * rinv);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double lb = 0.5 * fma(2.0 * halve(lo[d] + hi[d]), lq, lp[5 + d]);
    atomicAdd(&A.lB[d * N + Y], lb);
    atomicAdd(&A.lB[d * N + shift(D, Y, d, 1)], lb);
  }
}

// adjoint of the first-order (piecewise-constant + LLF) face problem on the d-face between cells
// Xl and Xr of S^n, with weights lf (flux, face frame), lap (alpha) and lus (u*)
__device__ __forceinline__ void fo_face_vjp(const AdjDev& A, int d, long long Xl, long long Xr, const double* lf,
                                            double lap, double lus) {
  const Dev& D = A.D;
  const int a = (d + 1) % 3, c = (d + 2) % 3;
  double wl[8], wr[8];
  prim_of(D, D.U0, D.B0, Xl, wl);
  prim_of(D, D.U0, D.B0, Xr, wr);
  const FaceState sl = {wl[0], wl[1 + d], wl[1 + a], wl[1 + c], wl[4], wl[5 + a], wl[5 + c]};
  const FaceState sr = {wr[0], wr[1 + d], wr[1 + a], wr[1 + c], wr[4], wr[5 + a], wr[5 + c]};
  FaceState dl, dr;
  double dbn;
  riemann_vjp<RS_LLF>(sl, sr, D.B0[d][Xr], D.gam, D.gm1inv, lf, lap, 0.0, lus, dl, dr, dbn);
  const FaceState* ds[2] = {&dl, &dr};
  const long long cells[2] = {Xl, Xr};
  for (int k = 0; k < 2; ++k) {
    double lp[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    lp[0] = ds[k]->rho;
    lp[1 + d] = ds[k]->u;
    lp[1 + a] = ds[k]->v;
    lp[1 + c] = ds[k]->w;
    lp[4] = ds[k]->p;
    lp[5 + a] = ds[k]->by;
    lp[5 + c] = ds[k]->bz;
    prim_vjp_atomic(A, cells[k], lp);
  }
  atomicAdd(&A.lB[d * D.N + Xr], dbn);
}

// Adjoint of the first-order fluxes and EMFs of S^n on masked faces and edges: weights
// M2 gF + M1 kF (faces) and M2 gE + M1 kE (edges), fl1 / fl2 the flags after stage 1 / 2. Adds to
// lU, lB (of S^n) and lEta. Exits at once when neither stage flagged a cell.
__global__ void __launch_bounds__(128) k_adj_fo(AdjDev A, const unsigned char* fl1, const unsigned char* fl2,
                                                const double* gF, const double* gE, const double* kF,
                                                const double* kE) {
  const Dev& D = A.D;
  if (*(volatile const unsigned long long*)(D.counters + 0) == 0 &&
      *(volatile const unsigned long long*)(D.counters + 1) == 0)
    return;
  const long long N = D.N;
  double etaacc = 0.0;
  for (long long X0 = (long long)blockIdx.x * blockDim.x; X0 < N; X0 += (long long)gridDim.x * blockDim.x) {
    const long long X = X0 + threadIdx.x;  // the warp stays together for warp_add below
    if (X < N) {
      for (int d = 0; d < 3; ++d) {
        const bool m1 = face_masked(D, fl1, d, X), m2 = face_masked(D, fl2, d, X);
        if (!(m1 || m2)) continue;
        const int a = (d + 1) % 3, c = (d + 2) % 3;
        double w[5];
        for (int v = 0; v < 5; ++v) {
          const long long I = (5LL * d + v) * N + X;
          w[v] = (m2 ? gF[I] : 0.0) + (m1 ? kF[I] : 0.0);
        }
        const double lf[5] = {w[0], w[1 + d], w[1 + a], w[1 + c], w[4]};
        fo_face_vjp(A, d, shift(D, X, d, -1), X, lf, 0.0, 0.0);
        if (D.resistive && w[4] != 0.0) etaacc += joule_adj(A, d, X, w[4]);  // the Joule flux from S^n
      }
      for (int e = 0; e < 3; ++e) {
        const bool m1 = edge_masked(D, fl1, e, X), m2 = edge_masked(D, fl2, e, X);
        if (!(m1 || m2)) continue;
        const double lam = (m2 ? gE[e * N + X] : 0.0) + (m1 ? kE[e * N + X] : 0.0);
        if (lam == 0.0) continue;
        const int a = (e + 1) % 3, c = (e + 2) % 3;
        const long long Xa = shift(D, X, a, -1), Xc = shift(D, X, c, -1), Xac = shift(D, Xa, c, -1);
        // the first-order edge EMF (corners of piecewise-constant values, LD04 with the LLF speeds)
        // as fo_edges_cell forms it: the four faces' alpha and u*, recomputed
        double f[5], apaB, apaT, apcL, apcR, uaB, uaT, ucL, ucR;
        fo_face(D, a, Xac, Xc, Xc, f, apaB, uaB);
        fo_face(D, a, Xa, X, X, f, apaT, uaT);
        fo_face(D, c, Xac, Xa, Xa, f, apcL, ucL);
        fo_face(D, c, Xc, X, X, f, apcR, ucR);
        const bool pickB = dbits(apaB) >= dbits(apaT), pickL = dbits(apcL) >= dbits(apcR);  // pmax
        const double apa = pickB ? apaB : apaT, apc = pickL ? apcL : apcR;
        const double baB = D.B0[a][Xc], baT = D.B0[a][X], bcL = D.B0[c][Xa], bcR = D.B0[c][X];
        double dba[2], dbc[2], dapa, dapc, dua[2] = {0.0, 0.0}, duc[2] = {0.0, 0.0};
        if (D.emf != EMF_Q26) {
          // piecewise-constant FS18 / B25a: corner q takes the velocity of the cell in that corner
          // (LB = X-a-c, RB = X-c, LT = X-a, RT = X), and FS18 the face fields of the edge, B25a
          // the cell's field (the mean of its two faces)
          const bool b25 = D.emf == EMF_B25A;
          const long long cellQ[4] = {Xac, Xc, Xa, X};
          double ua[4], uc[4], ri[4], e4[4], bas[4], bcs[4];
          for (int q = 0; q < 4; ++q) {
            const long long Q = cellQ[q];
            ri[q] = rcp(D.U0[Q]);
            ua[q] = D.U0[(1 + a) * N + Q] * ri[q];
            uc[q] = D.U0[(1 + c) * N + Q] * ri[q];
            bcs[q] = b25 ? halve(D.B0[c][Q] + D.B0[c][shift(D, Q, c, 1)]) : ((q & 1) ? bcR : bcL);
            bas[q] = b25 ? halve(D.B0[a][Q] + D.B0[a][shift(D, Q, a, 1)]) : ((q >> 1) ? baT : baB);
            e4[q] = fma(-ua[q], bcs[q], uc[q] * bas[q]);
          }
          double de[4], db[4], dal[4];
          ld04_vjp(apa, apa, apc, apc, e4, baB, baT, bcL, bcR, lam, de, db, dal);
          dba[0] = db[0]; dba[1] = db[1]; dbc[0] = db[2]; dbc[1] = db[3];
          dapa = dal[0] + dal[1];
          dapc = dal[2] + dal[3];
          for (int q = 0; q < 4; ++q) {
            const long long Q = cellQ[q];
            const double dva = -de[q] * bcs[q], dvc = de[q] * bas[q];
            if (b25) {  // the cell field b_k = (B_k[Q] + B_k[Q + k]) / 2
              const double hc = -0.5 * de[q] * ua[q], ha = 0.5 * de[q] * uc[q];
              atomicAdd(&A.lB[c * N + Q], hc);
              atomicAdd(&A.lB[c * N + shift(D, Q, c, 1)], hc);
              atomicAdd(&A.lB[a * N + Q], ha);
              atomicAdd(&A.lB[a * N + shift(D, Q, a, 1)], ha);
            } else {
              dbc[q & 1] -= de[q] * ua[q];
              dba[q >> 1] += de[q] * uc[q];
            }
            // u = m / rho
            atomicAdd(&A.lU[(1 + a) * N + Q], dva * ri[q]);
            atomicAdd(&A.lU[(1 + c) * N + Q], dvc * ri[q]);
            atomicAdd(&A.lU[Q], -fma(dva, ua[q], dvc * uc[q]) * ri[q]);
          }
        } else {
          const double in[12] = {baB, baT, uaB, uaT, bcL, bcR, ucL, ucR, apa, apa, apc, apc};
          double g[12];
          q26_edge_vjp(in, lam, g);
          dapa = g[8] + g[9];
          dapc = g[10] + g[11];
          dba[0] = g[0]; dba[1] = g[1]; dbc[0] = g[4]; dbc[1] = g[5];
          dua[0] = g[2]; dua[1] = g[3]; duc[0] = g[6]; duc[1] = g[7];
        }
        const double z[5] = {0, 0, 0, 0, 0};
        fo_face_vjp(A, a, Xac, Xc, z, pickB ? dapa : 0.0, dua[0]);
        fo_face_vjp(A, a, Xa, X, z, pickB ? 0.0 : dapa, dua[1]);
        fo_face_vjp(A, c, Xac, Xa, z, pickL ? dapc : 0.0, duc[0]);
        fo_face_vjp(A, c, Xc, X, z, pickL ? 0.0 : dapc, duc[1]);
        atomicAdd(&A.lB[a * N + Xc], dba[0]);
        atomicAdd(&A.lB[a * N + X], dba[1]);
        atomicAdd(&A.lB[c * N + Xa], dbc[0]);
        atomicAdd(&A.lB[c * N + X], dbc[1]);
        if (D.resistive) {  // + eta j from S^n
          const double j = (D.B0[c][X] - D.B0[c][Xa]) * D.hinv[a] - (D.B0[a][X] - D.B0[a][Xc]) * D.hinv[c];
          etaacc += lam * j;
          const double la = D.eta * lam * D.hinv[a], lc = D.eta * lam * D.hinv[c];
          atomicAdd(&A.lB[c * N + X], la);
          atomicAdd(&A.lB[c * N + Xa], -la);
          atomicAdd(&A.lB[a * N + X], -lc);
          atomicAdd(&A.lB[a * N + Xc], lc);
        }
      }
    }
    warp_add(etaacc, A.lEta);
    etaacc = 0.0;
  }
}

void launch_adj_mask(const Dev& D, const unsigned char* fl, const double* gF, const double* gE, double* lF,
                     double* lE, double scale, cudaStream_t st) {
  k_adj_mask<<<(unsigned)((D.N + 255) / 256), 256, 0, st>>>(D, fl, gF, gE, lF, lE, scale);
}
void launch_adj_fo(const AdjDev& A, const unsigned char* fl1, const unsigned char* fl2, const double* gF,
                   const double* gE, const double* kF, const double* kE, cudaStream_t st) {
  const long long nb = (A.D.N + 127) / 128;
  k_adj_fo<<<(unsigned)(nb < 1184 ? nb : 1184), 128, 0, st>>>(A, fl1, fl2, gF, gE, kF, kE);
}

// reverse sweeps of the PPM reconstructions along each direction (one launch per direction, so
// that every output element has one writer per launch); KIND 0 the edge values, 1 the face states,
// 2 B25a's cell EMF
template <int KIND, int EMF = EMF_Q26>
static void rec_sweeps(const AdjDev& A, cudaStream_t st) {
  const int nsrc = KIND == 1 ? 7 : (KIND == 2 ? 2 : (EMF == EMF_FS18 ? 10 : (EMF == EMF_B25A ? 6 : 4)));
  for (int s = 0; s < 3; ++s) {
    const int seg = 32;
    const long long n = sweep_threads(A.D, s, seg) * nsrc;
    k_adj_rec_sweep<KIND, EMF><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(A, s, seg);
  }
}

// B25a: the cell EMF of the stage input, eps_e = -u_a b_c + u_c b_a from its primitives (as the
// forward cell-to-face sweeps form it)
__global__ void __launch_bounds__(256) k_adj_eps_prep(AdjDev A) {
  const long long X = aid();
  const Dev& D = A.D;
  if (X >= D.N) return;
  const long long N = D.N;
  for (int e = 0; e < 3; ++e) {
    const int a = (e + 1) % 3, c = (e + 2) % 3;
    A.eps[e * N + X] = fma(-D.P[(1 + a) * N + X], D.P[(5 + c) * N + X], D.P[(1 + c) * N + X] * D.P[(5 + a) * N + X]);
  }
}
// point-wise reverse of the cell-EMF reconstructions (PC, PLM, PPM-EP)
template <int RC>
__global__ void __launch_bounds__(128) k_adj_eps_rec(AdjDev A) {
  const Dev& D = A.D;
  const long long X = aid();
  if (X >= D.N) return;
  const long long N = D.N;
  for (int e = 0; e < 3; ++e) {
    const int a = (e + 1) % 3, c = (e + 2) % 3;
    const double* lfL = A.lEf + 2LL * e * N;
    const double* lfB = A.lEf + 6 * N + 2LL * e * N;
    rec_scatter<RC>(D, A.eps + e * N, X, a, lfL[N + X], lfL[shift(D, X, a, 1)], A.leps + e * N);
    rec_scatter<RC>(D, A.eps + e * N, X, c, lfB[N + X], lfB[shift(D, X, c, 1)], A.leps + e * N);
  }
}
// the cell EMF's adjoint into the primitives' (one thread per cell, no other writer meanwhile)
__global__ void __launch_bounds__(256) k_adj_eps_to_prim(AdjDev A) {
  const long long X = aid();
  const Dev& D = A.D;
  if (X >= D.N) return;
  const long long N = D.N;
  for (int e = 0; e < 3; ++e) {
    const int a = (e + 1) % 3, c = (e + 2) % 3;
    const double l = A.leps[e * N + X];
    if (l == 0.0) continue;
    A.lP[(1 + a) * N + X] -= l * D.P[(5 + c) * N + X];
    A.lP[(5 + c) * N + X] -= l * D.P[(1 + a) * N + X];
    A.lP[(1 + c) * N + X] += l * D.P[(5 + a) * N + X];
    A.lP[(5 + a) * N + X] += l * D.P[(1 + c) * N + X];
  }
}

template <int RC, int EMF>
static void adj_edges_t(const AdjDev& A, cudaStream_t st) {
  const unsigned nb = (unsigned)((A.D.N + 127) / 128), nb256 = (unsigned)((A.D.N + 255) / 256);
  if (EMF == EMF_B25A) {
    cudaMemsetAsync(A.lEf, 0, 12 * A.D.N * sizeof(double), st);
    cudaMemsetAsync(A.leps, 0, 3 * A.D.N * sizeof(double), st);
    k_adj_eps_prep<<<nb256, 256, 0, st>>>(A);
  }
  k_adj_edges<RC, EMF><<<nb, 128, 0, st>>>(A);
  if (RC == REC_PPM) rec_sweeps<0, EMF>(A, st);
  else k_adj_edge_rec<RC, EMF><<<nb, 128, 0, st>>>(A);
  if (EMF == EMF_B25A) {  // the face EMF values back to the cell EMF, then to the primitives
    if (RC == REC_PPM) rec_sweeps<2>(A, st);
    else k_adj_eps_rec<RC><<<nb, 128, 0, st>>>(A);
    k_adj_eps_to_prim<<<nb256, 256, 0, st>>>(A);
  }
}

template <int RC>
static void adj_flux_r(const AdjDev& A, int rs, cudaStream_t st) {
  const unsigned nb = (unsigned)((A.D.N + 127) / 128);
  // the face-state adjoints accumulate (FS18's edge reconstructions of the face velocity states
  // add to them, then the face solve's reverse sweep)
  cudaMemsetAsync(A.lLR, 0, 42 * A.D.N * sizeof(double), st);
  if (A.D.emf == EMF_FS18) adj_edges_t<RC, EMF_FS18>(A, st);
  else if (A.D.emf == EMF_B25A) adj_edges_t<RC, EMF_B25A>(A, st);
  else adj_edges_t<RC, EMF_Q26>(A, st);
  for (int dir = 0; dir < 3; ++dir) {
    if (rs == RS_HLL) k_adj_faces<RC, RS_HLL><<<nb, 128, 0, st>>>(A, dir);
    else if (rs == RS_HLLD) k_adj_faces<RC, RS_HLLD><<<nb, 128, 0, st>>>(A, dir);
    else k_adj_faces<RC, RS_LLF><<<nb, 128, 0, st>>>(A, dir);
    if (A.D.resistive) k_adj_joule<<<nb, 128, 0, st>>>(A, dir);
  }
  if (RC == REC_PPM) rec_sweeps<1>(A, st);
  else k_adj_face_rec<RC><<<nb, 128, 0, st>>>(A);
  k_adj_prim<<<nb, 128, 0, st>>>(A);
}

// adjoint of the flux function at A.D's stage input (its P, Ap, Am, Us must be current)
void launch_adj_flux(const AdjDev& A, int recon, int rs, cudaStream_t st) {
  switch (recon) {
    case REC_PC: adj_flux_r<REC_PC>(A, rs, st); break;
    case REC_PLM_MC: adj_flux_r<REC_PLM_MC>(A, rs, st); break;
    case REC_PLM_MINMOD: adj_flux_r<REC_PLM_MINMOD>(A, rs, st); break;
    case REC_PPM: adj_flux_r<REC_PPM>(A, rs, st); break;
    default: adj_flux_r<REC_PPM_EP>(A, rs, st); break;
  }
}

void launch_adj_update(const Dev& D, const double* lU, const double* lB, double* lF, double* lE, double scale,
                       double s_old, cudaStream_t st) {
  k_adj_update<<<(unsigned)((D.N + 255) / 256), 256, 0, st>>>(D, lU, lB, lF, lE, scale, s_old);
}

__global__ void k_axpy3(long long n, double* y, const double* a, const double* b) {
  const long long i = aid();
  if (i < n) y[i] += a[i] + b[i];
}
void launch_axpy3(long long n, double* y, const double* a, const double* b, cudaStream_t st) {
  k_axpy3<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, y, a, b);
}

}  // namespace mhd
