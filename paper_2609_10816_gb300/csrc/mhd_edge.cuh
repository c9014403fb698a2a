// mhd_edge.cuh -- edge EMFs (Sec. 2.3-2.4): reconstruction of face fields and face velocities to
// the edges (Fig. b-common, Eqs. q26, fs18, b25a-*), the edge wavespeeds (Eq. alpha-edge), the
// LD04 average (Eq. ld04) and the Ohmic term (Eqs. current-stencil, emf-update).
//
// For an e-edge with a = e+1, c = e+2 (cyclic), the a-face quantities are reconstructed along c
// (bottom/top states) and the c-face quantities along a (left/right states). Two sweeps do this
// without recomputation: edge_bt_seg walks lines along c and stores the bottom/top values per
// edge; edge_lr_seg walks lines along a, forms the left/right values and finishes the EMF.
#pragma once
#include "mhd_device.cuh"
#include "mhd_index.cuh"
#include "mhd_internal.cuh"

namespace mhd {

// Sources reconstructed along c on the a-faces of e-edges, per EMF compute scheme, and where
// their bottom/top values go. Q26: b_a and u_a^* (Eq. q26); FS18: b_a and the left/right states
// of u_a and u_c on the a-faces (order "a then c" of Eq. fs18-average); B25a: b_a and the
// left/right values of the cell EMF on the a-faces (order "a then c" of Eq. b25a-average).
template <int EMF> struct BtSrc {
  static constexpr int NV = EMF == EMF_Q26 ? 2 : (EMF == EMF_FS18 ? 5 : 3);
  __device__ static void get(const Dev& D, int e, const double** src, double** dst) {
    const int a = (e + 1) % 3, c = (e + 2) % 3;
    const long long N = D.N;
    double* ep = D.Epart + 4LL * e * N;
    double* xp = D.Xpart + 8LL * e * N;
    src[0] = D.Bin[a];
    dst[0] = ep;
    dst[1] = ep + N;
    if (EMF == EMF_Q26) {
      src[1] = D.Us + a * N;
      dst[2] = ep + 2 * N;
      dst[3] = ep + 3 * N;
    } else if (EMF == EMF_FS18) {
      // (u_a L, u_a R, u_c L, u_c R) on a-faces -> Xpart slots 2v-2, 2v-1 = (B, T)
      src[1] = D.VL + (3LL * a + a) * N;
      src[2] = D.VR + (3LL * a + a) * N;
      src[3] = D.VL + (3LL * a + c) * N;
      src[4] = D.VR + (3LL * a + c) * N;
      for (int v = 1; v < 5; ++v) {
        dst[2 * v] = xp + (2 * v - 2) * N;
        dst[2 * v + 1] = xp + (2 * v - 1) * N;
      }
    } else {
      src[1] = D.EfL + (2LL * e + 0) * N;  // cell EMF, left value on the a-face
      src[2] = D.EfL + (2LL * e + 1) * N;  // right value
      for (int v = 1; v < 3; ++v) {
        dst[2 * v] = xp + (2 * v - 2) * N;
        dst[2 * v + 1] = xp + (2 * v - 1) * N;
      }
    }
  }
};

template <int RC, int EMF>
__device__ __forceinline__ void edge_bt_seg(const Dev& D, int e, const Line& ln, int m0, int m1) {
  constexpr int NV = BtSrc<EMF>::NV;
  const double* q[NV];
  double* out[2 * NV];
  BtSrc<EMF>::get(D, e, q, out);
  constexpr int LB = Rec<RC>::LB, LA = Rec<RC>::LA;
  Rec<RC> r[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double w[LB + LA];
#pragma unroll
    for (int t = 0; t < LB + LA; ++t) w[t] = q[v][ln.at(m0 - LB + t)];
    r[v].init(w);
  }
  // the next point's values are loaded one iteration ahead (this sweep does little arithmetic per
  // point, so the loads' latency would otherwise stall it)
  double nxt[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) nxt[v] = q[v][ln.at(m0 + LA)];
  for (int m = m0; m < m1; ++m) {
    const long long X = ln.at(m);
    double cur[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) cur[v] = nxt[v];
    if (m + 1 < m1) {
      const long long Xn = ln.at(m + 1 + LA);
#pragma unroll
      for (int v = 0; v < NV; ++v) nxt[v] = q[v][Xn];
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      double B, T;
      r[v].step(cur[v], B, T);
      out[2 * v][X] = B;
      out[2 * v + 1][X] = T;
    }
  }
}

// B25a, first reconstruction of the cell-centred EMF eps_e = -u_a b_c + u_c b_a
// (Eqs. b25a-b-avg, b25a-emf-centre) to faces: along a (to a-faces, left/right) when `to_a`,
// else along c (to c-faces, bottom/top).
template <int RC>
__device__ __forceinline__ void b25_seg(const Dev& D, int e, int to_a, const Line& ln, int m0, int m1) {
  const int a = (e + 1) % 3, c = (e + 2) % 3;
  const long long N = D.N;
  const double* ua = D.P + (1 + a) * N;
  const double* uc = D.P + (1 + c) * N;
  const double* ba = D.P + (5 + a) * N;
  const double* bc = D.P + (5 + c) * N;
  auto eps = [&](long long Y) { return fma(-ua[Y], bc[Y], uc[Y] * ba[Y]); };
  double* out = (to_a ? D.EfL : D.EfB) + 2LL * e * N;
  constexpr int LB = Rec<RC>::LB, LA = Rec<RC>::LA;
  Rec<RC> r;
  double w[LB + LA];
#pragma unroll
  for (int t = 0; t < LB + LA; ++t) w[t] = eps(ln.at(m0 - LB + t));
  r.init(w);
  for (int m = m0; m < m1; ++m) {
    const long long X = ln.at(m);
    double lo, hi;
    r.step(eps(ln.at(m + LA)), lo, hi);
    out[X] = lo;
    out[N + X] = hi;
  }
}

// Eq. (ld04) with the edge speeds of Eq. (alpha-edge), plus eta j (Eq. emf-update).
template <class T>
__device__ __forceinline__ T ld04(T apa, T ama, T apc, T amc, T eLB, T eRB, T eLT, T eRT, T baB, T baT, T bcL,
                                  T bcR) {
  const T sa = apa + ama, sc = apc + amc;
  const T w = rcp(sa * sc);  // one reciprocal gives 1/sa, 1/sc and their product
  const T ia = sc * w, ic = sa * w;
  const T up = fma(apc, fma(apa, eLB, ama * eRB), amc * fma(apa, eLT, ama * eRT)) * w;
  return fma(apa * ama * ia, bcR - bcL, fma(-apc * amc * ic, baT - baB, up));
}

// Q26 corner EMFs (Eq. q26) and their LD04 average, as a function of its 12 inputs. The corner
// EMF -u_a^{S_II} b_c^{S_I} + u_c^{S_I} b_a^{S_II} is bilinear, so the alpha-weighted sums of
// Eq. (ld04) factor through the two weighted sums BC, UC of the c-face values:
//   apa e_LB + ama e_RB = -u_a^B BC + b_a^B UC, and likewise on the top side
// (same value as forming the four corners, four fewer operations).
template <class T>
__device__ __forceinline__ T q26_edge_emf(T baB, T baT, T uaB, T uaT, T bcL, T bcR, T ucL, T ucR, T apa, T ama,
                                          T apc, T amc) {
  const T sa = apa + ama, sc = apc + amc;
  const T w = rcp(sa * sc);
  const T BC = fma(apa, bcL, ama * bcR), UC = fma(apa, ucL, ama * ucR);
  const T hB = fma(-uaB, BC, baB * UC), hT = fma(-uaT, BC, baT * UC);
  const T up = fma(apc, hB, amc * hT);
  return fma(apa * ama * sc, bcR - bcL, fma(-(apc * amc * sa), baT - baB, up)) * w;
}

// Sources reconstructed along a on the c-faces of e-edges (their left/right values), per scheme:
// Q26: b_c and u_c^*; FS18: b_c and the bottom/top states of u_a and u_c on the c-faces (order
// "c then a"); B25a: b_c and the bottom/top values of the cell EMF on the c-faces.
template <int EMF> struct LrSrc {
  static constexpr int NV = EMF == EMF_Q26 ? 2 : (EMF == EMF_FS18 ? 5 : 3);
  __device__ static void get(const Dev& D, int e, const double** src) {
    const int a = (e + 1) % 3, c = (e + 2) % 3;
    const long long N = D.N;
    src[0] = D.Bin[c];
    if (EMF == EMF_Q26) {
      src[1] = D.Us + c * N;
    } else if (EMF == EMF_FS18) {
      src[1] = D.VL + (3LL * c + a) * N;  // u_a, bottom state on the c-face
      src[2] = D.VR + (3LL * c + a) * N;  // u_a, top
      src[3] = D.VL + (3LL * c + c) * N;  // u_c, bottom
      src[4] = D.VR + (3LL * c + c) * N;  // u_c, top
    } else {
      src[1] = D.EfB + (2LL * e + 0) * N;
      src[2] = D.EfB + (2LL * e + 1) * N;
    }
  }
};

template <int RC, int EMF>
__device__ __forceinline__ void edge_lr_seg(const Dev& D, int e, const Line& ln, int m0, int m1) {
  const int a = (e + 1) % 3, c = (e + 2) % 3;
  const long long N = D.N;
  constexpr int NV = LrSrc<EMF>::NV;
  const double* q[NV];
  LrSrc<EMF>::get(D, e, q);
  constexpr int LB = Rec<RC>::LB, LA = Rec<RC>::LA;
  Rec<RC> r[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double w[LB + LA];
#pragma unroll
    for (int t = 0; t < LB + LA; ++t) w[t] = q[v][ln.at(m0 - LB + t)];
    r[v].init(w);
  }
  const double* part = D.Epart + 4LL * e * N;
  const double* xp = D.Xpart + 8LL * e * N;
  const double* Apa = D.Ap + a * N;
  const double* Ama = D.Am + a * N;
  const double* Apc = D.Ap + c * N;
  const double* Amc = D.Am + c * N;
  const double* Ba = D.Bin[a];
  const double* Bc = D.Bin[c];
  double* E = D.E + e * N;
  for (int m = m0; m < m1; ++m) {
    const long long X = ln.at(m);
    const long long Xa = ln.at(m - 1);  // X - a
    const long long Xc = shift(D, X, c, -1);
    const long long Xn = ln.at(m + LA);
    double lo[NV], hi[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) r[v].step(q[v][Xn], lo[v], hi[v]);
    const double bcL = lo[0], bcR = hi[0];
    const double baB = part[0 * N + X], baT = part[1 * N + X];
    // Eq. (alpha-edge): alpha_a from the two a-faces (c-neighbours), alpha_c from the c-faces
    const double apa = pmax(Apa[Xc], Apa[X]), ama = pmax(Ama[Xc], Ama[X]);
    const double apc = pmax(Apc[Xa], Apc[X]), amc = pmax(Amc[Xa], Amc[X]);
    double emf;
    double eLB, eRB, eLT, eRT;
    if (EMF == EMF_Q26) {
      // Eq. (q26) corners and Eq. (ld04), factored
      emf = q26_edge_emf(baB, baT, part[2 * N + X], part[3 * N + X], bcL, bcR, lo[1], hi[1], apa, ama, apc, amc);
      if (D.EdgeC) {
        double* ec = D.EdgeC + 4LL * e * N;
        ec[X] = bcL;
        ec[N + X] = bcR;
        ec[2 * N + X] = lo[1];
        ec[3 * N + X] = hi[1];
      }
    } else if (EMF == EMF_FS18) {
      // Eq. (fs18-average): mean of the two reconstruction orders per corner, then Eq. (fs18).
      // order a-then-c partials: slot 2k' + ... = (u_a L:B,T, u_a R:B,T, u_c L:B,T, u_c R:B,T)
      // order c-then-a: lo/hi[1] = u_a B:(L,R), [2] = u_a T:(L,R), [3] = u_c B, [4] = u_c T
      double ua[4], uc[4];  // corner q = sI + 2 sII: LB, RB, LT, RT
#pragma unroll
      for (int qq = 0; qq < 4; ++qq) {
        const int sI = qq & 1, sII = qq >> 1;
        const double o1a = xp[(2 * sI + sII) * N + X];
        const double o1c = xp[(4 + 2 * sI + sII) * N + X];
        const double o2a = sI ? hi[1 + sII] : lo[1 + sII];
        const double o2c = sI ? hi[3 + sII] : lo[3 + sII];
        ua[qq] = halve(o1a + o2a);
        uc[qq] = halve(o1c + o2c);
      }
      eLB = fma(-ua[0], bcL, uc[0] * baB);
      eRB = fma(-ua[1], bcR, uc[1] * baB);
      eLT = fma(-ua[2], bcL, uc[2] * baT);
      eRT = fma(-ua[3], bcR, uc[3] * baT);
      if (D.EdgeC) {  // the left/right values, for the adjoint (b_c, then lo/hi of the 4 states)
        double* ec = D.EdgeC + 10LL * e * N;
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          ec[(2 * v) * N + X] = lo[v];
          ec[(2 * v + 1) * N + X] = hi[v];
        }
      }
    } else {
      // Eq. (b25a-average): a-then-c partials (eps L:B,T, eps R:B,T); c-then-a lo/hi[1] = B:(L,R),
      // [2] = T:(L,R)
      double ec[4];
#pragma unroll
      for (int qq = 0; qq < 4; ++qq) {
        const int sI = qq & 1, sII = qq >> 1;
        const double o1 = xp[(2 * sI + sII) * N + X];
        const double o2 = sI ? hi[1 + sII] : lo[1 + sII];
        ec[qq] = halve(o1 + o2);
      }
      eLB = ec[0];
      eRB = ec[1];
      eLT = ec[2];
      eRT = ec[3];
      if (D.EdgeC) {  // the left/right values, for the adjoint (b_c, then lo/hi of the 2 EMF values)
        double* es = D.EdgeC + 10LL * e * N;
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          es[(2 * v) * N + X] = lo[v];
          es[(2 * v + 1) * N + X] = hi[v];
        }
      }
    }
    if (EMF != EMF_Q26) emf = ld04(apa, ama, apc, amc, eLB, eRB, eLT, eRT, baB, baT, bcL, bcR);
    if (D.resistive) {
      const double j = (Bc[X] - Bc[Xa]) * D.hinv[a] - (Ba[X] - Ba[Xc]) * D.hinv[c];
      emf = fma(D.eta, j, emf);
    }
    E[X] = D.combine ? halve(E[X] + emf) : emf;
  }
}

}  // namespace mhd
