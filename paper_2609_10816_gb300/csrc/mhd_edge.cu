// mhd_edge.cu -- edge EMFs (Sec. 2.3-2.4): reconstruction of face fields and face velocities
// to the edges (Fig. b-common, Eq. q26), the edge wavespeeds (Eq. alpha-edge), the LD04 average
// (Eq. ld04) and the Ohmic term (Eqs. current-stencil, emf-update).
//
// For an e-edge with a = e+1, c = e+2 (cyclic), the a-face quantities are reconstructed along c
// (bottom/top states) and the c-face quantities along a (left/right states). Two sweeps do
// this without recomputation: k_edge_bt walks lines along c and stores the four B/T values per
// edge; k_edge_lr walks lines along a, forms the L/R values and finishes the EMF.
#include "mhd_device.cuh"
#include "mhd_internal.cuh"
#include "mhd_index.cuh"

namespace mhd {

template <int RC>
__global__ void __launch_bounds__(128) k_edge_bt(Dev D, int e, int seg) {
  const int a = (e + 1) % 3, c = (e + 2) % 3;
  Line ln;
  int m0, m1;
  if (!sweep_line(D, c, seg, ln, m0, m1)) return;
  const long long N = D.N;
  const double* q[2] = {D.Bin[a], D.Us + a * N};
  constexpr int LB = Rec<RC>::LB, LA = Rec<RC>::LA;
  Rec<RC> r[2];
#pragma unroll
  for (int v = 0; v < 2; ++v) {
    double w[LB + LA];
#pragma unroll
    for (int t = 0; t < LB + LA; ++t) w[t] = q[v][ln.at(m0 - LB + t)];
    r[v].init(w);
  }
  double* out = D.Epart + 4LL * e * N;
  for (int m = m0; m < m1; ++m) {
    const long long X = ln.at(m);
    const long long Xn = ln.at(m + LA);
    double bB, bT, uB, uT;
    r[0].step(q[0][Xn], bB, bT);
    r[1].step(q[1][Xn], uB, uT);
    out[0 * N + X] = bB;
    out[1 * N + X] = bT;
    out[2 * N + X] = uB;
    out[3 * N + X] = uT;
  }
}

// Eq. (ld04) with the edge speeds of Eq. (alpha-edge), plus eta j (Eq. emf-update).
__device__ __forceinline__ double ld04(double apa, double ama, double apc, double amc, double eLB,
                                       double eRB, double eLT, double eRT, double baB, double baT,
                                       double bcL, double bcR) {
  const double ia = rcp(apa + ama), ic = rcp(apc + amc);
  const double w = ia * ic;
  const double up = fma(apc, fma(apa, eLB, ama * eRB), amc * fma(apa, eLT, ama * eRT)) * w;
  return fma(apa * ama * ia, bcR - bcL, fma(-apc * amc * ic, baT - baB, up));
}

template <int RC>
__global__ void __launch_bounds__(128) k_edge_lr(Dev D, int e, int seg) {
  const int a = (e + 1) % 3, c = (e + 2) % 3;
  Line ln;
  int m0, m1;
  if (!sweep_line(D, a, seg, ln, m0, m1)) return;
  const long long N = D.N;
  const double* q[2] = {D.Bin[c], D.Us + c * N};
  constexpr int LB = Rec<RC>::LB, LA = Rec<RC>::LA;
  Rec<RC> r[2];
#pragma unroll
  for (int v = 0; v < 2; ++v) {
    double w[LB + LA];
#pragma unroll
    for (int t = 0; t < LB + LA; ++t) w[t] = q[v][ln.at(m0 - LB + t)];
    r[v].init(w);
  }
  const double* part = D.Epart + 4LL * e * N;
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
    double bcL, bcR, ucL, ucR;
    r[0].step(q[0][Xn], bcL, bcR);
    r[1].step(q[1][Xn], ucL, ucR);
    const double baB = part[0 * N + X], baT = part[1 * N + X];
    const double uaB = part[2 * N + X], uaT = part[3 * N + X];
    // Eq. (q26): corner EMFs -u_a^{S_II} b_c^{S_I} + u_c^{S_I} b_a^{S_II}
    const double eLB = fma(-uaB, bcL, ucL * baB);
    const double eRB = fma(-uaB, bcR, ucR * baB);
    const double eLT = fma(-uaT, bcL, ucL * baT);
    const double eRT = fma(-uaT, bcR, ucR * baT);
    // Eq. (alpha-edge): alpha_a from the two a-faces (c-neighbours), alpha_c from the c-faces
    const double apa = pmax(Apa[Xc], Apa[X]), ama = pmax(Ama[Xc], Ama[X]);
    const double apc = pmax(Apc[Xa], Apc[X]), amc = pmax(Amc[Xa], Amc[X]);
    double emf = ld04(apa, ama, apc, amc, eLB, eRB, eLT, eRT, baB, baT, bcL, bcR);
    if (D.resistive) {
      const double j = (Bc[X] - Bc[Xa]) * D.hinv[a] - (Ba[X] - Ba[Xc]) * D.hinv[c];
      emf = fma(D.eta, j, emf);
    }
    E[X] = D.combine ? 0.5 * (E[X] + emf) : emf;
  }
}

template <int RC>
static void launch_bt_t(const Dev& d, int seg, cudaStream_t st) {
  const int bs = 128;
  for (int e = 0; e < 3; ++e) {
    const int c = (e + 2) % 3;
    const long long th = sweep_threads(d, c, seg);
    k_edge_bt<RC><<<(unsigned)((th + bs - 1) / bs), bs, 0, st>>>(d, e, seg);
  }
}
template <int RC>
static void launch_lr_t(const Dev& d, int seg, cudaStream_t st) {
  const int bs = 128;
  for (int e = 0; e < 3; ++e) {
    const int a = (e + 1) % 3;
    const long long th = sweep_threads(d, a, seg);
    k_edge_lr<RC><<<(unsigned)((th + bs - 1) / bs), bs, 0, st>>>(d, e, seg);
  }
}

void launch_edges_bt(const Dev& d, int recon, int seg, cudaStream_t st) {
  switch (recon) {
    case REC_PC: launch_bt_t<REC_PC>(d, seg, st); break;
    case REC_PLM_MC: launch_bt_t<REC_PLM_MC>(d, seg, st); break;
    case REC_PLM_MINMOD: launch_bt_t<REC_PLM_MINMOD>(d, seg, st); break;
    default: launch_bt_t<REC_PPM>(d, seg, st); break;
  }
}
void launch_edges_lr(const Dev& d, int recon, int seg, cudaStream_t st) {
  switch (recon) {
    case REC_PC: launch_lr_t<REC_PC>(d, seg, st); break;
    case REC_PLM_MC: launch_lr_t<REC_PLM_MC>(d, seg, st); break;
    case REC_PLM_MINMOD: launch_lr_t<REC_PLM_MINMOD>(d, seg, st); break;
    default: launch_lr_t<REC_PPM>(d, seg, st); break;
  }
}

}  // namespace mhd
