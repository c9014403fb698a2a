// mhd_face.cuh -- face sweep (Sec. 2.2): reconstruction along d + Riemann solve on every d-face,
// the Eq. (alpha-pm) speeds, the Q26 face velocity (Eq. q26-facevel), and the Joule energy flux of
// the Ohmic EMF (Sec. 2.4). One thread walks a segment of a periodic line along d; the
// reconstructed primitives sit in register sliding windows (Rec<> in mhd_device.cuh), so each
// cell's slope, interface value and limiter are evaluated once per direction and each face's
// Riemann problem once, with no halo recomputation.
#pragma once
#include "mhd_device.cuh"
#include "mhd_index.cuh"
#include "mhd_internal.cuh"

namespace mhd {

// Joule flux eta (j x b)_d on the d-face of cell X (reading: eta j from the mean of the face's
// two bounding edges per tangential direction, tangential b from the four nearest faces).
__device__ __forceinline__ double joule_flux(const Dev& D, int d, long long X) {
  const int a = (d + 1) % 3, c = (d + 2) % 3;
  const double* Ba = D.Bin[a];
  const double* Bc = D.Bin[c];
  // j_e on the e-edge stored at Y: (B_{c_e}[Y] - B_{c_e}[Y - a_e]) / h_{a_e}
  //                               - (B_{a_e}[Y] - B_{a_e}[Y - c_e]) / h_{c_e}
  auto jedge = [&](int e, long long Y) {
    const int ae = (e + 1) % 3, ce = (e + 2) % 3;
    const double* Bce = D.Bin[ce];
    const double* Bae = D.Bin[ae];
    return (Bce[Y] - Bce[shift(D, Y, ae, -1)]) * D.hinv[ae] - (Bae[Y] - Bae[shift(D, Y, ce, -1)]) * D.hinv[ce];
  };
  const long long Xc = shift(D, X, c, 1), Xa = shift(D, X, a, 1), Xmd = shift(D, X, d, -1);
  const double ea = 0.5 * D.eta * (jedge(a, X) + jedge(a, Xc));
  const double ec = 0.5 * D.eta * (jedge(c, X) + jedge(c, Xa));
  const double bcbar = 0.25 * (Bc[Xmd] + Bc[X] + Bc[shift(D, Xmd, c, 1)] + Bc[Xc]);
  const double babar = 0.25 * (Ba[Xmd] + Ba[X] + Ba[shift(D, Xmd, a, 1)] + Ba[Xa]);
  return fma(ea, bcbar, -ec * babar);
}

template <int RC, int RS>
__device__ __forceinline__ void face_seg(const Dev& D, int dir, const Line& ln, int m0, int m1) {
  const int a = (dir + 1) % 3, c = (dir + 2) % 3;
  const long long N = D.N;
  const double* q[7] = {D.P,           D.P + (1 + dir) * N, D.P + (1 + a) * N, D.P + (1 + c) * N,
                        D.P + 4 * N,   D.P + (5 + a) * N,   D.P + (5 + c) * N};
  constexpr int LB = Rec<RC>::LB, LA = Rec<RC>::LA;
  Rec<RC> r[7];
#pragma unroll
  for (int v = 0; v < 7; ++v) {
    double w[LB + LA];
#pragma unroll
    for (int t = 0; t < LB + LA; ++t) w[t] = q[v][ln.at(m0 - LB + t)];
    r[v].init(w);
  }
  const double* bnA = D.Bin[dir];
  // flux slots in the face frame (n, t1, t2): mass, the three momenta, energy
  double* Fs[5];
  {
    double* F = D.F + 5LL * dir * N;
    Fs[0] = F;
    Fs[1] = F + (1 + dir) * N;
    Fs[2] = F + (1 + a) * N;
    Fs[3] = F + (1 + c) * N;
    Fs[4] = F + 4 * N;
  }
  const bool fs18 = D.emf == EMF_FS18;
  for (int m = m0; m < m1; ++m) {
    const long long X = ln.at(m);
    const long long Xn = ln.at(m + LA);
    double Fold[5];  // stage 2: the stage-1 flux, loaded before the solve so its latency is hidden
    if (D.combine) {
#pragma unroll
      for (int v = 0; v < 5; ++v) Fold[v] = Fs[v][X];
    }
    double Lv[7], Rv[7];
#pragma unroll
    for (int v = 0; v < 7; ++v) r[v].step(q[v][Xn], Lv[v], Rv[v]);
    if (D.LR) {
      double* lr = D.LR + 14LL * dir * N;
#pragma unroll
      for (int v = 0; v < 7; ++v) {
        lr[v * N + X] = Lv[v];
        lr[(7 + v) * N + X] = Rv[v];
      }
    }
    const FaceState sl = {Lv[0], Lv[1], Lv[2], Lv[3], Lv[4], Lv[5], Lv[6]};
    const FaceState sr = {Rv[0], Rv[1], Rv[2], Rv[3], Rv[4], Rv[5], Rv[6]};
    double f[5], ap, am, us;
    riemann<RS>(sl, sr, bnA[X], D.gam, D.gm1inv, f, ap, am, us);
    if (D.resistive) f[4] += joule_flux(D, dir, X);
    if (D.combine) {
#pragma unroll
      for (int v = 0; v < 5; ++v) Fs[v][X] = halve(Fold[v] + f[v]);
    } else {
#pragma unroll
      for (int v = 0; v < 5; ++v) Fs[v][X] = f[v];
    }
    D.Ap[dir * N + X] = ap;
    D.Am[dir * N + X] = am;
    D.Us[dir * N + X] = us;
    if (fs18) {
      double* VL = D.VL + 3LL * dir * N;
      double* VR = D.VR + 3LL * dir * N;
      VL[dir * N + X] = Lv[1]; VR[dir * N + X] = Rv[1];
      VL[a * N + X] = Lv[2];   VR[a * N + X] = Rv[2];
      VL[c * N + X] = Lv[3];   VR[c * N + X] = Rv[3];
    }
  }
}

}  // namespace mhd
