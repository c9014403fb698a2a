// TEST INFRASTRUCTURE ONLY -- not part of the product path.
//
// A plain, slow, single-threaded CPU implementation of one time step of the second-order
// constrained-transport (CT) MHD method of "Magnetising the QUOKKA code" (Sec. 2), written
// from the paper's equations, step by step and in the paper's order, over a triply periodic
// uniform box. No tiling, no fusion, no reordering: every quantity the paper names is a full
// array. Only tests/, the smoke check and the benchmark's CPU-baseline leg load this library.
//
// It is templated on the scalar type: `double` for parity, and `Dual` (forward-mode dual
// numbers, one tangent) to give exact directional derivatives of a step for gradient checks.
//
// Layout (structure of arrays, x fastest), shared by every array here:
//   cell X = (i, j, k) -> index (k*ny + j)*nx + i, periodic in every direction;
//   cons[v][X]  v = 0 rho, 1..3 rho*u_d, 4 e_tot                         (Eq. state:conserved)
//   b[d][X]     normal field on the d-face at index_d - 1/2 of cell X     (Sec. 2.1, Yee mesh)
//   emf[e][X]   EMF on the e-edge at (index_a - 1/2, index_c - 1/2) of X, a=(e+1)%3, c=(e+2)%3
//   flux[d][v][X] flux of cons[v] across the d-face of X at index_d - 1/2.
//
// Readings taken where the paper is silent, ambiguous or garbled (each is also listed in the
// design notes, and the GPU path takes the same reading):
//   R1 energy flux: the paper's Eq. (mhd:conservation-laws) prints e_int in the energy flux;
//      the total energy e_tot is used (the system is not conservative otherwise).
//   R2 PLM limiters (Sec. 2.2): MC slope = sgn * min(2|dl|, 2|dr|, |dl+dr|/2) and minmod,
//      both zero unless dl and dr are strictly of the same sign.
//   R3 PPM (Sec. 2.2, close to Colella & Woodward 1984 in the paper's description): CW84 Eqs. 1.6-1.8 interface
//      interpolation with van Leer limited slopes, then the CW84 Eq. 1.10 monotonicity
//      constraints; no flattening, steepening or characteristic tracing (method of lines).
//   R4 fast speed along d (Eq. waves:fast-speed) with cos^2(theta) = b_d^2 / b^2; the square
//      root's argument is clamped at zero.
//   R5 HLL flux built from the Eq. (alpha-pm) speeds; if alpha+ + alpha- = 0 the left state's
//      flux (and left normal velocity) is taken.
//   R6 HLLD (Miyoshi & Kusano 2005), without the Minoshima fixes (not defined in the paper);
//      the star-state degeneracy test is |den| <= 1e-12 (rho (S-u)^2 + bn^2).
//   R7 LLF: alpha+ = alpha- = max(|u_L| + c_L, |u_R| + c_R) fed to the same formula.
//   R8 Joule flux (Sec. 2.4): eta (j x b) on each face, with eta j taken as the mean of the
//      face's two bounding edges of each tangential direction, and each tangential b as the mean
//      of the four nearest faces of that direction.
//   R9 FOFC (Sec. 2.5): first-order (PC + LLF) fluxes and EMFs use the chosen EMF compute and
//      averaging scheme; masked faces/edges are those of flagged cells; every cell and face that
//      touches a masked face or edge is recomputed; a cell is invalid if rho <= 0 (bit 0),
//      p <= 0 (bit 1), or any value is not finite; bit 2 is a user criterion that invalidates
//      every cell; invalid first-order results are accepted.
//   R10 time step (Sec. 2.4): per-cell signal speed max_d (|u_d| + c_f,d) dx_min/dx_d and
//      2 eta / dx_min; dt = CFL dx_min / max speed.
//   R11 PPM-EP (Sec. 2.2 cites Rider, Greenough & Kamm 2007 and does not define it): the
//      parabola of PPM with the unlimited fourth-order interface value, and the monotonicity
//      limiting in its median-function form, switched off at extrema that are smooth. With the
//      differences d_{j+1/2} = q_{j+1} - q_j and curvatures D_j = d_{j+1/2} - d_{j-1/2}:
//      interface j+1/2 lies at an extremum when two of d_{j-1/2}, d_{j+1/2}, d_{j+3/2} have
//      strictly opposite signs (a peak or trough in one cell, or shared by two equal cells), and
//      cell j when one of its two interfaces does. The interface value is
//      (7 (q_j + q_{j+1}) - (q_{j-1} + q_{j+2})) / 12, bounded to median(q_j, ., q_{j+1}) unless it
//      lies at an extremum with D_j, D_{j+1} both > 0 or both < 0. Cell j then takes the CW84
//      Eq. 1.10 constraints (in median form aR <- median(q_j, aR, 3 q_j - 2 aL) and
//      aL <- median(q_j, aL, 3 q_j - 2 aR)) unless it lies at an extremum with D_{j-1}, D_j, D_{j+1}
//      all > 0 or all < 0: a smooth extremum keeps its parabola, while a discontinuity (where the
//      curvature changes sign) and the monotone foot of a jump are limited as in PPM.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

// ---------------------------------------------------------------------------------------
// Scalars
// ---------------------------------------------------------------------------------------
struct Dual {
  double v, t;
  Dual() : v(0), t(0) {}
  Dual(double x) : v(x), t(0) {}  // NOLINT: implicit promotion of constants
  Dual(double x, double dx) : v(x), t(dx) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.t + b.t); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.t - b.t); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.t); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.t * b.v + a.v * b.t); }
inline Dual operator/(Dual a, Dual b) {
  const double q = a.v / b.v;
  return Dual(q, (a.t - q * b.t) / b.v);
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }

// Operation counting (used only to state the algorithmic FP64 work per unit of the method):
// every +, -, *, / and sqrt of a Cnt adds one to the counter of the current phase; comparisons,
// negation and |x| are not counted.
enum { PH_PRIM = 0, PH_RECON = 1, PH_RIEMANN = 2, PH_EDGE = 3, PH_JOULE = 4, PH_UPDATE = 5,
       PH_FLAG = 6, PH_FO = 7, NPHASE = 8 };
long long g_ops[NPHASE];
// Operations of the HLLD solve that a solver forming only what the face's region of the Riemann
// fan needs would not form (the other side's star state and the double-star states outside the
// rotational waves); counted on the side so the roofline can state both figures.
long long g_hlld_unused = 0;
int g_phase = 0;
bool g_fo = false;
inline void set_phase(int p) { g_phase = g_fo ? PH_FO : p; }
struct Cnt {
  double v;
  Cnt() : v(0) {}
  Cnt(double x) : v(x) {}  // NOLINT: implicit promotion of constants
};
inline Cnt operator+(Cnt a, Cnt b) { ++g_ops[g_phase]; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { ++g_ops[g_phase]; return Cnt(a.v - b.v); }
inline Cnt operator*(Cnt a, Cnt b) { ++g_ops[g_phase]; return Cnt(a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { ++g_ops[g_phase]; return Cnt(a.v / b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline Cnt& operator+=(Cnt& a, Cnt b) { a = a + b; return a; }
inline Cnt& operator-=(Cnt& a, Cnt b) { a = a - b; return a; }

inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }
inline double val(const Cnt& x) { return x.v; }
inline Cnt sqrt_(Cnt a) { ++g_ops[g_phase]; return Cnt(std::sqrt(a.v)); }
inline double sqrt_(double x) { return std::sqrt(x); }
inline Dual sqrt_(Dual a) {
  const double s = std::sqrt(a.v);
  return Dual(s, s > 0 ? a.t / (2.0 * s) : 0.0);
}
// max/min return their first argument on ties; |x| and sgn follow the value.
template <class T> inline T mx(T a, T b) { return val(a) >= val(b) ? a : b; }
template <class T> inline T mn(T a, T b) { return val(a) <= val(b) ? a : b; }
template <class T> inline T absv(T a) { return val(a) < 0 ? -a : a; }
template <class T> inline double sgn(T a) { return val(a) > 0 ? 1.0 : (val(a) < 0 ? -1.0 : 0.0); }
template <class T> inline bool same_sign(T a, T b) {
  return (val(a) > 0 && val(b) > 0) || (val(a) < 0 && val(b) < 0);
}

// ---------------------------------------------------------------------------------------
// Configuration and grid
// ---------------------------------------------------------------------------------------
enum { REC_PC = 0, REC_PLM_MC = 1, REC_PLM_MINMOD = 2, REC_PPM = 3, REC_PPM_EP = 4 };
enum { RS_HLL = 0, RS_HLLD = 1, RS_LLF = 2 };
enum { EMF_Q26 = 0, EMF_FS18 = 1, EMF_B25A = 2 };

struct Grid {
  int n[3];
  long N;
  double h[3];
  double gamma;
  long at(int i, int j, int k) const {
    i %= n[0]; if (i < 0) i += n[0];
    j %= n[1]; if (j < 0) j += n[1];
    k %= n[2]; if (k < 0) k += n[2];
    return ((long)k * n[1] + j) * n[0] + i;
  }
  // cell X shifted by s cells along direction d (periodic)
  long sh(long X, int d, int s) const {
    int c[3];
    c[0] = (int)(X % n[0]);
    c[1] = (int)((X / n[0]) % n[1]);
    c[2] = (int)(X / ((long)n[0] * n[1]));
    c[d] += s;
    return at(c[0], c[1], c[2]);
  }
};

template <class T> struct Scheme {
  int recon, riemann, emf;
  T eta;
  bool resistive;  // include the Ohmic EMF and Joule flux (eta or its tangent non-zero)
};

// Primitive array slots (Eq. state:primitive): rho, u0, u1, u2, p, b0, b1, b2 (cell averages).
enum { P_RHO = 0, P_U = 1, P_P = 4, P_B = 5, NPRIM = 8 };

// ---------------------------------------------------------------------------------------
// Sec. 2.2: conserved -> primitive, with the cell-averaged field from the two faces.
// ---------------------------------------------------------------------------------------
template <class T>
void cons_to_prim(const Grid& g, const std::vector<T>& U, const std::vector<T>& B,
                  std::vector<T>& P) {
  const long N = g.N;
  set_phase(PH_PRIM);
  P.assign(NPRIM * N, T(0.0));
  for (long X = 0; X < N; ++X) {
    const T rho = U[X];
    T u[3], bc[3];
    for (int d = 0; d < 3; ++d) {
      u[d] = U[(1 + d) * N + X] / rho;
      bc[d] = 0.5 * (B[d * N + X] + B[d * N + g.sh(X, d, 1)]);
    }
    const T kin = 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const T mag = 0.5 * (bc[0] * bc[0] + bc[1] * bc[1] + bc[2] * bc[2]);
    P[P_RHO * N + X] = rho;
    for (int d = 0; d < 3; ++d) {
      P[(P_U + d) * N + X] = u[d];
      P[(P_B + d) * N + X] = bc[d];
    }
    P[P_P * N + X] = (g.gamma - 1.0) * (U[4 * N + X] - kin - mag);
  }
}

// ---------------------------------------------------------------------------------------
// Sec. 2.2: 1D reconstruction of a periodic array q along direction d. For every point X it
// returns the value at its lower side (qm, at X - 1/2) and upper side (qp, at X + 1/2).
// The interface between X-1 and X therefore has left state qp[X-1] and right state qm[X].
// ---------------------------------------------------------------------------------------
template <class T> T slope_mc(T dl, T dr) {  // reading R2
  if (!same_sign(dl, dr)) return T(0.0);
  const T m = mn(mn(2.0 * absv(dl), 2.0 * absv(dr)), 0.5 * absv(dl + dr));
  return sgn(dl) * m;
}
template <class T> T slope_minmod(T dl, T dr) {  // reading R2
  if (!same_sign(dl, dr)) return T(0.0);
  return sgn(dl) * mn(absv(dl), absv(dr));
}
// CW84 Eqs. 1.7-1.8: van Leer limited average slope.
template <class T> T slope_vl(T qm1, T q0, T qp1) {
  const T dl = q0 - qm1, dr = qp1 - q0;
  if (!same_sign(dl, dr)) return T(0.0);
  const T dc = 0.5 * (qp1 - qm1);
  return sgn(dc) * mn(mn(absv(dc), 2.0 * absv(dl)), 2.0 * absv(dr));
}

// CW84 Eq. 1.10: the parabola (aL, a, aR) of a cell made monotone.
template <class T> void cw84_monotone(T a, T& aL, T& aR) {
  if (!same_sign(aR - a, a - aL)) {
    aL = a;
    aR = a;
  } else {
    const T da = aR - aL;
    const T a6 = 6.0 * (a - 0.5 * (aL + aR));
    if (val(da * a6) > val(da * da)) {
      aL = 3.0 * a - 2.0 * aR;
    } else if (val(-(da * da)) > val(da * a6)) {
      aR = 3.0 * a - 2.0 * aL;
    }
  }
}
// the middle one of three values
template <class T> T median3(T a, T b, T c) { return mx(mn(a, b), mn(mx(a, b), c)); }

template <class T>
void recon_field(const Grid& g, int method, const T* q, int d, std::vector<T>& qm,
                 std::vector<T>& qp) {
  const long N = g.N;
  qm.assign(N, T(0.0));
  qp.assign(N, T(0.0));
  if (method == REC_PC) {
    for (long X = 0; X < N; ++X) qm[X] = qp[X] = q[X];
    return;
  }
  if (method == REC_PLM_MC || method == REC_PLM_MINMOD) {
    for (long X = 0; X < N; ++X) {
      const T dl = q[X] - q[g.sh(X, d, -1)];
      const T dr = q[g.sh(X, d, 1)] - q[X];
      const T s = (method == REC_PLM_MC) ? slope_mc(dl, dr) : slope_minmod(dl, dr);
      qm[X] = q[X] - 0.5 * s;
      qp[X] = q[X] + 0.5 * s;
    }
    return;
  }
  if (method == REC_PPM_EP) {  // reading R11
    // dif[X] = d_{X-1/2} = q[X] - q[X-1]; curv[X] = D_X; face[X] = interface value at X - 1/2,
    // ext[X] = whether interface X - 1/2 lies at an extremum
    std::vector<T> dif(N), curv(N), face(N);
    std::vector<char> ext(N);
    for (long X = 0; X < N; ++X) dif[X] = q[X] - q[g.sh(X, d, -1)];
    for (long X = 0; X < N; ++X) curv[X] = dif[g.sh(X, d, 1)] - dif[X];
    auto opposite = [](T a, T b) { return (val(a) > 0 && val(b) < 0) || (val(a) < 0 && val(b) > 0); };
    for (long X = 0; X < N; ++X) {
      const T dm = dif[g.sh(X, d, -1)], d0 = dif[X], dp = dif[g.sh(X, d, 1)];
      ext[X] = opposite(dm, d0) || opposite(d0, dp) || opposite(dm, dp);
    }
    for (long X = 0; X < N; ++X) {
      const long Xm = g.sh(X, d, -1);
      face[X] = (7.0 * (q[Xm] + q[X]) - (q[g.sh(X, d, -2)] + q[g.sh(X, d, 1)])) / 12.0;
      if (!(ext[X] && same_sign(curv[Xm], curv[X]))) face[X] = median3(q[Xm], face[X], q[X]);
    }
    for (long X = 0; X < N; ++X) {
      const long Xp = g.sh(X, d, 1);
      T aL = face[X], aR = face[Xp];
      const T cm = curv[g.sh(X, d, -1)], c0 = curv[X], cp = curv[Xp];
      const bool smooth_extremum = (ext[X] || ext[Xp]) && same_sign(cm, c0) && same_sign(c0, cp);
      if (!smooth_extremum) cw84_monotone(q[X], aL, aR);
      qm[X] = aL;
      qp[X] = aR;
    }
    return;
  }
  // PPM, reading R3.
  std::vector<T> dq(N), face(N);  // face[X] = interface value at X - 1/2
  for (long X = 0; X < N; ++X) dq[X] = slope_vl(q[g.sh(X, d, -1)], q[X], q[g.sh(X, d, 1)]);
  for (long X = 0; X < N; ++X) {
    const long Xm = g.sh(X, d, -1);
    // CW84 Eq. 1.6, a_{j+1/2} = a_j + (a_{j+1} - a_j)/2 - (da_{j+1} - da_j)/6, written with
    // the first two terms as the mean of the two cell values.
    face[X] = 0.5 * (q[Xm] + q[X]) - (dq[X] - dq[Xm]) / 6.0;
  }
  for (long X = 0; X < N; ++X) {
    T aL = face[X], aR = face[g.sh(X, d, 1)];
    cw84_monotone(q[X], aL, aR);  // CW84 Eq. 1.10
    qm[X] = aL;
    qp[X] = aR;
  }
}

// ---------------------------------------------------------------------------------------
// Sec. 2.2 / 2.3: Riemann solvers in the face frame (n, t1, t2) = (d, d+1, d+2).
// W = {rho, u_n, u_t1, u_t2, p, b_t1, b_t2}; bn is the stored face field.
// Out: flux of {rho, m_n, m_t1, m_t2, e_tot}, alpha+/alpha- (Eq. alpha-pm), and the
// wavespeed-weighted normal velocity of Eq. (q26-facevel).
// ---------------------------------------------------------------------------------------
template <class T> T fast_speed(double gam, const T* W, T bn) {  // Eq. waves:fast-speed, R4
  const T a2 = gam * W[4] / W[0];
  const T b2 = bn * bn + W[5] * W[5] + W[6] * W[6];
  const T s = a2 + b2 / W[0];
  const T disc = mx(s * s - 4.0 * a2 * (bn * bn) / W[0], T(0.0));
  return sqrt_(0.5 * (s + sqrt_(disc)));
}

// Eq. (mhd:conservation-laws) in the face frame, with e_tot in the energy flux (reading R1).
template <class T> void phys_flux(double gam, const T* W, T bn, T* U, T* F) {
  const T rho = W[0], u = W[1], v = W[2], w = W[3], p = W[4], by = W[5], bz = W[6];
  const T b2 = bn * bn + by * by + bz * bz;
  const T e = p / (gam - 1.0) + 0.5 * rho * (u * u + v * v + w * w) + 0.5 * b2;
  const T pt = p + 0.5 * b2;
  const T ub = u * bn + v * by + w * bz;
  U[0] = rho;
  U[1] = rho * u;
  U[2] = rho * v;
  U[3] = rho * w;
  U[4] = e;
  F[0] = rho * u;
  F[1] = rho * u * u + pt - bn * bn;
  F[2] = rho * u * v - bn * by;
  F[3] = rho * u * w - bn * bz;
  F[4] = (e + pt) * u - ub * bn;
}

// Two-state formula shared by HLL and LLF (reading R5, R7).
template <class T>
void two_state(const T* UL, const T* FL, const T* UR, const T* FR, T ap, T am, T* F) {
  const T sum = ap + am;
  if (val(sum) == 0.0) {
    for (int v = 0; v < 5; ++v) F[v] = FL[v];
    return;
  }
  for (int v = 0; v < 5; ++v) F[v] = (ap * FL[v] + am * FR[v] - ap * am * (UR[v] - UL[v])) / sum;
}

// Miyoshi & Kusano (2005) HLLD, reading R6.
template <class T>
void hlld(const T* WL, const T* WR, T bn, T SL, T SR, const T* UL, const T* FL,
          const T* UR, const T* FR, T* F) {
  if (val(SL) > 0.0) { for (int v = 0; v < 5; ++v) F[v] = FL[v]; return; }
  if (val(SR) < 0.0) { for (int v = 0; v < 5; ++v) F[v] = FR[v]; return; }
  const T rhoL = WL[0], uL = WL[1], pL = WL[4];
  const T rhoR = WR[0], uR = WR[1], pR = WR[4];
  const T ptL = pL + 0.5 * (bn * bn + WL[5] * WL[5] + WL[6] * WL[6]);
  const T ptR = pR + 0.5 * (bn * bn + WR[5] * WR[5] + WR[6] * WR[6]);
  const T sluL = SL - uL, sruR = SR - uR;
  const T den = sruR * rhoR - sluL * rhoL;
  // MK05 Eqs. 38 and 41: contact speed and star total pressure.
  const T SM = ((sruR * rhoR * uR - sluL * rhoL * uL) + (ptL - ptR)) / den;
  const T ptS = (sruR * rhoR * ptL - sluL * rhoL * ptR + rhoL * rhoR * sruR * sluL * (uR - uL)) / den;
  const T bn2 = bn * bn;
  // star states, MK05 Eqs. 43-48
  T Us[2][5], vS[2], wS[2], byS[2], bzS[2], rS[2];
  const T* Ws[2] = {WL, WR};
  const T* Uo[2] = {UL, UR};
  const T Ss[2] = {SL, SR};
  long long side_ops[2];  // operations of each side's star state (counting pass only)
  for (int s = 0; s < 2; ++s) {
    const long long o_side = g_ops[g_phase];
    const T* W = Ws[s];
    const T S = Ss[s];
    const T rho = W[0], u = W[1], v = W[2], w = W[3], by = W[5], bz = W[6];
    const T su = S - u, ssm = S - SM;
    const T rs = rho * su / ssm;
    const T dd = rho * su * ssm - bn2;
    T vs, ws, bys, bzs;
    if (std::fabs(val(dd)) <= 1e-12 * val(rho * su * su + bn2)) {
      vs = v; ws = w; bys = by; bzs = bz;
    } else {
      const T cv = bn * (SM - u) / dd;
      const T cb = (rho * su * su - bn2) / dd;
      vs = v - by * cv;
      ws = w - bz * cv;
      bys = by * cb;
      bzs = bz * cb;
    }
    const T pt = (s == 0) ? ptL : ptR;
    const T vb = u * bn + v * by + w * bz;
    const T vbs = SM * bn + vs * bys + ws * bzs;
    const T es = (su * Uo[s][4] - pt * u + ptS * SM + bn * (vb - vbs)) / ssm;
    rS[s] = rs; vS[s] = vs; wS[s] = ws; byS[s] = bys; bzS[s] = bzs;
    Us[s][0] = rs; Us[s][1] = rs * SM; Us[s][2] = rs * vs; Us[s][3] = rs * ws; Us[s][4] = es;
    side_ops[s] = g_ops[g_phase] - o_side;
  }
  const long long o_double = g_ops[g_phase];
  // double-star states, MK05 Eqs. 49-63
  const T sqL = sqrt_(rS[0]), sqR = sqrt_(rS[1]);
  const T SsL = SM - absv(bn) / sqL, SsR = SM + absv(bn) / sqR;
  const double sb = sgn(bn);
  const T inv = 1.0 / (sqL + sqR);
  const T vss = (sqL * vS[0] + sqR * vS[1] + (byS[1] - byS[0]) * sb) * inv;
  const T wss = (sqL * wS[0] + sqR * wS[1] + (bzS[1] - bzS[0]) * sb) * inv;
  const T byss = (sqL * byS[1] + sqR * byS[0] + sqL * sqR * (vS[1] - vS[0]) * sb) * inv;
  const T bzss = (sqL * bzS[1] + sqR * bzS[0] + sqL * sqR * (wS[1] - wS[0]) * sb) * inv;
  const T vbss = SM * bn + vss * byss + wss * bzss;
  T Uss[2][5];
  for (int s = 0; s < 2; ++s) {
    const T sq = (s == 0) ? sqL : sqR;
    const double side = (s == 0) ? -1.0 : 1.0;
    const T vbs = SM * bn + vS[s] * byS[s] + wS[s] * bzS[s];
    Uss[s][0] = rS[s];
    Uss[s][1] = rS[s] * SM;
    Uss[s][2] = rS[s] * vss;
    Uss[s][3] = rS[s] * wss;
    Uss[s][4] = Us[s][4] + side * sq * (vbs - vbss) * sb;
  }
  // outside both rotational waves the double-star states are not needed (deciding that takes
  // S_M^2 rho* against b_n^2: two operations), nor the other side's star state
  const long long double_ops = g_ops[g_phase] - o_double;
  if (val(SsL) >= 0.0) g_hlld_unused += side_ops[1] + double_ops - 2;
  else if (val(SsR) < 0.0) g_hlld_unused += side_ops[0] + double_ops - 2;
  // MK05 Eqs. 64-66 and the fan selection.
  if (val(SsL) >= 0.0) {
    for (int v = 0; v < 5; ++v) F[v] = FL[v] + SL * (Us[0][v] - UL[v]);
  } else if (val(SM) >= 0.0) {
    for (int v = 0; v < 5; ++v)
      F[v] = FL[v] + SL * (Us[0][v] - UL[v]) + SsL * (Uss[0][v] - Us[0][v]);
  } else if (val(SsR) >= 0.0) {
    for (int v = 0; v < 5; ++v)
      F[v] = FR[v] + SR * (Us[1][v] - UR[v]) + SsR * (Uss[1][v] - Us[1][v]);
  } else {
    for (int v = 0; v < 5; ++v) F[v] = FR[v] + SR * (Us[1][v] - UR[v]);
  }
}

template <class T>
void riemann(int solver, double gam, const T* WL, const T* WR, T bn, T* F, T& ap, T& am,
             T& ustar) {
  T UL[5], FL[5], UR[5], FR[5];
  phys_flux(gam, WL, bn, UL, FL);
  phys_flux(gam, WR, bn, UR, FR);
  const T cL = fast_speed(gam, WL, bn), cR = fast_speed(gam, WR, bn);
  const T uL = WL[1], uR = WR[1];
  if (solver == RS_LLF) {
    const T a = mx(absv(uL) + cL, absv(uR) + cR);
    ap = a;
    am = a;
    two_state(UL, FL, UR, FR, ap, am, F);
  } else {
    // Eq. (alpha-pm): MK05 Eq. 67 bounding speeds, clamped at zero for the magnitudes.
    const T cmax = mx(cL, cR);
    const T SR = mx(uL, uR) + cmax;
    const T SL = mn(uL, uR) - cmax;
    ap = mx(T(0.0), SR);
    am = mx(T(0.0), cmax - mn(uL, uR));
    if (solver == RS_HLL)
      two_state(UL, FL, UR, FR, ap, am, F);
    else
      hlld(WL, WR, bn, SL, SR, UL, FL, UR, FR, F);
  }
  // Eq. (q26-facevel)
  const T sum = ap + am;
  ustar = (val(sum) == 0.0) ? uL : (ap * uL + am * uR) / sum;
}

// ---------------------------------------------------------------------------------------
// Fluxes and EMFs of one state (Secs. 2.2-2.4).
// ---------------------------------------------------------------------------------------
template <class T> struct FluxSet {
  std::vector<T> F;  // [3][5][N]
  std::vector<T> E;  // [3][N]
  bool keep_corners = false;  // also return the four corner EMFs of every edge (pins only)
  std::vector<T> C;  // [3][4][N], corners LB, RB, LT, RT before the averaging of Eq. (ld04)
};

template <class T>
void fluxes_and_emfs(const Grid& g, const Scheme<T>& sc, const std::vector<T>& U,
                     const std::vector<T>& B, FluxSet<T>& out) {
  const long N = g.N;
  const double gam = g.gamma;
  std::vector<T> P;
  cons_to_prim(g, U, B, P);

  out.F.assign(15 * N, T(0.0));
  out.E.assign(3 * N, T(0.0));
  if (out.keep_corners) out.C.assign(12 * N, T(0.0));
  std::vector<T> Ap(3 * N), Am(3 * N), Us(3 * N);
  // face-centred left/right velocity states (FS18 only): [d][k][N]
  std::vector<T> VL, VR;
  if (sc.emf == EMF_FS18) {
    VL.assign(9 * N, T(0.0));
    VR.assign(9 * N, T(0.0));
  }

  // --- Sec. 2.2: reconstruction along each direction and the Riemann problem on each face.
  for (int d = 0; d < 3; ++d) {
    const int a = (d + 1) % 3, c = (d + 2) % 3;
    // primitive slots in face order {rho, u_n, u_t1, u_t2, p, b_t1, b_t2}
    const int slot[7] = {P_RHO, P_U + d, P_U + a, P_U + c, P_P, P_B + a, P_B + c};
    std::vector<T> qm[7], qp[7];
    set_phase(PH_RECON);
    for (int v = 0; v < 7; ++v) recon_field(g, sc.recon, &P[slot[v] * N], d, qm[v], qp[v]);
    set_phase(PH_RIEMANN);
    for (long X = 0; X < N; ++X) {
      const long Xl = g.sh(X, d, -1);
      T WL[7], WR[7];
      for (int v = 0; v < 7; ++v) {
        WL[v] = qp[v][Xl];
        WR[v] = qm[v][X];
      }
      T Fr[5], ap, am, us;
      riemann(sc.riemann, gam, WL, WR, B[d * N + X], Fr, ap, am, us);
      T* F = &out.F[(5 * d) * N];
      F[0 * N + X] = Fr[0];
      F[(1 + d) * N + X] = Fr[1];
      F[(1 + a) * N + X] = Fr[2];
      F[(1 + c) * N + X] = Fr[3];
      F[4 * N + X] = Fr[4];
      Ap[d * N + X] = ap;
      Am[d * N + X] = am;
      Us[d * N + X] = us;
      if (sc.emf == EMF_FS18) {
        // global velocity components k = d, a, c sit in face slots 1, 2, 3
        VL[(3 * d + d) * N + X] = WL[1]; VR[(3 * d + d) * N + X] = WR[1];
        VL[(3 * d + a) * N + X] = WL[2]; VR[(3 * d + a) * N + X] = WR[2];
        VL[(3 * d + c) * N + X] = WL[3]; VR[(3 * d + c) * N + X] = WR[3];
      }
    }
  }

  // --- Sec. 2.3: EMF on every e-edge. For edge direction e, a = e+1 and c = e+2 play the
  // roles of x0 and x1 in the paper's x2-edge description (cyclic permutation).
  std::vector<T> rm, rp, rm2, rp2;
  set_phase(PH_EDGE);
  for (int e = 0; e < 3; ++e) {
    const int a = (e + 1) % 3, c = (e + 2) % 3;
    // Fig. (b-common): b_a reconstructed along c (B/T), b_c along a (L/R).
    std::vector<T> baB(N), baT(N), bcL(N), bcR(N);
    recon_field(g, sc.recon, &B[a * N], c, rm, rp);
    for (long X = 0; X < N; ++X) { baB[X] = rp[g.sh(X, c, -1)]; baT[X] = rm[X]; }
    recon_field(g, sc.recon, &B[c * N], a, rm, rp);
    for (long X = 0; X < N; ++X) { bcL[X] = rp[g.sh(X, a, -1)]; bcR[X] = rm[X]; }

    // four corner EMFs: index 0 LB, 1 RB, 2 LT, 3 RT
    std::vector<T> corner(4 * N);
    if (sc.emf == EMF_Q26) {
      // Eq. (q26): u_a* reconstructed along c, u_c* along a.
      std::vector<T> uaB(N), uaT(N), ucL(N), ucR(N);
      recon_field(g, sc.recon, &Us[a * N], c, rm, rp);
      for (long X = 0; X < N; ++X) { uaB[X] = rp[g.sh(X, c, -1)]; uaT[X] = rm[X]; }
      recon_field(g, sc.recon, &Us[c * N], a, rm, rp);
      for (long X = 0; X < N; ++X) { ucL[X] = rp[g.sh(X, a, -1)]; ucR[X] = rm[X]; }
      for (long X = 0; X < N; ++X) {
        corner[0 * N + X] = -uaB[X] * bcL[X] + ucL[X] * baB[X];
        corner[1 * N + X] = -uaB[X] * bcR[X] + ucR[X] * baB[X];
        corner[2 * N + X] = -uaT[X] * bcL[X] + ucL[X] * baT[X];
        corner[3 * N + X] = -uaT[X] * bcR[X] + ucR[X] * baT[X];
      }
    } else if (sc.emf == EMF_FS18) {
      // Eqs. (fs18-average) and (fs18). For each velocity component k in {a, c}:
      //   order (a then c): a-face L/R states reconstructed along c -> (S_I, S_II);
      //   order (c then a): c-face B/T states reconstructed along a -> (S_I, S_II).
      std::vector<T> ubar[2];  // [k: 0 -> u_a, 1 -> u_c][4 corners * N]
      const int comp[2] = {a, c};
      for (int kk = 0; kk < 2; ++kk) {
        const int k = comp[kk];
        ubar[kk].assign(4 * N, T(0.0));
        // order a then c
        for (int side = 0; side < 2; ++side) {  // S_I = L (0) or R (1)
          const T* src = side == 0 ? &VL[(3 * a + k) * N] : &VR[(3 * a + k) * N];
          recon_field(g, sc.recon, src, c, rm, rp);
          for (long X = 0; X < N; ++X) {
            ubar[kk][(0 + side) * N + X] += 0.5 * rp[g.sh(X, c, -1)];  // S_II = B
            ubar[kk][(2 + side) * N + X] += 0.5 * rm[X];               // S_II = T
          }
        }
        // order c then a
        for (int side = 0; side < 2; ++side) {  // S_II = B (0) or T (1)
          const T* src = side == 0 ? &VL[(3 * c + k) * N] : &VR[(3 * c + k) * N];
          recon_field(g, sc.recon, src, a, rm, rp);
          for (long X = 0; X < N; ++X) {
            ubar[kk][(2 * side + 0) * N + X] += 0.5 * rp[g.sh(X, a, -1)];  // S_I = L
            ubar[kk][(2 * side + 1) * N + X] += 0.5 * rm[X];               // S_I = R
          }
        }
      }
      for (long X = 0; X < N; ++X) {
        const T bcS[2] = {bcL[X], bcR[X]};
        const T baS[2] = {baB[X], baT[X]};
        for (int q = 0; q < 4; ++q) {
          const int sI = q & 1, sII = q >> 1;
          corner[q * N + X] = -ubar[0][q * N + X] * bcS[sI] + ubar[1][q * N + X] * baS[sII];
        }
      }
    } else {
      // B25a, Eqs. (b25a-b-avg), (b25a-emf-centre), (b25a-average).
      std::vector<T> ec(N);
      for (long X = 0; X < N; ++X)
        ec[X] = -P[(P_U + a) * N + X] * P[(P_B + c) * N + X] +
                P[(P_U + c) * N + X] * P[(P_B + a) * N + X];
      for (int q = 0; q < 4; ++q)
        for (long X = 0; X < N; ++X) corner[q * N + X] = T(0.0);
      // order a then c: to a-faces (L/R), then along c
      recon_field(g, sc.recon, ec.data(), a, rm, rp);
      std::vector<T> fL(N), fR(N);
      for (long X = 0; X < N; ++X) { fL[X] = rp[g.sh(X, a, -1)]; fR[X] = rm[X]; }
      for (int side = 0; side < 2; ++side) {
        recon_field(g, sc.recon, side == 0 ? fL.data() : fR.data(), c, rm2, rp2);
        for (long X = 0; X < N; ++X) {
          corner[(0 + side) * N + X] += 0.5 * rp2[g.sh(X, c, -1)];
          corner[(2 + side) * N + X] += 0.5 * rm2[X];
        }
      }
      // order c then a: to c-faces (B/T), then along a
      recon_field(g, sc.recon, ec.data(), c, rm, rp);
      for (long X = 0; X < N; ++X) { fL[X] = rp[g.sh(X, c, -1)]; fR[X] = rm[X]; }
      for (int side = 0; side < 2; ++side) {
        recon_field(g, sc.recon, side == 0 ? fL.data() : fR.data(), a, rm2, rp2);
        for (long X = 0; X < N; ++X) {
          corner[(2 * side + 0) * N + X] += 0.5 * rp2[g.sh(X, a, -1)];
          corner[(2 * side + 1) * N + X] += 0.5 * rm2[X];
        }
      }
    }

    if (out.keep_corners)
      for (long I = 0; I < 4 * N; ++I) out.C[4 * e * N + I] = corner[I];

    // Eq. (alpha-edge) and Eq. (ld04).
    for (long X = 0; X < N; ++X) {
      const long Xc = g.sh(X, c, -1), Xa = g.sh(X, a, -1);
      const T apa = mx(Ap[a * N + Xc], Ap[a * N + X]);
      const T ama = mx(Am[a * N + Xc], Am[a * N + X]);
      const T apc = mx(Ap[c * N + Xa], Ap[c * N + X]);
      const T amc = mx(Am[c * N + Xa], Am[c * N + X]);
      const T sa = apa + ama, sc2 = apc + amc;
      const T eLB = corner[0 * N + X], eRB = corner[1 * N + X];
      const T eLT = corner[2 * N + X], eRT = corner[3 * N + X];
      T emf = (apa * apc * eLB + ama * apc * eRB) / (sa * sc2) +
              (apa * amc * eLT + ama * amc * eRT) / (sa * sc2) -
              apc * amc / sc2 * (baT[X] - baB[X]) + apa * ama / sa * (bcR[X] - bcL[X]);
      // Eqs. (resistivity:current-stencil) and (resistivity:emf-update)
      if (sc.resistive) {
        const T j = (B[c * N + X] - B[c * N + Xa]) / g.h[a] - (B[a * N + X] - B[a * N + Xc]) / g.h[c];
        emf = emf + sc.eta * j;
      }
      out.E[e * N + X] = emf;
    }
  }

  // --- Sec. 2.4: Joule-heating energy flux eta (j x b) on each face (reading R8).
  if (sc.resistive) {
    set_phase(PH_JOULE);
    std::vector<T> J(3 * N);
    for (int e = 0; e < 3; ++e) {
      const int a = (e + 1) % 3, c = (e + 2) % 3;
      for (long X = 0; X < N; ++X) {
        const long Xc = g.sh(X, c, -1), Xa = g.sh(X, a, -1);
        J[e * N + X] = sc.eta * ((B[c * N + X] - B[c * N + Xa]) / g.h[a] -
                                 (B[a * N + X] - B[a * N + Xc]) / g.h[c]);
      }
    }
    for (int d = 0; d < 3; ++d) {
      const int a = (d + 1) % 3, c = (d + 2) % 3;
      for (long X = 0; X < N; ++X) {
        const long Xmd = g.sh(X, d, -1);
        const T ea = 0.5 * (J[a * N + X] + J[a * N + g.sh(X, c, 1)]);
        const T ec = 0.5 * (J[c * N + X] + J[c * N + g.sh(X, a, 1)]);
        const T bcbar = 0.25 * (B[c * N + Xmd] + B[c * N + X] + B[c * N + g.sh(Xmd, c, 1)] +
                                B[c * N + g.sh(X, c, 1)]);
        const T babar = 0.25 * (B[a * N + Xmd] + B[a * N + X] + B[a * N + g.sh(Xmd, a, 1)] +
                                B[a * N + g.sh(X, a, 1)]);
        out.F[(5 * d + 4) * N + X] += ea * bcbar - ec * babar;
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// Sec. 2.5: update increments, Eqs. (rk:increment-state) and (rk:increment-bfield).
// ---------------------------------------------------------------------------------------
template <class T> T incr_cell(const Grid& g, const FluxSet<T>& f, int v, long X, double dt) {
  const long N = g.N;
  const T* F0 = &f.F[(5 * 0 + v) * N];
  const T* F1 = &f.F[(5 * 1 + v) * N];
  const T* F2 = &f.F[(5 * 2 + v) * N];
  return dt * ((F0[X] - F0[g.sh(X, 0, 1)]) / g.h[0] + (F1[X] - F1[g.sh(X, 1, 1)]) / g.h[1] +
               (F2[X] - F2[g.sh(X, 2, 1)]) / g.h[2]);
}
template <class T> T incr_face(const Grid& g, const FluxSet<T>& f, int d, long X, double dt) {
  const long N = g.N;
  const int a = (d + 1) % 3, c = (d + 2) % 3;
  const T* Ec = &f.E[c * N];  // edges at (d: -1/2, a: -1/2) of the cell
  const T* Ea = &f.E[a * N];  // edges at (c: -1/2, d: -1/2)
  return dt / (g.h[a] * g.h[c]) *
         (g.h[c] * Ec[X] + g.h[a] * Ea[g.sh(X, c, 1)] - g.h[c] * Ec[g.sh(X, a, 1)] - g.h[a] * Ea[X]);
}

template <class T> bool cell_invalid(const Grid& g, const std::vector<T>& U, const std::vector<T>& B,
                                     long X, int criteria) {
  const long N = g.N;
  const T rho = U[X];
  T bc[3];
  bool finite = true;
  for (int v = 0; v < 5; ++v) finite = finite && std::isfinite(val(U[v * N + X]));
  for (int d = 0; d < 3; ++d) {
    finite = finite && std::isfinite(val(B[d * N + X]));
    bc[d] = 0.5 * (B[d * N + X] + B[d * N + g.sh(X, d, 1)]);
  }
  if (!finite) return true;
  if (criteria & 4) return true;  // user criterion "every cell invalid" (Sec. 2.5 allows user criteria)
  if ((criteria & 1) && val(rho) <= 0.0) return true;
  if (criteria & 2) {
    T u2 = T(0.0);
    for (int d = 0; d < 3; ++d) {
      const T u = U[(1 + d) * N + X] / rho;
      u2 = u2 + u * u;
    }
    const T p = (g.gamma - 1.0) * (U[4 * N + X] - 0.5 * rho * u2 -
                                   0.5 * (bc[0] * bc[0] + bc[1] * bc[1] + bc[2] * bc[2]));
    if (!(val(p) > 0.0)) return true;
  }
  return false;
}

// Masks of Sec. 2.5 / Fig. (fofc): faces and edges of flagged cells.
void build_masks(const Grid& g, const std::vector<char>& flag, std::vector<char>& fmask,
                 std::vector<char>& emask) {
  const long N = g.N;
  fmask.assign(3 * N, 0);
  emask.assign(3 * N, 0);
  for (long X = 0; X < N; ++X) {
    if (!flag[X]) continue;
    for (int d = 0; d < 3; ++d) {
      fmask[d * N + X] = 1;
      fmask[d * N + g.sh(X, d, 1)] = 1;
      const int a = (d + 1) % 3, c = (d + 2) % 3;
      // the four d-edges of cell X sit at (a, c) offsets {0,1} x {0,1}
      emask[d * N + X] = 1;
      emask[d * N + g.sh(X, a, 1)] = 1;
      emask[d * N + g.sh(X, c, 1)] = 1;
      emask[d * N + g.sh(g.sh(X, a, 1), c, 1)] = 1;
    }
  }
}
bool cell_touched(const Grid& g, const std::vector<char>& fmask, long X) {
  const long N = g.N;
  for (int d = 0; d < 3; ++d)
    if (fmask[d * N + X] || fmask[d * N + g.sh(X, d, 1)]) return true;
  return false;
}
bool face_touched(const Grid& g, const std::vector<char>& emask, int d, long X) {
  const long N = g.N;
  const int a = (d + 1) % 3, c = (d + 2) % 3;
  return emask[c * N + X] || emask[c * N + g.sh(X, a, 1)] || emask[a * N + X] ||
         emask[a * N + g.sh(X, c, 1)];
}

struct StepOut {
  long long flagged[2];
};

// One full step: RK2-SSP with first-order flux correction (Sec. 2.5, Fig. flowchart).
// user_flags[s] (optional, one byte per cell) marks cells a user criterion invalidates after
// stage s (Sec. 2.5 lets users add their own validity criteria).
template <class T>
void step(const Grid& g, const Scheme<T>& sc, int fofc_criteria, std::vector<T>& U,
          std::vector<T>& B, double dt, StepOut& so,
          const unsigned char* const* user_flags = nullptr) {
  const long N = g.N;
  const std::vector<T> U0 = U, B0 = B;
  const Scheme<T> fo = {REC_PC, RS_LLF, sc.emf, sc.eta, sc.resistive};
  FluxSet<T> ffo;
  bool have_fo = false;

  // Stage 1: S^{n+1/2} = S^n + D^n (Eq. rk1:update).
  FluxSet<T> f0;
  fluxes_and_emfs(g, sc, U0, B0, f0);
  set_phase(PH_UPDATE);
  std::vector<T> U1(5 * N), B1(3 * N);
  for (long X = 0; X < N; ++X)
    for (int v = 0; v < 5; ++v) U1[v * N + X] = U0[v * N + X] + incr_cell(g, f0, v, X, dt);
  for (int d = 0; d < 3; ++d)
    for (long X = 0; X < N; ++X) B1[d * N + X] = B0[d * N + X] + incr_face(g, f0, d, X, dt);

  std::vector<char> flag(N, 0), fmask, emask;
  so.flagged[0] = so.flagged[1] = 0;
  if (fofc_criteria) {
    set_phase(PH_FLAG);
    for (long X = 0; X < N; ++X)
      flag[X] = cell_invalid(g, U1, B1, X, fofc_criteria) || (user_flags && user_flags[0] && user_flags[0][X]);
    for (long X = 0; X < N; ++X) so.flagged[0] += flag[X];
  }
  if (so.flagged[0] > 0) {
    g_fo = true;
    set_phase(PH_FO);
    fluxes_and_emfs(g, fo, U0, B0, ffo);
    have_fo = true;
    build_masks(g, flag, fmask, emask);
    for (int d = 0; d < 3; ++d)
      for (long X = 0; X < N; ++X) {
        if (fmask[d * N + X])
          for (int v = 0; v < 5; ++v) f0.F[(5 * d + v) * N + X] = ffo.F[(5 * d + v) * N + X];
        if (emask[d * N + X]) f0.E[d * N + X] = ffo.E[d * N + X];
      }
    for (long X = 0; X < N; ++X)
      if (cell_touched(g, fmask, X))
        for (int v = 0; v < 5; ++v) U1[v * N + X] = U0[v * N + X] + incr_cell(g, f0, v, X, dt);
    for (int d = 0; d < 3; ++d)
      for (long X = 0; X < N; ++X)
        if (face_touched(g, emask, d, X)) B1[d * N + X] = B0[d * N + X] + incr_face(g, f0, d, X, dt);
    g_fo = false;
  }

  // Stage 2: S^{n+1} = S^n + (D^n + D^{n+1/2}) / 2 (Eq. rk2:update).
  FluxSet<T> f1;
  fluxes_and_emfs(g, sc, U1, B1, f1);
  set_phase(PH_UPDATE);
  for (long X = 0; X < N; ++X)
    for (int v = 0; v < 5; ++v)
      U[v * N + X] = U0[v * N + X] + 0.5 * (incr_cell(g, f0, v, X, dt) + incr_cell(g, f1, v, X, dt));
  for (int d = 0; d < 3; ++d)
    for (long X = 0; X < N; ++X)
      B[d * N + X] = B0[d * N + X] + 0.5 * (incr_face(g, f0, d, X, dt) + incr_face(g, f1, d, X, dt));

  if (fofc_criteria) {
    set_phase(PH_FLAG);
    std::fill(flag.begin(), flag.end(), 0);
    for (long X = 0; X < N; ++X)
      flag[X] = cell_invalid(g, U, B, X, fofc_criteria) || (user_flags && user_flags[1] && user_flags[1][X]);
    for (long X = 0; X < N; ++X) so.flagged[1] += flag[X];
  }
  if (so.flagged[1] > 0) {
    g_fo = true;
    set_phase(PH_FO);
    if (!have_fo) fluxes_and_emfs(g, fo, U0, B0, ffo);
    build_masks(g, flag, fmask, emask);
    // RK-averaged fluxes, replaced outright by the cached first-order ones on masked faces.
    FluxSet<T> fm;
    fm.F.resize(15 * N);
    fm.E.resize(3 * N);
    for (int d = 0; d < 3; ++d)
      for (long X = 0; X < N; ++X) {
        for (int v = 0; v < 5; ++v) {
          const long I = (5 * d + v) * N + X;
          fm.F[I] = fmask[d * N + X] ? ffo.F[I] : 0.5 * (f0.F[I] + f1.F[I]);
        }
        fm.E[d * N + X] = emask[d * N + X] ? ffo.E[d * N + X] : 0.5 * (f0.E[d * N + X] + f1.E[d * N + X]);
      }
    for (long X = 0; X < N; ++X)
      if (cell_touched(g, fmask, X))
        for (int v = 0; v < 5; ++v) U[v * N + X] = U0[v * N + X] + incr_cell(g, fm, v, X, dt);
    for (int d = 0; d < 3; ++d)
      for (long X = 0; X < N; ++X)
        if (face_touched(g, emask, d, X)) B[d * N + X] = B0[d * N + X] + incr_face(g, fm, d, X, dt);
    g_fo = false;
  }
}

// Sec. 2.4 time step, reading R10.
double max_dt(const Grid& g, const std::vector<double>& U, const std::vector<double>& B,
              double cfl, double eta) {
  std::vector<double> P;
  cons_to_prim(g, U, B, P);
  const long N = g.N;
  const double hmin = std::fmin(g.h[0], std::fmin(g.h[1], g.h[2]));
  double smax = 2.0 * eta / hmin;
  for (long X = 0; X < N; ++X) {
    for (int d = 0; d < 3; ++d) {
      const int a = (d + 1) % 3, c = (d + 2) % 3;
      double W[7] = {P[P_RHO * N + X], P[(P_U + d) * N + X], P[(P_U + a) * N + X],
                     P[(P_U + c) * N + X], P[P_P * N + X], P[(P_B + a) * N + X],
                     P[(P_B + c) * N + X]};
      const double cf = fast_speed(g.gamma, W, P[(P_B + d) * N + X]);
      const double s = (std::fabs(W[1]) + cf) / g.h[d] * hmin;
      if (s > smax) smax = s;
    }
  }
  return cfl * hmin / smax;
}

Grid make_grid(const int* n, const double* h, double gamma) {
  Grid g;
  for (int d = 0; d < 3; ++d) { g.n[d] = n[d]; g.h[d] = h[d]; }
  g.N = (long)n[0] * n[1] * n[2];
  g.gamma = gamma;
  return g;
}

}  // namespace

// ---------------------------------------------------------------------------------------
// C interface (ctypes). Arrays are plain host doubles in the layout given at the top.
// ---------------------------------------------------------------------------------------
extern "C" {

typedef struct {
  int n[3];
  double h[3];
  double gamma;
  int recon, riemann, emf;
  int fofc_criteria;  // bit 0: rho <= 0, bit 1: p <= 0, bit 2: every cell; 0 disables correction
  double eta;
} oracle_cfg;

static Scheme<double> scheme_of(const oracle_cfg* c) {
  return Scheme<double>{c->recon, c->riemann, c->emf, c->eta, c->eta != 0.0};
}

// One full step in place. cons: 5N, b: 3N. counts[2] <- flagged cells per stage.
int oracle_step(const oracle_cfg* c, double* cons, double* b, double dt, long long* counts) {
  Grid g = make_grid(c->n, c->h, c->gamma);
  std::vector<double> U(cons, cons + 5 * g.N), B(b, b + 3 * g.N);
  StepOut so;
  step(g, scheme_of(c), c->fofc_criteria, U, B, dt, so);
  std::memcpy(cons, U.data(), sizeof(double) * 5 * g.N);
  std::memcpy(b, B.data(), sizeof(double) * 3 * g.N);
  if (counts) { counts[0] = so.flagged[0]; counts[1] = so.flagged[1]; }
  return 0;
}

// One full step with user-flagged cells per stage (NULL = none) on top of the criteria.
int oracle_step_flags(const oracle_cfg* c, double* cons, double* b, double dt,
                      const unsigned char* user1, const unsigned char* user2, long long* counts) {
  Grid g = make_grid(c->n, c->h, c->gamma);
  std::vector<double> U(cons, cons + 5 * g.N), B(b, b + 3 * g.N);
  StepOut so;
  const unsigned char* uf[2] = {user1, user2};
  step(g, scheme_of(c), c->fofc_criteria, U, B, dt, so, uf);
  std::memcpy(cons, U.data(), sizeof(double) * 5 * g.N);
  std::memcpy(b, B.data(), sizeof(double) * 3 * g.N);
  if (counts) { counts[0] = so.flagged[0]; counts[1] = so.flagged[1]; }
  return 0;
}

// Fluxes (15N: [d][v][X]) and EMFs (3N) of one state, with the configured scheme.
int oracle_fluxes(const oracle_cfg* c, const double* cons, const double* b, double* flux,
                  double* emf) {
  Grid g = make_grid(c->n, c->h, c->gamma);
  std::vector<double> U(cons, cons + 5 * g.N), B(b, b + 3 * g.N);
  FluxSet<double> f;
  fluxes_and_emfs(g, scheme_of(c), U, B, f);
  std::memcpy(flux, f.F.data(), sizeof(double) * 15 * g.N);
  std::memcpy(emf, f.E.data(), sizeof(double) * 3 * g.N);
  return 0;
}

// The four corner EMFs of every edge (12N: [e][q][X], q = 0 LB, 1 RB, 2 LT, 3 RT, where L/R
// are the sides of the a-face and B/T those of the c-face, a = e+1, c = e+2) of one state,
// as the configured EMF compute scheme forms them before the averaging of Eq. (ld04).
int oracle_corner_emfs(const oracle_cfg* c, const double* cons, const double* b, double* corners) {
  Grid g = make_grid(c->n, c->h, c->gamma);
  std::vector<double> U(cons, cons + 5 * g.N), B(b, b + 3 * g.N);
  FluxSet<double> f;
  f.keep_corners = true;
  fluxes_and_emfs(g, scheme_of(c), U, B, f);
  std::memcpy(corners, f.C.data(), sizeof(double) * 12 * g.N);
  return 0;
}

// Fluxes and EMFs of one state with their directional derivative along (dcons, db), on dual
// numbers (the branches taken on the values): flux, emf as in oracle_fluxes, dflux, demf tangents.
int oracle_fluxes_jvp(const oracle_cfg* c, const double* cons, const double* b, const double* dcons,
                      const double* db, double* flux, double* emf, double* dflux, double* demf) {
  Grid g = make_grid(c->n, c->h, c->gamma);
  const long N = g.N;
  std::vector<Dual> U(5 * N), B(3 * N);
  for (long i = 0; i < 5 * N; ++i) U[i] = Dual(cons[i], dcons[i]);
  for (long i = 0; i < 3 * N; ++i) B[i] = Dual(b[i], db[i]);
  const Scheme<Dual> sc = {c->recon, c->riemann, c->emf, Dual(c->eta, 0.0), c->eta != 0.0};
  FluxSet<Dual> f;
  fluxes_and_emfs(g, sc, U, B, f);
  for (long i = 0; i < 15 * N; ++i) { flux[i] = f.F[i].v; dflux[i] = f.F[i].t; }
  for (long i = 0; i < 3 * N; ++i) { emf[i] = f.E[i].v; demf[i] = f.E[i].t; }
  return 0;
}

// Primitive variables (8N) of one state.
int oracle_prim(const oracle_cfg* c, const double* cons, const double* b, double* prim) {
  Grid g = make_grid(c->n, c->h, c->gamma);
  std::vector<double> U(cons, cons + 5 * g.N), B(b, b + 3 * g.N), P;
  cons_to_prim(g, U, B, P);
  std::memcpy(prim, P.data(), sizeof(double) * 8 * g.N);
  return 0;
}

// Reconstruction of one periodic array along direction d: qm/qp at X -/+ 1/2.
int oracle_recon(const oracle_cfg* c, int method, const double* q, int d, double* qm, double* qp) {
  Grid g = make_grid(c->n, c->h, c->gamma);
  std::vector<double> m, p;
  recon_field(g, method, q, d, m, p);
  std::memcpy(qm, m.data(), sizeof(double) * g.N);
  std::memcpy(qp, p.data(), sizeof(double) * g.N);
  return 0;
}

// One face Riemann problem in the face frame: out = {F[5], alpha+, alpha-, u*}.
int oracle_riemann(int solver, double gamma, const double* WL, const double* WR, double bn,
                   double* out) {
  double F[5], ap, am, us;
  riemann(solver, gamma, WL, WR, bn, F, ap, am, us);
  for (int v = 0; v < 5; ++v) out[v] = F[v];
  out[5] = ap; out[6] = am; out[7] = us;
  return 0;
}

double oracle_max_dt(const oracle_cfg* c, const double* cons, const double* b, double cfl) {
  Grid g = make_grid(c->n, c->h, c->gamma);
  std::vector<double> U(cons, cons + 5 * g.N), B(b, b + 3 * g.N);
  return max_dt(g, U, B, cfl, c->eta);
}

// max over cells of |sum_d (b_d(+1/2) - b_d(-1/2)) / h_d| and max over faces of |b_d|.
void oracle_divb(const oracle_cfg* c, const double* b, double* maxdiv, double* maxb) {
  Grid g = make_grid(c->n, c->h, c->gamma);
  const long N = g.N;
  double md = 0, mb = 0;
  for (long X = 0; X < N; ++X) {
    double dv = 0;
    for (int d = 0; d < 3; ++d) {
      dv += (b[d * N + g.sh(X, d, 1)] - b[d * N + X]) / g.h[d];
      mb = std::fmax(mb, std::fabs(b[d * N + X]));
    }
    md = std::fmax(md, std::fabs(dv));
  }
  *maxdiv = md;
  *maxb = mb;
}

// Forward-mode derivative of `nsteps` steps with a frozen dt sequence: the state advances in
// place and (dcons, db) advance as its tangent; deta is the tangent of eta.
int oracle_steps_jvp(const oracle_cfg* c, double* cons, double* b, double* dcons, double* db,
                     double deta, const double* dts, int nsteps) {
  Grid g = make_grid(c->n, c->h, c->gamma);
  const long N = g.N;
  std::vector<Dual> U(5 * N), B(3 * N);
  for (long i = 0; i < 5 * N; ++i) U[i] = Dual(cons[i], dcons[i]);
  for (long i = 0; i < 3 * N; ++i) B[i] = Dual(b[i], db[i]);
  const Scheme<Dual> sc = {c->recon, c->riemann, c->emf, Dual(c->eta, deta),
                           c->eta != 0.0 || deta != 0.0};
  for (int s = 0; s < nsteps; ++s) {
    StepOut so;
    step(g, sc, c->fofc_criteria, U, B, dts[s], so);
  }
  for (long i = 0; i < 5 * N; ++i) { cons[i] = U[i].v; dcons[i] = U[i].t; }
  for (long i = 0; i < 3 * N; ++i) { b[i] = B[i].v; db[i] = B[i].t; }
  return 0;
}

// FP64 operations (+, -, *, /, sqrt) of one step, by phase: prim, face reconstruction, Riemann
// solves, edge EMFs, Joule flux, update, flags, first-order correction; *hlld_unused (if not NULL)
// the Riemann-phase operations that a one-sided HLLD would not form. Returns the phase count.
int oracle_count_ops(const oracle_cfg* c, const double* cons, const double* b, double dt,
                     long long* ops_by_phase, long long* counts, long long* hlld_unused) {
  Grid g = make_grid(c->n, c->h, c->gamma);
  const long N = g.N;
  std::vector<Cnt> U(5 * N), B(3 * N);
  for (long i = 0; i < 5 * N; ++i) U[i] = Cnt(cons[i]);
  for (long i = 0; i < 3 * N; ++i) B[i] = Cnt(b[i]);
  for (int p = 0; p < NPHASE; ++p) g_ops[p] = 0;
  g_hlld_unused = 0;
  g_fo = false;
  const Scheme<Cnt> sc = {c->recon, c->riemann, c->emf, Cnt(c->eta), c->eta != 0.0};
  StepOut so;
  step(g, sc, c->fofc_criteria, U, B, dt, so);
  for (int p = 0; p < NPHASE; ++p) ops_by_phase[p] = g_ops[p];
  if (hlld_unused) *hlld_unused = g_hlld_unused;
  if (counts) { counts[0] = so.flagged[0]; counts[1] = so.flagged[1]; }
  return NPHASE;
}

}  // extern "C"
