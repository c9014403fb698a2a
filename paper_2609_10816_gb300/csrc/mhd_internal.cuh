// mhd_internal.cuh -- parameters shared by the kernel translation units and the host API.
#pragma once
#include <cuda_runtime.h>

#include "../../include/mhd.h"

namespace mhd {

// three device pointers passed by value
struct Ptr3 {
  const double* p[3];
};

// Everything one stage's kernels need, passed by value. Arrays are SoA over the N cells of a
// periodic box, x fastest; face arrays and edge arrays use the cell's linear index (the face or
// edge at the cell's lower half-index, as documented in include/mhd.h).
struct Dev {
  int n[3];
  long long N;
  long long stride[3];  // 1, nx, nx*ny
  double h[3];
  double hinv[3];
  double gam, gm1inv;
  double dt, eta;
  double dth[3];        // dt / h_d
  const double* dthp;   // when set, dt / h_d are read from device memory here instead (a step whose
                        // dt comes from the device-side CFL reduction)
  int resistive;        // eta != 0
  int combine;          // stage 2: store (old + new) / 2 into fluxes and EMFs
  int fofc_criteria;    // bit 0 rho <= 0, bit 1 p <= 0
  int emf;              // EMF compute scheme
  // S^n (caller, read only), stage input, stage output
  const double* U0;
  const double* B0[3];
  const double* Uin;
  const double* Bin[3];
  double* Uout;
  double* Bout[3];
  // scratch
  double* P;      // [8][N] rho, u0, u1, u2, p, bc0, bc1, bc2 of the stage input
  double* F;      // [3][5][N] face fluxes (flux of cons[v] across the d-face at X - d/2)
  double* Ap;     // [3][N] alpha+ on d-faces
  double* Am;     // [3][N] alpha-
  double* Us;     // [3][N] Q26 face-normal velocity u_d^*
  double* Epart;  // [3][4][N] per e-edge: b_a^B, b_a^T, u_a^B, u_a^T (reconstructed along c)
  double* E;      // [3][N] edge EMFs
  // FS18 / B25a extras
  double* VL;     // [3][3][N] FS18: left velocity states on d-faces, component k
  double* VR;     // [3][3][N]
  double* Xpart;  // [3][8][N] FS18/B25a per e-edge corner partials of the a-faces sweep
  double* EfL;    // [3][2][N] B25a e-EMF on a-faces (L/R) for order (a then c)
  double* EfB;    // [3][2][N] B25a e-EMF on c-faces (B/T) for order (c then a)
  unsigned char* flag;         // [N]
  double* Pnext;  // when set, the flag pass also writes the primitives of its state here (the next
                  // stage's input, whose prim pass then runs only if flux correction changed it)
  double* LR;     // when set, the face sweep also stores its reconstructed left (7) and right (7)
                  // face states here, [3][14][N] (for the adjoint)
  double* EdgeC;  // when set, the c-face edge sweep also stores its reconstructed left / right
                  // values here (for the adjoint): Q26 b_c and u_c*, [3][4][N]; FS18 b_c and the
                  // four c-face velocity states, [3][10][N]; B25a b_c and the two c-face EMF
                  // values, in the first 6 of [3][10][N]
  unsigned long long* counters;  // [0] stage-1 flagged cells, [1] stage-2, [2..3] reductions
  // work-list cursors of the dynamically scheduled sweeps ([dir] face, [3 + e] edge_bt,
  // [6 + e] edge_lr), zeroed before every stage; NULL: one segment per thread, no cursor
  unsigned long long* work;
  int stage;      // 0 or 1 (which counter the flux correction reads)
};

// Work slots of the dynamically scheduled sweeps of one stage.
constexpr int kWorkSlots = 9;

// Adjoint of the flux function at a stage input state (mhd_adjoint.cu).
struct AdjDev {
  Dev D;                // forward parameters at the state (P, Ap, Am, Us recomputed for it)
  const double* lF;     // [3][5][N] adjoint of the face fluxes
  const double* lE;     // [3][N] adjoint of the edge EMFs
  double* lAp;          // [3][N] adjoint of alpha+ on faces
  double* lAm;          // [3][N] adjoint of alpha-
  double* lUs;          // [3][N] adjoint of the Q26 face velocity
  double* lEdge;        // adjoint of the reconstructed edge values per e-edge: Q26 [3][8][N] baB, baT,
                        // uaB, uaT, bcL, bcR, ucL, ucR; FS18 [3][20][N] baB, baT, bcL, bcR, the 8
                        // a-then-c velocity partials, the 8 c-then-a ones; B25a [3][12][N] baB, baT,
                        // bcL, bcR, the 4 a-then-c EMF partials, the 4 c-then-a ones
  double* lEf;          // B25a: [2][3][2][N] adjoint of the face EMF values (EfL, then EfB)
  double* eps;          // B25a: [3][N] the cell-centred EMF of the stage input (formed here)
  double* leps;         // B25a: [3][N] its adjoint
  double* lLR;          // [3][14][N] adjoint of the left (7) and right (7) face states (accumulated)
  double* lP;           // [8][N] adjoint of the primitives
  double* lU;           // [5][N] output: adjoint of the conserved variables (accumulated)
  double* lB;           // [3][N] output: adjoint of the face field (accumulated, atomics)
  double* lEta;         // [1] output: d/d(eta) (accumulated, atomics)
};

void launch_adj_flux(const AdjDev& A, int recon, int rs, cudaStream_t st);
void launch_adj_update(const Dev& D, const double* lU, const double* lB, double* lF, double* lE, double scale,
                       double s_old, cudaStream_t st);
void launch_axpy3(long long n, double* y, const double* a, const double* b, cudaStream_t st);
void launch_adj_mask(const Dev& D, const unsigned char* fl, const double* gF, const double* gE, double* lF,
                     double* lE, double scale, cudaStream_t st);
void launch_adj_fo(const AdjDev& A, const unsigned char* fl1, const unsigned char* fl2, const double* gF,
                   const double* gE, const double* kF, const double* kE, cudaStream_t st);
void launch_vjp_check(long long n, unsigned long long seed, double gam, int rs, unsigned long long* out,
                      cudaStream_t st);

// blocks of `threads` threads of kernel `fn` that fit on the device at once (all SMs), for the
// persistent launches of the dynamically scheduled sweeps; cached per kernel
int resident_blocks(const void* fn, int threads);

// message reported by mhd_create_error() for calls that have no context
void set_call_error(const char* msg);

// launchers (each enqueues on `st`)
void launch_prim(const Dev& d, cudaStream_t st);
void launch_face(const Dev& d, int dir, int recon, int rs, int seg, cudaStream_t st);
// the three face sweeps (one launch when d.work holds cursors, else one per direction); returns
// the number of launches
int launch_faces(const Dev& d, int recon, int rs, int seg, cudaStream_t st);
void launch_edges_bt(const Dev& d, int recon, int seg, cudaStream_t st);
void launch_edges_lr(const Dev& d, int recon, int seg, cudaStream_t st);
void launch_update(const Dev& d, cudaStream_t st);
void launch_flag(const Dev& d, cudaStream_t st);
// dt of Eq. (resistivity:cfl) from the reduction's maximum signal speed (bit pattern at smax_bits):
// out[0] = dt, out[1..3] = dt / h_d, out[4] = 1 when the speed is zero or not finite (dt = 0)
void launch_set_dt(const unsigned long long* smax_bits, double cfl, double eta, double hmin, const double* hinv,
                   double* out, cudaStream_t st);
void launch_prim_if_flagged(const Dev& d, int prev_stage, cudaStream_t st);
void launch_fofc(const Dev& d, cudaStream_t st);
// Pout (may be NULL): the primitives of U, B written as the reduction forms them
void launch_maxspeed(const Dev& d, const double* U, Ptr3 B, unsigned long long* out, cudaStream_t st,
                     double* Pout = nullptr);
void launch_divb(const Dev& d, Ptr3 B, unsigned long long* out, cudaStream_t st);
void launch_math_check(long long n, unsigned long long* out, cudaStream_t st);

}  // namespace mhd
