/*
 * mhd.h -- C ABI of the GB300 constrained-transport MHD step library (libmhd.so).
 *
 * The library advances the cell-centred conserved state and the face-centred magnetic field
 * of one uniform, triply periodic patch by one step of the second-order constrained-transport
 * (CT) MHD method of "Magnetising the QUOKKA code" (Sec. 2): reconstruction of primitive
 * states (Sec. 2.2), Riemann fluxes (Sec. 2.2), edge EMFs from a compute scheme and the LD04
 * average (Sec. 2.3, Eqs. q26, fs18, b25a-*, alpha-edge, ld04), a constant-eta Ohmic EMF with
 * its Joule energy flux (Sec. 2.4, Eqs. current-stencil, emf-update), the discrete Stokes
 * update of the face field (Eqs. dbdt:discrete, rk:increment-bfield) and RK2-SSP with
 * first-order flux correction (Sec. 2.5, Eqs. rk:increment-state, rk1:update, rk2:update).
 * Every computation runs in FP64 CUDA kernels on the device; nothing falls back to the host.
 *
 * Memory layout (all arrays are caller-owned DEVICE memory, float64, x fastest):
 *   cell X = (i, j, k), 0 <= i < nx, ... ; linear index X = (k*ny + j)*nx + i
 *   cons : [5][nz][ny][nx]  rho, rho*u0, rho*u1, rho*u2, e_tot        (Eq. state:conserved)
 *   b0   : [nz][ny][nx]     b0 on the x0-face of cell X at i - 1/2    (Sec. 2.1)
 *   b1   : [nz][ny][nx]     b1 on the x1-face at j - 1/2
 *   b2   : [nz][ny][nx]     b2 on the x2-face at k - 1/2
 * Periodicity means face i = nx is face i = 0.
 *
 * Errors: every call returns an mhd_status; no call traps on the device. Argument errors are
 * detected on the host before any launch. mhd_last_error() gives a message for the last
 * failure on a context. Calls are asynchronous on the context's stream unless stated.
 */
#ifndef MHD_GB300_H
#define MHD_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MHD_OK = 0,
  MHD_ERR_ARG = 1,         /* bad argument (null pointer, size, dt <= 0, eta < 0, scheme bits) */
  MHD_ERR_CUDA = 2,        /* a CUDA runtime call failed; see mhd_last_error */
  MHD_ERR_NONFINITE = 3,   /* a non-finite value was produced and flux correction was off */
  MHD_ERR_UNSUPPORTED = 4, /* a scheme the paper names but does not define (B25b averaging) */
  MHD_ERR_TIMEOUT = 5      /* a bounded device wait gave up (persistent batched kernel) */
} mhd_status;

/* Scheme bit field (Sec. 2.2-2.5). Reconstruction in bits 0-3, Riemann solver in bits 4-7,
 * EMF compute in bits 8-11, EMF averaging in bits 12-15, flags above. */
enum {
  MHD_RECON_PC = 0,          /* piecewise constant (Sec. 2.2) */
  MHD_RECON_PLM_MC = 1,      /* piecewise linear, monotonised-central limiter */
  MHD_RECON_PLM_MINMOD = 2,  /* piecewise linear, minmod limiter */
  MHD_RECON_PPM = 3,         /* piecewise parabolic, Colella & Woodward 1984 limiting */
  MHD_RECON_PPM_EP = 4,      /* extremum-preserving PPM (Sec. 2.2, citing Rider, Greenough & Kamm
                                2007): fourth-order interfaces, CW84 limiting relaxed at smooth
                                extrema */
  MHD_RIEMANN_HLL = 0 << 4,  /* two-wave HLL with the Eq. (alpha-pm) speeds */
  MHD_RIEMANN_HLLD = 1 << 4, /* Miyoshi & Kusano 2005 HLLD */
  MHD_RIEMANN_LLF = 2 << 4,  /* local Lax-Friedrichs (Rusanov) */
  MHD_EMF_Q26 = 0 << 8,      /* the paper's new compute scheme, Eqs. (q26-facevel), (q26) */
  MHD_EMF_FS18 = 1 << 8,     /* Felker & Stone 2018, Eqs. (fs18-average), (fs18) */
  MHD_EMF_B25A = 2 << 8,     /* Balsara 2025a, Eqs. (b25a-b-avg), (b25a-emf-centre), (b25a-average) */
  MHD_AVG_LD04 = 0 << 12,    /* Londrillo & Del Zanna 2004 2D-HLL average, Eq. (ld04) */
  MHD_AVG_B25B = 1 << 12,    /* Balsara 2025b 2D Riemann solver: not defined -> UNSUPPORTED */
  MHD_FOFC_OFF = 1 << 16     /* disable first-order flux correction */
};

typedef struct {
  int nx, ny, nz;          /* cells per direction, each >= 1 */
  double dx, dy, dz;       /* cell widths, > 0 */
  double gamma;            /* adiabatic index, > 1 */
  int fofc_criteria;       /* bit 0: rho <= 0, bit 1: p <= 0 invalidate a cell; 0 means 3.
                              A non-finite value always invalidates a cell. */
} mhd_config;

typedef struct {
  double *cons;            /* [5][nz][ny][nx], device */
  double *b0, *b1, *b2;    /* [nz][ny][nx] each, device */
} mhd_state;

typedef struct mhd_ctx mhd_ctx; /* opaque: owns the scratch of one patch size and a stream */

/* Create a context for one patch size. `cuda_stream` is a cudaStream_t (NULL = legacy default
 * stream); all work of the context is enqueued on it. Allocates the step's scratch
 * (109 doubles and one byte per cell, the FS18 / B25a intermediates included) with cudaMalloc on
 * the current device; the first mhd_step_adjoint adds 414 doubles per cell. *out is NULL on
 * error. */
mhd_status mhd_create(const mhd_config *cfg, void *cuda_stream, mhd_ctx **out);

/* Free the context and its scratch (synchronises the stream first). NULL is ignored. */
void mhd_destroy(mhd_ctx *ctx);

/* One full step of size dt in place (Sec. 2.5): stage 1, flux correction, stage 2, flux
 * correction; state->cons/b* hold S^{n+1} when the stream reaches the end of the call.
 * dt > 0 is fixed within the step, eta >= 0 is the constant Ohmic resistivity (Eq.
 * resistivity:ohms-law; eta = 0 reduces exactly to the ideal scheme). Asynchronous. */
mhd_status mhd_step(mhd_ctx *ctx, const mhd_state *state, double dt, int scheme, double eta);

/* Largest stable step (Sec. 2.4, Eq. resistivity:cfl): dt = cfl * dx_min / max over cells of
 * max(max_d (|u_d| + c_fm,d) dx_min / dx_d, 2 eta / dx_min). Synchronous (reads one double).
 * MHD_ERR_NONFINITE when a cell holds a value that is not finite, or the largest speed is zero or
 * infinite (a speed that is not a number, which a cell with p < 0 or rho <= 0 can give, is passed
 * over). */
mhd_status mhd_max_dt(mhd_ctx *ctx, const mhd_state *state, double cfl, double eta, double *dt_out);

/* mhd_max_dt followed by mhd_step without the host in between: the CFL reduction, dt (the same
 * formula and value as mhd_max_dt's) and dt / dx_d stay in the context's device memory and the
 * step's kernels read them there, so consecutive calls queue on the stream without a
 * synchronisation (and a sequence of them can be recorded in a CUDA graph). cfl > 0 and eta >= 0
 * finite. Where mhd_max_dt would report MHD_ERR_NONFINITE, the step runs with dt = 0 (the state
 * is then unchanged wherever its fluxes are finite) and mhd_last_dt reports MHD_ERR_NONFINITE.
 * Asynchronous. On boxes of at most 128^3 cells, a call with the same state arrays, scheme, cfl
 * and eta as the previous call (not while profiling, not while the stream is being captured)
 * records the step's launches once as a CUDA graph on a private stream and replays it with one
 * launch per call, for as long as the arguments repeat: the same kernels and results, without
 * the host's launch cost. */
mhd_status mhd_step_cfl(mhd_ctx *ctx, const mhd_state *state, double cfl, int scheme, double eta);

/* The dt of the last mhd_step_cfl on this context (0 before any). Synchronous (reads two
 * doubles); MHD_ERR_NONFINITE when that step found no finite, positive signal speed. */
mhd_status mhd_last_dt(mhd_ctx *ctx, double *dt_out);

/* Discrete divergence diagnostic (Sec. 2.1; Sec. 4.6 validation): max over cells of
 * |sum_d (b_d(+1/2) - b_d(-1/2)) / dx_d| and max over faces of |b_d|. Synchronous. */
mhd_status mhd_divb(mhd_ctx *ctx, const mhd_state *state, double *max_abs_divb, double *max_abs_b);

/* Cells flagged invalid by first-order flux correction in stage 1 and stage 2 of the last
 * mhd_step or mhd_step_cfl (Sec. 2.5). Synchronous. */
mhd_status mhd_stats(mhd_ctx *ctx, long long *fofc_cells_stage1, long long *fofc_cells_stage2);

/* Kernel classes reported by mhd_profile_read (one entry per class; a class may cover several
 * launches per stage). */
enum {
  MHD_K_PRIM = 0,      /* cons -> prim */
  MHD_K_FACE = 1,      /* reconstruction + Riemann sweeps, 1 launch per stage (all directions) */
  MHD_K_EDGE_BT = 2,   /* a-face quantities to edges along c, 1 launch per stage (B25a: + 6) */
  MHD_K_EDGE_LR = 3,   /* c-face quantities to edges along a + LD04 + eta j, 1 per stage */
  MHD_K_UPDATE = 4,    /* flux divergence and CT update */
  MHD_K_FLAG = 5,      /* validity flags */
  MHD_K_FOFC = 6,      /* first-order flux correction, 3 launches per stage (exit early if no flag) */
  MHD_K_MAXSPEED = 7,  /* CFL reduction (and, in mhd_step_cfl, the dt kernel) */
  MHD_K_DIVB = 8,      /* divergence reduction */
  MHD_K_EXTRA = 9,     /* scheme-specific extras (FS18 / B25a sweeps) */
  MHD_K_COUNT = 16
};

/* Start (enable != 0) or stop per-kernel timing on ctx: while enabled, every launch of the
 * library is bracketed by CUDA events on the context's stream. Starting clears the totals.
 * Launch counts are kept whether or not timing is enabled. */
mhd_status mhd_profile(mhd_ctx *ctx, int enable);

/* Synchronise the stream and return, per kernel class, the summed device time in ms of the
 * launches timed since mhd_profile(ctx, 1) (NULL allowed) and the number of launches since the
 * context was created or the counts were last read with reset != 0. Arrays hold MHD_K_COUNT. */
mhd_status mhd_profile_read(mhd_ctx *ctx, double *total_ms, long long *launches, int reset);

/* Adjoint (vector-Jacobian product) of one mhd_step with a frozen dt: on entry `lam` holds
 * dL/dS^{n+1} (same layout as the state), on return dL/dS^n; *dL_deta (if not NULL) is increased
 * by the step's contribution to dL/d(eta). `state` is S^n (unchanged). Limiters, min/max and
 * Riemann-fan branches are differentiated on the branch the forward step takes (the forward
 * stages are recomputed inside, up to the stage-2 flags). Flux correction (Sec. 2.5) is
 * differentiated with the cells it flagged held fixed: the first-order fluxes and EMFs of S^n on
 * the masked faces and edges get their share of the adjoint, the high-order ones the rest. The
 * paper has no counterpart; it makes the step usable inside gradient-based workflows. Covers every
 * EMF compute scheme (Q26, FS18, B25a); the first call allocates 414 doubles per cell of adjoint
 * scratch. Synchronous when dL_deta is not NULL. */
mhd_status mhd_step_adjoint(mhd_ctx *ctx, const mhd_state *state, const mhd_state *lam, double dt, int scheme,
                            double eta, double *dL_deta);

/* Self-check of the arithmetic the kernels use in place of FP64 instructions: on n pseudo-random
 * positive inputs spread over [2^-40, 2^40], max_rel_err[0..2] receive the largest relative
 * differences of the reciprocal, reciprocal square root and square root (hardware approximation +
 * one third-order Newton correction) from CUDA's IEEE 1/x, 1/sqrt(x) and sqrt(x); on n raw bit
 * patterns (subnormal, smallest, largest and non-finite binades among them), max_rel_err[3] and
 * [4] receive how many times the integer-pipe halving and quadrupling differ in any bit from the
 * FP64 multiplies by 0.5 and 4, and max_rel_err[5] on n pairs of non-NaN doubles (zeros,
 * subnormals, extreme binades and infinities among them) how many times an integer-pipe sign
 * test, comparison, min/max, |x|, sign copy or sign flip disagrees with the IEEE operation;
 * max_rel_err[6] on n pairs (nearby and extreme exponents, few significand bits for exact
 * products and ties, any bit pattern, small integers and zeros) how many times the integer-pipe
 * multiply of mhd_fp64_rate's kinds 4-6 differs in any bit from the FP64 multiply (0 expected
 * for all four; -0 and +0 are ordered -0 < +0 by the kernels' comparisons, which the check
 * allows). max_rel_err holds 7 doubles. Synchronous. The paper has no counterpart. */
mhd_status mhd_math_check(mhd_ctx *ctx, long long n, double *max_rel_err);

/* Measured rate of one FP64 instruction kind on the current GPU (the pipe that bounds every
 * kernel of the step, hence the denominator of its roofline; the paper has no counterpart):
 * kind 0 DFMA, 1 DADD, 2 DMUL, 3 FP32 FFMA for comparison. Independent chains (eight per
 * thread, 8 blocks of 256 threads per SM) run `iters` steps each, timed with CUDA events on
 * `cuda_stream` after a shorter warm-up; *ops_per_s receives instructions per second (per
 * thread-lane). Kinds 4-6 measure a binary64 multiply done on the integer pipe (bit for bit the
 * FP64 multiply; mhd_math_check verifies it) that the step's kernels do not use: 4 eight chains
 * of it, 5 four chains of it beside four DFMA chains, 6 the same mix at 2 blocks of 128 threads
 * per SM (the face sweep's occupancy); *ops_per_s counts the operations of all chains. Kinds 7
 * and 8 run the DFMA chains on 16 and 8 lanes of every warp (the other lanes exit at once) and
 * count the active lanes' operations only: the cost of FP64 work in a divergent branch.
 * Synchronous; allocates 8 bytes of device memory for the duration of the call.
 * MHD_ERR_ARG for a kind outside 0-8 or iters outside [1, 2^30]. */
mhd_status mhd_fp64_rate(int kind, long long iters, void *cuda_stream, double *ops_per_s);

/* Self-check of the adjoint's reverse sweep through the face solve (the Riemann solver of
 * `scheme`'s bits 4-7; mhd_step_adjoint uses it): on n hashed face problems (seed), from equal
 * states to extreme ones, with zero normal field and field along the normal among them, and
 * random output weights, it compares the reverse-mode gradient of the weighted fluxes, speeds
 * and face velocity in the 15 inputs with the same gradient from 15 forward-mode dual-number
 * passes. max_rel_err (7 doubles) receives the largest |difference| / |dual gradient|_inf over
 * all problems, then per kind of problem: equal states, nearby states, no normal field, field
 * along the normal, near-vacuum pressure, large velocities and fields. Synchronous. The paper
 * has no counterpart. */
mhd_status mhd_adjoint_check(mhd_ctx *ctx, long long n, int scheme, unsigned long long seed, double *max_rel_err);

/* Message of the last failure on ctx ("" if none). Valid until the next call on ctx. */
const char *mhd_last_error(const mhd_ctx *ctx);

/* Message for a failure of a call that returns no context (mhd_create, mhd_step_noalloc). */
const char *mhd_create_error(void);

/* Largest box (nx * ny * nz) that mhd_step_noalloc accepts. */
#define MHD_NOALLOC_MAX_CELLS 32768

/* mhd_step without any device allocation, for callers that cannot let a library allocate:
 * applications whose own memory manager owns all device memory (a pool that hands out every byte
 * and cannot have a library allocate beside it), and loops that cannot afford cudaMalloc's
 * implicit device synchronisation. The paper has no counterpart: this is a deployment variant of
 * mhd_step, with the same arguments and results, for boxes of at most MHD_NOALLOC_MAX_CELLS
 * cells and the Q26 EMF compute (FS18/B25a -> MHD_ERR_UNSUPPORTED). Larger boxes are rejected
 * with MHD_ERR_ARG (message from mhd_create_error) before any device work.
 *
 * The step's scratch is one fixed device array (about 14.5 MB) built into libmhd.so; every GPU
 * that loads the library holds it until the process exits. The first call on a device looks up
 * that array's device address (cudaGetSymbolAddress, with that device current), so make the
 * first call on each device before any stream capture. All calls share the one array and the
 * array keeps the last call's contents (the call clears what must start at zero): calls whose
 * work overlaps on the GPU (other streams, other host threads without ordering) race and give
 * wrong results. The caller passes inputs and outputs (state, in place) and the stream;
 * errors as for mhd_step. Asynchronous on `cuda_stream`. */
mhd_status mhd_step_noalloc(const mhd_config *cfg, const mhd_state *state, double dt, int scheme,
                            double eta, void *cuda_stream);

/* ---- batched form: many uneven periodic patches advanced together ----------------------
 * A batch is a list of independent triply periodic patches of sizes dims[3p..3p+2] = (nx, ny, nz)
 * and common cell width h (one refinement level of an AMR hierarchy, each patch its own periodic
 * box). One step advances every patch by the same dt = cfl h / (max over all cells of all patches
 * of the CFL signal speed, Eq. resistivity:cfl), computed on the device. Each RK stage runs as one
 * persistent cooperative launch over all patches (grid-wide barriers with a bounded wait between
 * its phases), or as three (mhd_batch_set_launches): the face sweeps at the face kernel's register
 * budget; the edge sweeps, update and validity flags at half that budget (twice the warps per
 * SM); and, with flux correction on, the first-order correction (returning at once when the stage
 * flagged nothing). The whole step is captured once
 * as a CUDA graph and replayed while the state arrays, scheme, eta and cfl stay the same. Every
 * EMF compute scheme (Q26, FS18, B25a) with LD04 averaging; B25b -> MHD_ERR_UNSUPPORTED. */
typedef struct mhd_batch mhd_batch;

/* Batch state, patch-major, all device memory: patch p (cell offset off[p] from
 * mhd_batch_offsets) holds cons at cons + 5 off[p] as [5][nz][ny][nx] and its face fields at
 * b + 3 off[p] as [3][nz][ny][nx] (b0, b1, b2 of the patch, same layout as mhd_state). */
typedef struct {
  double *cons;
  double *b;
} mhd_batch_state;

/* Create a batch of npatch patches (dims: 3 ints per patch, each >= 1, fewer than 2^31 cells per
 * patch) with cell width h > 0. Allocates 55 doubles and one byte of scratch per cell (the first
 * FS18 or B25a step 54 doubles per cell more, kept until mhd_batch_destroy). Errors: message from
 * mhd_batch_last_error(NULL). */
mhd_status mhd_batch_create(const int *dims, int npatch, double h, double gamma, void *cuda_stream,
                            mhd_batch **out);
void mhd_batch_destroy(mhd_batch *batch);

/* cell_offsets[0..npatch]: first cell of each patch in schedule-independent patch order, and the total. */
mhd_status mhd_batch_offsets(const mhd_batch *batch, long long *cell_offsets);

/* One step of every patch in place (see above). Asynchronous; the first call for a state, scheme,
 * eta and cfl captures the graph. The return code covers the enqueue only: check
 * mhd_batch_last_dt (or mhd_batch_stats) after each step. If a grid barrier of a step gives up
 * waiting, that step leaves the state unchanged, and so does every later step until one of those
 * two calls reports MHD_ERR_TIMEOUT (which re-arms the batch). */
mhd_status mhd_batch_step(mhd_batch *batch, const mhd_batch_state *state, double cfl, int scheme, double eta);

/* dt of the last step (synchronous); MHD_ERR_TIMEOUT if a grid barrier gave up waiting in any
 * step since the last report (those steps left the state unchanged; the report clears the
 * condition), MHD_ERR_NONFINITE if the signal speed was not finite (then no step was taken). */
mhd_status mhd_batch_last_dt(mhd_batch *batch, double *dt);

/* Flagged cells of the last step's two stages, summed over patches (synchronous); reports and
 * clears a barrier timeout as mhd_batch_last_dt does. */
mhd_status mhd_batch_stats(mhd_batch *batch, long long *fofc_cells_stage1, long long *fofc_cells_stage2);

/* Device time of the phases of the last step's two stages (synchronous), as measured by block 0
 * of the persistent launches with the GPU global timer at each launch start and grid barrier:
 * ms[6 * stage + j] for j = 0 cons->prim, 1 face sweeps (reconstruction + Riemann), 2 a-face
 * quantities to edges, 3 c-face quantities to edges + LD04 EMFs, 4 increments, update and
 * validity flags, 5 first-order fluxes of flagged cells (0 when the phase did not run: no
 * flagged cell, or flux correction off). `ms` holds 12 doubles, written by this call. */
mhd_status mhd_batch_phase_ms(mhd_batch *batch, double *ms);

/* Schedule of the persistent stage launches: sweep segment length seg (points per thread), patch
 * order (0 as given, 1 largest first), CTAs per SM of the stage's first launch (0 = as many as
 * fit; with three launches per stage the others take as many as fit), and whether steps are
 * captured and replayed as a CUDA graph. */
mhd_status mhd_batch_set_schedule(mhd_batch *batch, int seg, int order, int blocks_per_sm, int use_graph);

/* Launches per RK stage: 1 (default) runs every phase of the stage in one persistent cooperative
 * launch at the face sweep's register budget; 3 runs the face phase, then the edge, update and
 * flag phases at half that budget (twice the warps per SM), then the first-order correction.
 * Same results bit for bit. MHD_ERR_ARG for any other value. Synchronises the batch's stream. */
mhd_status mhd_batch_set_launches(mhd_batch *batch, int launches_per_stage);

/* Autotuner: times one step for every candidate schedule (1 or 3 launches per stage; seg in
 * {16, 32, 64, 128}; both orders; 1 .. max CTAs per SM of the first launch) on a scratch copy of
 * `state` (left unchanged; the copy is allocated and freed here), keeps the fastest and returns
 * it (any output pointer may be NULL). The choice is remembered for the process, keyed by the
 * device, the scheme, whether eta is zero and the histogram of patch sizes: a later call with the
 * same key (on this batch or another) sets that schedule without timing anything. */
mhd_status mhd_batch_tune(mhd_batch *batch, const mhd_batch_state *state, double cfl, int scheme, double eta,
                          int *seg, int *order, int *blocks_per_sm, int *launches_per_stage);

/* Test hook for the bounded barrier: every grid barrier waits for extra_blocks blocks more than
 * were launched and gives up after spin_limit polls (~100 ns each), so the next step ends with
 * MHD_ERR_TIMEOUT from mhd_batch_last_dt; (0, 1 << 25) restores normal operation. */
mhd_status mhd_batch_test_barrier(mhd_batch *batch, int extra_blocks, long long spin_limit);

const char *mhd_batch_last_error(const mhd_batch *batch);

#ifdef __cplusplus
}
#endif
#endif /* MHD_GB300_H */
