/*
 * libgksl -- SU(N) unfolding of a GKSL master equation and RK4 propagation of the
 * Bloch vector on one GB300 (sm_103a).  C ABI: plain pointers and sizes only.
 *
 * The method (arXiv:1812.11626):
 *   Eq. 1   d rho/dt = -i[H(t), rho] + sum_p gamma_p (L_p rho L_p^+ - 1/2 {L_p^+ L_p, rho})
 *   Eq. 6   rho = 1/N + sum_j v_j F_j over the N^2-1 traceless generators F_j of the
 *           Sec. II list (S^(j,k), J^(j,k), D^l)
 *   Eq. 8   dv/dt = (Q(t) + R) v + K, a real system of D = N^2-1 equations, with
 *           Q from Eq. 7, R from Eq. 10 and K from Eq. 11
 *   Sec. IV step 3.1: classical RK4 integration of Eq. 8.
 * The Hamiltonian is H(t) = sum_k theta_k H0_k + eps(t) H1 with
 * eps(t) = E + A sin(omega t), so Q(t) = Q0 + eps(t) Q1 with Q0 = sum_k theta_k Q(H0_k)
 * + sum_p gamma_p R_p, and K = sum_p gamma_p K_p.
 *
 * Conventions shared by every call:
 *  - Generator order: index s in [0, P2) is S^(j,k), j<k lexicographic, P2 = N(N-1)/2;
 *    [P2, 2 P2) is J^(j,k) in the same order; [2 P2, D) is D^l, l = 1..N-1.  D^l is
 *    real: (sum_{k<l} |k><k| - l |l><l|)/sqrt(l(l+1)) (the paper's list prints a
 *    spurious factor i).  All indices are 0-based.
 *  - N x N operator inputs are CSR with int32 row pointers (N+1) and column indices,
 *    and separate float64 real and imaginary arrays; rows need not be sorted but an
 *    (row, column) pair may appear only once.  Inputs are copied: the caller keeps
 *    ownership and may free them when the call returns.
 *  - Any pointer argument may point to host memory or to device memory of the
 *    context's GPU; the library decides with cudaPointerGetAttributes.  Outputs are
 *    written into caller-owned buffers of the stated size.
 *  - Every call returns a gksl_status and never aborts; the message of the last
 *    failure is kept per context (gksl_last_error).  A call made before the state it
 *    needs exists (e.g. propagate before assemble) returns GKSL_ERR_STATE.
 *  - All device work runs on the stream given to gksl_create, in stream order; calls
 *    that return data to host memory synchronise that stream first.
 *  - The library owns all device memory it allocates for a context and frees it in
 *    gksl_destroy.
 */
#ifndef GKSL_H
#define GKSL_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GKSL_OK = 0,
    GKSL_ERR_ARG = 1,       /* invalid argument: null pointer, size out of range, malformed CSR */
    GKSL_ERR_CUDA = 2,      /* a CUDA runtime call failed (message in gksl_last_error) */
    GKSL_ERR_OOM = 3,       /* a device allocation failed */
    GKSL_ERR_STATE = 4,     /* call out of order */
    GKSL_ERR_UNSTABLE = 5,  /* step size above the RK4 stability bound (checked runs only) */
    GKSL_ERR_DIVERGED = 6,  /* the propagated state became non-finite */
    GKSL_ERR_TIMEOUT = 7    /* a bounded device-side wait gave up */
} gksl_status;

typedef struct gksl_ctx gksl_ctx;
typedef struct gksl_batch gksl_batch;

#define GKSL_MAX_H0 8   /* Hamiltonian components H0_k, k < GKSL_MAX_H0 */
#define GKSL_MAX_P 8    /* dissipative channels p < GKSL_MAX_P */

/* ------------------------------------------------------------------ lifetime */

/* Create a context for N x N operators (2 <= N <= 4096) on CUDA device `device`;
 * `cuda_stream` is a cudaStream_t (NULL: the legacy default stream). */
gksl_status gksl_create(int N, int device, void *cuda_stream, gksl_ctx **out);
/* Free every device buffer of the context.  NULL is allowed. */
void gksl_destroy(gksl_ctx *ctx);
/* Message of the last failed call on this context ("" if none); valid until the next call. */
const char *gksl_last_error(const gksl_ctx *ctx);

/* ------------------------------------------------------------------ inputs (Eq. 1) */

/* Hamiltonian component H0_k with weight theta_k (Eq. 1; H(t) = sum_k theta_k H0_k + eps(t) H1).
 * Must be Hermitian; the trace part is irrelevant (Sec. II assumes H traceless).
 * Passing nnz = 0 removes the component. */
gksl_status gksl_set_h0_component(gksl_ctx *ctx, int k, double theta_k, const int *rowptr, const int *col,
                                  const double *re, const double *im, int nnz);
/* Change theta_k of an existing component without re-expanding it. */
gksl_status gksl_set_theta(gksl_ctx *ctx, int k, double theta_k);
/* Driven part H1 (Hermitian), multiplied by eps(t). */
gksl_status gksl_set_h1(gksl_ctx *ctx, const int *rowptr, const int *col, const double *re, const double *im,
                        int nnz);
/* Dissipator L_p with rate gamma_p >= 0 (Eq. 1).  Any complex matrix; a nonzero trace part
 * Tr(L_p)/N is folded into an effective Hamiltonian.  nnz = 0 removes the channel. */
gksl_status gksl_set_dissipator(gksl_ctx *ctx, int p, double gamma_p, const int *rowptr, const int *col,
                                const double *re, const double *im, int nnz);
/* Dissipator given as a Kossakowski matrix A over the generators (Eq. 8): D x D row-major real and
 * imaginary parts (a_im may be NULL), Hermitian and positive semidefinite; replaces every
 * previously set channel.  A is first factorised as sum_p c_p c_p^+ (pivoted Cholesky, pivots
 * <= tol * max diag(A) end it): when at most GKSL_MAX_P pivots exhaust it and N <= 64, channel p
 * is set to L_p = sum_j c_pj F_j / |c_p| with gamma_p = |c_p|^2 (GKSL_ERR_ARG if A is not
 * positive semidefinite).  Otherwise (higher rank, or N > 64) A itself is kept on the device and
 * channel 0 holds the whole Eq. 8 dissipator at gamma_0 = 1, assembled by the dense route
 * (N <= 128; A, its kernel M and the transient take about 16 (D^2 + 2 N^4) bytes); positive
 * semidefiniteness is then checked through the diagonal and the 2 x 2 principal minors only
 * (a_jj >= 0, |a_jk|^2 <= a_jj a_kk).  GKSL_ERR_ARG if A is not Hermitian or fails those checks.
 * a_re and a_im may be host or device memory; above N = 64 A is copied to the device first and
 * checked there (the same conditions), and a rejected A leaves the previous channels in place.
 * GKSL_ERR_OOM if the device cannot hold A (plus a planar copy of host input) during the call. */
gksl_status gksl_set_kossakowski(gksl_ctx *ctx, const double *a_re, const double *a_im, double tol);
/* Change gamma_p of an existing channel without re-expanding it. */
gksl_status gksl_set_gamma(gksl_ctx *ctx, int p, double gamma_p);
/* eps(t) = E + A sin(omega t), omega > 0; the period is T = 2 pi / omega (Sec. III). */
gksl_status gksl_set_drive(gksl_ctx *ctx, double E, double A, double omega);

#define GKSL_DRIVE_SIN 0     /* theta(t) = sin(omega t) (default) */
#define GKSL_DRIVE_SQUARE 1  /* theta(t) = +1 on [0, T/2), -1 on [T/2, T), periodic (Sec. III, driving (i)) */
/* Shape of theta in eps(t) = E + A theta(t).  With the square shape every RK4 step uses theta at
 * its midpoint for all four stages (the drive is constant on each step of a grid that contains
 * the jumps), so propagation requires an even steps_per_period and a start time on the step grid
 * (GKSL_ERR_ARG otherwise).  Batches take the shape of their group contexts. */
gksl_status gksl_set_drive_shape(gksl_ctx *ctx, int shape);

/* ------------------------------------------------------------------ expansion (Sec. IV step 2.1) */

/* Coefficients x_s = Tr(F_s X), s < D, of an N x N CSR matrix X (host or device arrays).
 * coef_re/coef_im: D doubles each (coef_im may be NULL). */
gksl_status gksl_expand(gksl_ctx *ctx, const int *rowptr, const int *col, const double *re, const double *im,
                        int nnz, double *coef_re, double *coef_im);

/* ------------------------------------------------------------------ structure constants (Eq. 5) */

#define GKSL_STRUCT_F 0   /* f_mns = -i Tr(F_s [F_m, F_n]) */
#define GKSL_STRUCT_D 1   /* d_mns = Tr(F_s {F_m, F_n}) */

/* Number of nonzero ordered triples (m, n, s) of f or d for dimension N, counted on the device
 * by enumerating the closed-form nonzero set (Sec. IV step 2.2 gives 5N^3-9N^2-2N+6 and
 * 6N^3-N(21N+7)/2+1).  Uses the current device; allocates a few bytes. */
gksl_status gksl_structure_count(int N, int which, long long *count);
/* Every nonzero (m, n, s, value) of f or d, written to caller buffers of `capacity` entries
 * (host or device).  *count receives the total; if it exceeds capacity nothing is written and
 * GKSL_ERR_ARG is returned. */
gksl_status gksl_structure_enumerate(int N, int which, long long capacity, int *m, int *n, int *s,
                                     double *value, long long *count);

/* ------------------------------------------------------------------ assembly (Sec. IV steps 2.1-2.5) */

#define GKSL_ASM_FP32 1u        /* also build the FP32 copies used by precision 32 */
#define GKSL_ASM_TRANSPOSE 2u   /* also build the transposes used by the adjoint */
#define GKSL_ASM_NO_DROP 4u     /* keep entries |q| <= 64 eps max|Q| in Q0 */
/* Keep Q1 as a separate stream of the RK4 stages.  By default, when every row of Q1 has at most
 * one entry and that entry's column is among the row's entries of Q0 + E Q1 (a pair rotation,
 * as for any diagonal H1), Q1 is folded into that slot: the stage forms q0 + (eps(t) - E) q1
 * there and reads no Q1 column indices.  Both forms compute the same map; they differ by
 * rounding only. */
#define GKSL_ASM_NO_FOLD 16u
/* Build no 16-bit copy of the RK4 stage columns.  By default, when Q1 is folded, a copy holds
 * each stored entry's column as a 16-bit offset from its row or from the row's S/J partner (the
 * generator of the same pair (j, k) in the other half of the basis); rows with a column beyond
 * +-16383 of both get threads of their own that read the 32-bit columns, and the long rows keep
 * their warps.  The copy is dropped when more than one short row in eight would escape.  The
 * first propagation in each precision times the stage kernels with either column width and keeps
 * the 16-bit columns only when they are at least 2 % faster (gksl_info.rk4_compact; the
 * environment variable GKSL_RK4_COLUMNS=32 skips them).  Both compute the same map with the same
 * arithmetic (bit-identical results). */
#define GKSL_ASM_WIDE_COLUMNS 32u
/* Form every dissipator channel by the dense route: R_p = Re Tr(F_s D_p(F_m)) entry by entry from
 * the matrix-unit form of L_p rho L_p^+ - 1/2 {L_p^+ L_p, rho} (trace part of L_p included), in
 * O(N^4) work with at most 1 GB of transient memory, N <= 200.  Without the flag a
 * channel takes this route by itself when the sparse route's F''^T Z'' product would have more
 * than 2 D^2 terms (a dense L at N = 100 has 5.5e9) and N <= 200, otherwise the sparse route
 * (Sec. IV step 2.5).  Both give the same matrix up to rounding; the dense route stores R_p
 * without its exact zeros. */
#define GKSL_ASM_DENSE_DISSIPATORS 64u
/* Matrix-free form: build no CSR matrix; keep H0 (+ E H1), H1, Gamma = 1/2 sum_p gamma_p L_p^+ L_p
 * and sqrt(gamma_p) L_p as complex diagonals (O(N) data) and let gksl_propagate apply Q(t) v + K on
 * the fly, as Tr(F_s L_t(rho)) with rho = 1/N + sum v F (Eq. 1, 6, 8), from tiles of rho rebuilt
 * from v in shared memory.  Every operator must be banded with half-bandwidth <= 4 (else
 * GKSL_ERR_ARG).  Excludes GKSL_ASM_TRANSPOSE; gksl_get_csr, gksl_get_k*, the adjoint and the
 * batched form need a CSR assembly and return GKSL_ERR_STATE. */
#define GKSL_ASM_MATRIX_FREE 8u

/* Build Q(H0_k), Q(H1), R_p, K_p on the device from the structure constants (Eq. 7, 10, 11),
 * then Q0, Q1 and K.  `seconds` (may be NULL) receives the wall time of the call. */
gksl_status gksl_assemble(gksl_ctx *ctx, unsigned flags, double *seconds);

#define GKSL_MAT_Q0 0      /* sum_k theta_k Q(H0_k) + sum_p gamma_p R_p (no eps term) */
#define GKSL_MAT_Q1 1      /* Q(H1) */
#define GKSL_MAT_H0 16     /* + k: Q(H0_k) alone (Eq. 7) */
#define GKSL_MAT_R 32      /* + p: R_p at unit rate (Eq. 10), including the trace-part Hamiltonian */

/* Copy one assembled D x D matrix as CSR (rows sorted by column) into caller buffers:
 * rowptr (D+1 int32), col (nnz int32), val (nnz float64).  With rowptr == NULL only *nnz is set. */
gksl_status gksl_get_csr(gksl_ctx *ctx, int which, long long *nnz, int *rowptr, int *col, double *val);
/* K = sum_p gamma_p K_p (Eq. 11), D doubles. */
gksl_status gksl_get_k(gksl_ctx *ctx, double *K);
/* K_p at unit rate, D doubles. */
gksl_status gksl_get_k_channel(gksl_ctx *ctx, int p, double *K);

/* ------------------------------------------------------------------ state (Eq. 6) */

/* v(0) = Tr(F_j rho0) from a dense N x N rho0 (row-major re and im, im may be NULL); t = 0
 * (Sec. IV step 2.6). */
gksl_status gksl_set_rho0(gksl_ctx *ctx, const double *re, const double *im);
gksl_status gksl_set_state(gksl_ctx *ctx, const double *v, double t);
gksl_status gksl_get_state(gksl_ctx *ctx, double *v, double *t);

/* ------------------------------------------------------------------ propagation (Sec. IV step 3.1) */

/* Smallest steps per period for which h * (Gershgorin bound of ||Q(t)||) <= 2.6 for all t
 * (RK4 is stable on the imaginary axis up to 2 sqrt 2).  Needs gksl_assemble. */
gksl_status gksl_min_stable_steps(gksl_ctx *ctx, long long *steps_per_period);

/* Advance the state by n_steps classical RK4 steps of h = T / steps_per_period from the
 * current (v, t).  precision 64: FP64 throughout.  precision 32: FP32 matrix, stage vectors
 * and arithmetic, FP64 master state (the FP32 increment is added to it every step) and,
 * every `correction_every` steps (<= 0: never), one full FP64 step in place of an FP32 one.
 * Every `emit_every` steps (<= 0: never) the FP64 state is copied to v_out, which holds
 * (n_steps / emit_every) rows of D doubles.  Returns GKSL_ERR_DIVERGED if the state is
 * non-finite at an emission point or at the end.  Small systems (up to D + 1 = 256 rows in FP64,
 * 576 in FP32) run each stretch of steps between emissions in one thread block with the state in
 * shared memory, with the same results bit for bit as the per-stage kernels; the environment
 * variable GKSL_RK4_BLOCK=0 turns that off, =1 uses it wherever D + 1 <= 4096. */
gksl_status gksl_propagate(gksl_ctx *ctx, long long steps_per_period, long long n_steps, int precision,
                           long long correction_every, long long emit_every, double *v_out);

/* ------------------------------------------------------------------ observables (Eq. 6) */

/* <O> = Tr(O)/N + sum_j v_j Tr(O F_j) for a diagonal O (o_diag: N doubles) and `count` state
 * vectors stored back to back in v (count x D doubles); out: count doubles. */
gksl_status gksl_observable_diag(gksl_ctx *ctx, const double *o_diag, const double *v, long long count,
                                 double *out);
/* Dense rho = 1/N + sum_j v_j F_j (Eq. 6), row-major N x N re and im. */
gksl_status gksl_rho(gksl_ctx *ctx, const double *v, double *re, double *im);

/* ------------------------------------------------------------------ adjoint */

/* Loss = trapezoid mean of <O> over the steps_per_period+1 grid points of period
 * `period_index` (1-based) of an RK4 run from the current state, and its exact gradient by
 * the discrete adjoint of the RK4 map (per-period checkpoints, recomputation in between).
 * grad receives n_grad doubles in the order [d/dA, d/dgamma_0 .. d/dgamma_{P-1},
 * d/dtheta_0 .. d/dtheta_{K-1}] over the set channels and components in index order.
 * Requires gksl_assemble with GKSL_ASM_TRANSPOSE.  The state is left unchanged.  For small
 * systems (at most 4 parameter channels, 64-thread reverse blocks) the FP64 reverse stages load
 * the channels' first slots together; the environment variable GKSL_ADJ_PIPE=0 or 1 turns that
 * off or on in either precision (the results are the same bit for bit).  With at most 4 channels
 * whose ELL slots total at most 32, the FP32 reverse stages load all of a row's slots at once
 * and sum each channel in float (as the FP32 forward stage does; the FP64 stages sum in double);
 * GKSL_ADJ_WIDE=0 or 1 turns that form off, or on in both precisions (in FP64 it gives the same
 * results bit for bit as the channel-by-channel form). */
gksl_status gksl_adjoint_timeavg(gksl_ctx *ctx, const double *o_diag, long long steps_per_period,
                                 long long period_index, int precision, double *loss, double *grad, int n_grad);

/* ------------------------------------------------------------------ batched instances */

/* A batch of instances that share the unfolded components of an assembled context per
 * group and differ in the drive amplitude A_b and a dissipation scale g_b:
 *   dv_b/dt = (Q0_H + eps_b(t) Q1 + g_b R) v_b + g_b K,  eps_b(t) = E + A_b sin(omega t),
 * where Q0_H = sum_k theta_k Q(H0_k) and R, K are the context's gamma-weighted dissipator
 * terms.  groups[i] must stay alive while the batch exists.  A and g hold one value per
 * instance, group by group (n_inst[0] values of group 0 first). */
gksl_status gksl_batch_create(int n_groups, gksl_ctx *const *groups, const int *n_inst, const double *A,
                              const double *g, gksl_batch **out);
void gksl_batch_destroy(gksl_batch *b);
/* Message of the last failed call on this batch; with b == NULL, of the calling thread's last
 * failed gksl_batch_create. */
const char *gksl_batch_last_error(const gksl_batch *b);
/* Give every instance its own weight theta_b of Hamiltonian component `component` (a parameter
 * scan, e.g. the interaction U of a bifurcation diagram): instance b then uses theta_b in place of
 * its group context's theta_k.  theta_b holds one value per instance in the batch's order (host or
 * device).  Adds a fourth value channel Q(H0_k) to every group; the tile autotuning is redone. */
gksl_status gksl_batch_set_scan(gksl_batch *b, int component, const double *theta_b);
/* Reset every instance to its group's current state vector, t = 0. */
gksl_status gksl_batch_reset(gksl_batch *b);
/* Advance group i by n_steps[i] RK4 steps of h = T / steps_per_period[i] from the batch's current
 * time (FP32 bulk, FP64 master state, an FP64 step every correction_every steps, <= 0: never);
 * groups with fewer steps stop early.  `seconds` (may be NULL) receives the device time of the
 * whole run. */
gksl_status gksl_batch_propagate(gksl_batch *b, const long long *steps_per_period, const long long *n_steps,
                                 long long correction_every, double *seconds);
/* Long-time (Floquet) asymptotic state of every instance (Sec. I: the asymptotic state is
 * T-periodic; Sec. V: populations read at phase 0 after a transient of 10 T).  Propagates
 * `transient` whole periods, then period by period until every instance's period-map residual
 *     r_b = max_s |v_b(kT) - v_b((k-1)T)|
 * is <= tol, or max_periods periods after the transient.  Group g advances steps_per_period[g]
 * steps per period with the arithmetic of gksl_batch_propagate (FP32 bulk, one FP64 step every
 * correction_every steps; 1: FP64 throughout).  residual (n_instances doubles, batch instance
 * order, host memory) receives each instance's last r_b (+inf where the state went non-finite);
 * periods (may be NULL) the total periods run, transient included.  Returns GKSL_OK whether or
 * not tol was met; the states are left at the last period end. */
gksl_status gksl_batch_asymptotic(gksl_batch *b, const long long *steps_per_period, long long transient,
                                  long long max_periods, double tol, long long correction_every, double *residual,
                                  long long *periods);
/* State of instance i (D_i doubles, FP64 master). */
gksl_status gksl_batch_get_state(gksl_batch *b, int instance, double *v);
/* Tile width chosen by the autotuner for group `group` (instances per lane; one warp covers
 * 32 * instances_per_lane instances of a row; 4 also for the path with one 16-byte gather of 4
 * instances per lane and entry) and its timed
 * cost per FP32 step in microseconds.  Both are 0 before the first gksl_batch_propagate.  The
 * autotuner also times each width on pair units (see gksl_batch_group_stats).  The environment
 * variable GKSL_BATCH_TILE=0 forces the 16-byte-gather path, 1..4 the scalar path on rows with
 * that many instances per lane, p1..p4 the same on pair units (no timing; the cost is then
 * reported as 0). */
gksl_status gksl_batch_info(gksl_batch *b, int group, int *instances_per_lane, double *tuned_us_per_step);
/* Size and path of group `group`: rows D, instances, the stored entries of its value channels
 * summed (QH, Q1, [R | K] and a scanned component), which the row paths stream once per stage and
 * instance chunk, the entries of its pair units (rows S^(j,k) and J^(j,k) of one pair share one
 * merged column list; the D rows stand alone), which the pair path streams instead, and the FP32
 * path in use: 0 the 16-byte gathers on rows, 1 scalar gathers on rows, 2 scalar gathers on pair
 * units.  Any pointer may be NULL. */
gksl_status gksl_batch_group_stats(gksl_batch *b, int group, long long *rows, int *instances,
                                   long long *channel_entries, long long *pair_entries, int *path);

/* ------------------------------------------------------------------ allocation-free propagation */

/* Largest D accepted by gksl_propagate_csr_noalloc (N <= 512). */
#define GKSL_NOALLOC_MAX_D 262144

/* The paper has no counterpart to this call; it exists for callers that cannot let a library
 * allocate device memory (a service whose memory pool owns the whole GPU, or a loop that must
 * not stall the device the way cudaMalloc/cudaFree can).
 * Advances v by n_steps classical RK4 steps of dv/dt = (A0 + eps(t) A1) v + K from time t0 with
 * step h, eps(t) = E + A sin(omega t), stage times t_n, t_n + h/2 (twice), t_n + h -- the same
 * map as gksl_propagate.  A0 and A1 are D x D CSR matrices (int32 rowptr of D+1, int32 col,
 * float64 val) in DEVICE memory; A1 may be NULL (all three a1 pointers), K may be NULL; v (D
 * float64, device) is updated in place.  Everything is caller-owned and nothing is copied or
 * allocated: the RK4 work vectors live in a fixed array compiled into the library (3 x
 * GKSL_NOALLOC_MAX_D float64 per GPU, held until the process exits).  The first call on each
 * device looks the array's address up (cudaGetSymbolAddress) with that device current and keeps
 * it for the life of the process, so make the first call before any stream capture, and do not
 * call this again on a device after cudaDeviceReset.  Calls whose work overlaps on the GPU share
 * the array and race.  The kernels index the arrays without checks: rowptr must run from 0 to at
 * most the length of col/val, columns must lie in [0, D), and every array must be on the current
 * device.  Returns GKSL_ERR_ARG for D > GKSL_NOALLOC_MAX_D, a null pointer, h <= 0 or
 * n_steps < 0; GKSL_ERR_CUDA when a CUDA error is already pending at entry (nothing is launched
 * and that error is left for its owner) or a launch fails.  Work is enqueued on cuda_stream
 * (NULL: legacy default stream) and the call does not synchronise. */
gksl_status gksl_propagate_csr_noalloc(long long D, const int *a0_rowptr, const int *a0_col, const double *a0_val,
                                       const int *a1_rowptr, const int *a1_col, const double *a1_val,
                                       const double *K, double *v, double t0, double h, long long n_steps, double E,
                                       double A, double omega, void *cuda_stream);

/* ------------------------------------------------------------------ measured rates */

/* The paper has no counterpart to this call; it measures two rates of GPU `device` that bound
 * this library's kernels and for which no vendor figure applies as measured: the FP64 fused
 * multiply-add rate (FMA per second, each counted once) of a grid of independent FMA chains, and
 * the rate of reading an L2-resident 32 MiB buffer (bytes per second).  Either pointer may be
 * NULL (not measured).  Each probe checks its own result (the FMA chains against the same
 * recurrence on the host, the L2 sum against its exact value) and returns GKSL_ERR_STATE if it
 * fails; GKSL_ERR_CUDA on a CUDA error.  Takes about 0.2 s; restores the calling thread's device. */
gksl_status gksl_measure_rates(int device, double *fp64_fma_per_s, double *l2_read_bytes_per_s);

/* ------------------------------------------------------------------ introspection */

typedef struct {
    int N;
    long long D;
    long long nnz_q0;          /* propagation matrix Q0 + E Q1 after the drop */
    long long nnz_q1;
    long long nnz_r[GKSL_MAX_P];
    int ell_width_q0;          /* ELL slots per row of the propagation format */
    int ell_width_q1;
    long long long_rows;       /* rows handled warp-per-row */
    long long device_bytes;    /* device memory held by the context */
    double assemble_seconds;
    double max_abs_q0;
    int rk4_variant[2];           /* stage-kernel variant in use, [0]: FP64, [1]: FP32 (chosen by timing) */
    double rk4_variant_us[2][4];  /* timed cost per RK4 step of each variant, microseconds (0: not timed) */
    int q1_folded;                /* 1: Q1 folded into the propagation format (see GKSL_ASM_NO_FOLD) */
    int compact_columns[2];       /* 1: 16-bit stage columns built (GKSL_ASM_WIDE_COLUMNS), [0]: FP64, [1]: FP32 */
    long long compact_escaped_rows; /* short rows that read 32-bit columns in the 16-bit form */
    long long tail_nnz;           /* stored entries of the long rows (read warp-per-row) */
    int rk4_compact[2];           /* 1: the variant in use reads the 16-bit columns (chosen by timing with it) */
    double rk4_variant_us_c16[2][4]; /* as rk4_variant_us, with 16-bit columns (0: not timed) */
} gksl_info;

gksl_status gksl_get_info(gksl_ctx *ctx, gksl_info *out);

#ifdef __cplusplus
}
#endif
#endif /* GKSL_H */
