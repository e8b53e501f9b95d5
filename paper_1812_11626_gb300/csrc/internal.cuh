// Cross-file entry points of the library (inside namespace gk).
#pragma once

#include "common.cuh"

namespace gk {

// ---- expand.cu (Sec. IV steps 2.1 and 2.6, Eq. 6)
// Dense coefficient vector Tr(F_s X), s < D, of an input operator (complex, D entries).
void expand_op(gksl_ctx *c, const Op &op, DBuf<double2> &coef);
// v = Re Tr(F_s rho) of a dense device matrix (re, im may be null), written to v_dev (D entries).
void expand_dense(gksl_ctx *c, const double *re_dev, const double *im_dev, double *v_dev);
// <O> for count vectors (device) -> out_dev
void observable_diag(gksl_ctx *c, const double *o_diag_dev, const double *v_dev, long long count, long long ldv,
                     double *out_dev);
void rho_dense(gksl_ctx *c, const double *v_dev, double *re_dev, double *im_dev);
// observable weights w_l = Tr(O D^l) into a dense length-D vector (zeros off the D block) and c0
void observable_weights(gksl_ctx *c, const double *o_diag_dev, double *w_dev, double *c0_dev);
// <O> = c0 + w.v for count vectors with weights from observable_weights (no synchronisation)
void observable_apply(gksl_ctx *c, const double *w, const double *c0, const double *v, long long count, long long ldv,
                      double *out);

// ---- assemble.cu (Sec. IV steps 2.2-2.5)
void assemble(gksl_ctx *c, unsigned flags);

// ---- rk4.cu (Sec. IV step 3.1)
void propagate(gksl_ctx *c, long long spp, long long n_steps, int precision, long long corr_every,
               long long emit_every, double *v_out, bool out_on_device);
void ensure_work(gksl_ctx *c, bool fp32);
void clear_graphs(gksl_ctx *c);
bool state_finite(gksl_ctx *c);
// small systems (CSR form; by default up to D + 1 = 256 rows in FP64, 576 in FP32): a chunk of
// RK4 steps by one thread block with the state in shared memory (rk4_block.cu);
// GKSL_RK4_BLOCK=0/1 forces it off/on (on: wherever D + 1 <= 4096)
bool rk4_block_applies(const gksl_ctx *c, int precision);
void rk4_block_run(gksl_ctx *c, int precision, double h, const double *tab, long long first, long long count);
// drive table eps(t) - E for steps [0, n) of a run starting at t0
void fill_eps_table(gksl_ctx *c, double t0, double h, long long n);
// time the stage-kernel variants on this context once per precision (as the first gksl_propagate
// does) with the drive table filled from the current time for at least 8 steps
void tune_stage_variant(gksl_ctx *c, int precision, double h);
// the square drive's jumps must fall on the step grid (even steps/period, time on the grid)
void check_drive_grid(const gksl_ctx *c, long long spp, double h);
// `count` RK4 steps on the context state starting at global step `first` (drive table index)
void advance(gksl_ctx *c, int precision, double h, long long first, long long count);
// one CSR-form RK4 step on the context state at step *step_base + local, writing its stage inputs
// Y2, Y3, Y4 (FP64: double*, FP32: float*; each D + 1 long with 1 at index D) instead of the
// context's work vectors
void step_into(gksl_ctx *c, int precision, double h, long long local, void *Y2, void *Y3, void *Y4);
// device-side step counter base read by the stage kernels (and graphs of them)
void set_step_base(gksl_ctx *c, long long g);
// theta(t) (the drive shape without its amplitude) at the three stage times of steps [0, n)
void fill_theta_table(gksl_ctx *c, double t0, double h, long long n, double *tab);
void to_f32(const double *v, float *o, long long n, cudaStream_t s);

// ---- mfree.cu (matrix-free stages, GKSL_ASM_MATRIX_FREE)
void mf_build(gksl_ctx *c, bool fp32);
// diagonal image of the state's D coefficients before a run of steps, and back after it
void mf_prep(gksl_ctx *c, int precision);
void mf_post(gksl_ctx *c, int precision);
// the four stages of one RK4 step
void mf_step(gksl_ctx *c, int precision, double h, const double *tab, long long local);

// ---- dense_diss.cu (dissipators through their matrix-unit form, O(N^4); Eq. 8)
constexpr int kDenseDissMaxN = 200;   // dense R: D^2 < 2^31 entries
constexpr int kDenseKmMaxN = 128;     // Kossakowski kernel M: N^4 complex (4.3 GB at N = 128)
// device memory of `device` (or managed memory), which this library's kernels on it may read in
// place; host memory and other GPUs' memory is copied in first
bool device_local_ptr(const void *p, int device);
// Copy a D x D Kossakowski matrix (planar re / im, host or device; im may be null) into A
// (interleaved, device) and check on the device that it is finite, Hermitian to 1e-12 max|a| and
// passes the diagonal and 2 x 2 minor conditions of positive semidefiniteness; GKSL_ERR_ARG
// otherwise.  Returns its trace (summed on the host in index order).
double kossakowski_upload_checked(gksl_ctx *c, const double *a_re, const double *a_im, DBuf<double2> &A);
// R (unit rate, CSR without exact zeros) and K of one jump operator, any N x N matrix
void dense_dissipator_channel(gksl_ctx *c, const Op &op, CsrR &R, DBuf<double> &K);
// R and K of the Eq. 8 dissipator of a D x D Kossakowski matrix (device, row-major)
void dense_dissipator_kossakowski(gksl_ctx *c, const double2 *A, CsrR &R, DBuf<double> &K);

// ---- adjoint.cu
void adjoint_timeavg(gksl_ctx *c, const double *o_diag_dev, long long spp, long long period, int precision,
                     double *loss, double *grad, int n_grad);

// ---- structure.cu (Eq. 5 closed forms)
long long structure_count(int N, int which, cudaStream_t s);
long long structure_enumerate(int N, int which, long long cap, int *m, int *n, int *sidx, double *val,
                              cudaStream_t s);

// ---- hyb.cu: CSR -> hybrid ELL/warp-row format
void build_hyb_pair(const CsrR &a0, const CsrR &a1, long long rows, Hyb<double> &h0, Hyb<double> &h1,
                    Hyb<float> *h0f, Hyb<float> *h1f, cudaStream_t s);
void build_hyb_single(const CsrR &a, long long rows, Hyb<double> &h, Hyb<float> *hf, double scale, cudaStream_t s);
// Fold Q1 into slot 0 of the propagation ELL of q0e = [Q0 + E Q1 | K] when every short row has
// at most one Q1 entry and its column is among the row's entries; returns whether it did
bool fold_q1(const CsrR &q0e, const CsrR &q1, long long rows, Hyb<double> &h0, Hyb<float> *h0f, DBuf<double> &q1v,
             DBuf<float> &q1vf, cudaStream_t s);
// 16-bit relative copy of h's ELL columns (Hyb::ell_c16) for the S/J/D basis with `pairs` =
// N(N-1)/2 pairs; kept when at most one short row in eight falls back to 32-bit columns
template <typename VT>
bool build_c16(Hyb<VT> &h, long long pairs, cudaStream_t s);
template <typename VT>
void drop_c16(Hyb<VT> &h);   // release the 16-bit copy and its escape list
// several matrices applied together (one long-row set; entries scaled by `scales`)
void build_hyb_multi(const std::vector<const CsrR *> &ms, const std::vector<double> &scales, long long rows,
                     const std::vector<Hyb<double> *> &out, const std::vector<Hyb<float> *> &outf, cudaStream_t s);

// CSR helpers (assemble.cu)
// sum_i w_i M_i (+ Kcol as column D when given) -> CSR without exact zeros, on the context's stream
void merge_terms(gksl_ctx *c, const std::vector<std::pair<const CsrR *, double>> &terms, const double *Kcol,
                 CsrR &out);
void csr_transpose(const CsrR &a, CsrR &t, cudaStream_t s);
void csr_copy_out(gksl_ctx *c, const CsrR &m, long long *nnz, int *rowptr, int *col, double *val);

}  // namespace gk
