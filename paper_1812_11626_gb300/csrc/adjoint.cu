// Gradient of a time-averaged observable by the discrete adjoint of the RK4 map.
//
// Loss: the trapezoid mean of <O> = c0 + w.v over the S+1 grid points of period p (1-based)
// of an RK4 run of S steps per period from the current state.  For one step with
// Y1 = v, Y2 = v + h/2 k1, Y3 = v + h/2 k2, Y4 = v + h k3, k_i = A_i Y_i + b, the reverse
// sweep for the adjoint lam' of the step's output is
//   kb4 = h/6 lam';            Yb4 = A4^T kb4;   kb3 = h/3 lam' + h   Yb4
//   Yb3 = A3^T kb3;            kb2 = h/3 lam' + h/2 Yb3
//   Yb2 = A2^T kb2;            kb1 = h/6 lam' + h/2 Yb2
//   Yb1 = A1^T kb1;            lam = lam' + Yb1 + Yb2 + Yb3 + Yb4
// and every parameter theta gains sum_i kb_i . (dA_i/dtheta Y_i + db/dtheta).  A^T is applied
// as a sum of per-parameter channels C_c = (dA/dtheta_c)^T: Q(H0_k)^T = -Q(H0_k), Q1^T = -Q1,
// R_p^T, so one pass over the channels gives both A^T kb (weighted sum) and the parameter
// products u_c . Y_i.  Each stage is one fused kernel; gradient partial sums are kept per
// block in fixed slots and reduced in a fixed order at the end (deterministic).
//
// Memory: period checkpoints, then per period sqrt(S)-spaced checkpoints, then the states of
// one segment; each state is recomputed at most twice.
#include <cmath>
#include <vector>

#include "internal.cuh"
#include "prim.cuh"

namespace gk {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxCh = gksl_ctx::kMaxCh;
constexpr int kMaxPar = kMaxCh;

template <typename VT>
struct AdjArgs {
    HybView<VT> ch[kMaxCh];
    double chw[kMaxCh];     // weight of channel c in A^T
    int gidx[kMaxCh];       // gradient slot of channel c
    double gfac[kMaxCh];    // factor of u_c . Y in that slot (sin(omega t) for the drive amplitude)
    int nch;
    const double *kp[GKSL_MAX_P];   // K_p per unit rate: d b / d gamma_p
    int kp_gidx[GKSL_MAX_P];
    int nkp;
    int npar;
    double alpha;   // kb = alpha * x
    double h, h2, h3, h6;   // h, h/2, h/3, h/6 (computed on the host)
    double beta;    // stage 1: lam += beta * w
    const int *long_rows;
    long long n_long;
    int nb_long;
    long long D;
};

template <typename VT>
__device__ inline double ell_row(const HybView<VT> &H, long long r, const VT *__restrict__ x) {
    double s = 0.0;
    for (int j = 0; j < H.width; ++j) {
        long long p = (long long)j * H.ld + r;
        s += (double)__ldcs(H.ell_val + p) * (double)__ldg(x + __ldcs(H.ell_col + p));
    }
    return s;
}

template <typename VT>
__device__ inline double tail_row(const HybView<VT> &H, long long i, int lane, const VT *__restrict__ x) {
    double s = 0.0;
    for (int e = H.tail_ptr[i] + lane; e < H.tail_ptr[i + 1]; e += 32)
        s += (double)__ldcs(H.tail_val + e) * (double)__ldg(x + H.tail_col[e]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

template <int STAGE, typename VT>
__device__ inline void adj_epilogue(const AdjArgs<VT> &a, long long r, double ybar, const double *__restrict__ lam,
                                    double *__restrict__ lacc, VT *__restrict__ kb_out, const double *__restrict__ w,
                                    double *lam_out) {
    if (STAGE == 4) { kb_out[r] = (VT)(a.h3 * lam[r] + a.h * ybar); lacc[r] = lam[r] + ybar; }
    if (STAGE == 3) { kb_out[r] = (VT)(a.h3 * lam[r] + a.h2 * ybar); lacc[r] = lacc[r] + ybar; }
    if (STAGE == 2) { kb_out[r] = (VT)(a.h6 * lam[r] + a.h2 * ybar); lacc[r] = lacc[r] + ybar; }
    if (STAGE == 1) { lam_out[r] = lacc[r] + ybar + a.beta * w[r]; }
}

// x: gathered vector (lam' for stage 4, kb_i otherwise); Y: forward stage input Y_i (own row)
template <int STAGE, typename VT>
__global__ void __launch_bounds__(kThreads) k_adjoint(AdjArgs<VT> a, const VT *__restrict__ x,
                                                     const VT *__restrict__ Y, const double *lam, double *lacc,
                                                     VT *__restrict__ kb_out, const double *__restrict__ w,
                                                     double *lam_out, double *__restrict__ part) {
    double g[kMaxPar];
#pragma unroll
    for (int k = 0; k < kMaxPar; ++k) g[k] = 0.0;
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    bool active = false;
    long long r = -1;
    double u[kMaxCh];
    if ((int)blockIdx.x < a.nb_long) {
        long long i = (long long)blockIdx.x * kWarps + warp;
        if (i < a.n_long) {
            r = a.long_rows[i];
#pragma unroll
            for (int c = 0; c < kMaxCh; ++c)
                if (c < a.nch) u[c] = tail_row<VT>(a.ch[c], i, lane, x);
            active = lane == 0;
        }
    } else {
        r = (long long)(blockIdx.x - a.nb_long) * kThreads + threadIdx.x;
        if (r < a.D && __ldcs(a.ch[0].ell_col + r) >= 0) {
#pragma unroll
            for (int c = 0; c < kMaxCh; ++c)
                if (c < a.nch) u[c] = ell_row<VT>(a.ch[c], r, x);
            active = true;
        }
    }
    if (active) {
        double ybar = 0.0;
        double yr = (double)Y[r];
#pragma unroll
        for (int c = 0; c < kMaxCh; ++c)
            if (c < a.nch) {
                double uc = a.alpha * u[c];
                ybar += a.chw[c] * uc;
#pragma unroll
                for (int k = 0; k < kMaxPar; ++k)
                    if (k == a.gidx[c]) g[k] += a.gfac[c] * uc * yr;
            }
        double xr = a.alpha * (double)x[r];
        for (int q = 0; q < a.nkp; ++q) {
            double kv = a.kp[q][r];
#pragma unroll
            for (int k = 0; k < kMaxPar; ++k)
                if (k == a.kp_gidx[q]) g[k] += xr * kv;
        }
        adj_epilogue<STAGE, VT>(a, r, ybar, lam, lacc, kb_out, w, lam_out);
    }
    // block reduction of the gradient partials into this block's fixed slots
    __shared__ double red[kWarps][kMaxPar];
#pragma unroll
    for (int k = 0; k < kMaxPar; ++k) {
        double v = g[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < a.npar) {
        double s = 0.0;
        for (int ww = 0; ww < kWarps; ++ww) s += red[ww][threadIdx.x];
        part[(long long)blockIdx.x * a.npar + threadIdx.x] += s;
    }
}

__global__ void k_fill_scaled(double *__restrict__ y, const double *__restrict__ x, double a, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = a * x[i];
}

}  // namespace

void adjoint_timeavg(gksl_ctx *c, const double *o_diag, long long S, long long period, int precision, double *loss,
                     double *grad, int n_grad) {
    GK_REQUIRE(c->assembled, GKSL_ERR_STATE, "gksl_assemble must be called first");
    GK_REQUIRE(c->has_adj, GKSL_ERR_STATE, "gksl_adjoint_timeavg needs gksl_assemble with GKSL_ASM_TRANSPOSE");
    GK_REQUIRE(c->state_set, GKSL_ERR_STATE, "no state: call gksl_set_rho0 or gksl_set_state first");
    GK_REQUIRE(precision == 64 || precision == 32, GKSL_ERR_ARG, "precision must be 64 or 32");
    if (precision == 32)
        GK_REQUIRE(c->asm_flags & GKSL_ASM_FP32, GKSL_ERR_STATE, "precision 32 needs gksl_assemble with GKSL_ASM_FP32");
    cudaStream_t s = c->stream;
    const long long D = c->D, D1 = D + 1;
    // parameter layout [A, gamma_p..., theta_k...]
    int nP = 0, nK = 0;
    for (int p = 0; p < GKSL_MAX_P; ++p) nP += c->has_r[p];
    for (int k = 0; k < GKSL_MAX_H0; ++k) nK += c->has_h0[k];
    const int npar = 1 + nP + nK;
    GK_REQUIRE(n_grad == npar, GKSL_ERR_ARG,
               "n_grad must equal 1 + (number of dissipators) + (number of H0 components) = " + std::to_string(npar));
    ensure_work(c, precision == 32);
    const double T = 2.0 * M_PI / c->omega;
    const double h = T / (double)S;
    const long long nsteps = period * S, first = (period - 1) * S;
    const double t0 = c->t;
    check_drive_grid(c, S, h);
    fill_eps_table(c, t0, h, nsteps);

    // channel descriptors
    int slot_gamma[GKSL_MAX_P], slot_theta[GKSL_MAX_H0];
    {
        int q = 1;
        for (int p = 0; p < GKSL_MAX_P; ++p) slot_gamma[p] = c->has_r[p] ? q++ : -1;
        for (int k = 0; k < GKSL_MAX_H0; ++k) slot_theta[k] = c->has_h0[k] ? q++ : -1;
    }
    AdjArgs<double> a64{};
    AdjArgs<float> a32{};
    auto setup = [&](auto &a, auto view_of) {
        a.nch = c->adj_n;
        a.npar = npar;
        for (int i = 0; i < c->adj_n; ++i) {
            a.ch[i] = view_of(i);
            int kind = c->adj_kind[i], idx = c->adj_index[i];
            if (kind == 0) { a.chw[i] = c->h0[idx].weight; a.gidx[i] = slot_theta[idx]; a.gfac[i] = 1.0; }
            if (kind == 1) { a.chw[i] = 0.0; a.gidx[i] = 0; a.gfac[i] = 0.0; }   // set per stage
            if (kind == 2) { a.chw[i] = c->diss[idx].weight; a.gidx[i] = slot_gamma[idx]; a.gfac[i] = 1.0; }
        }
        a.nkp = 0;
        for (int p = 0; p < GKSL_MAX_P; ++p)
            if (c->has_r[p]) { a.kp[a.nkp] = c->Kp[p].p; a.kp_gidx[a.nkp++] = slot_gamma[p]; }
        a.h = h;
        a.h2 = 0.5 * h;
        a.h3 = h / 3.0;
        a.h6 = h / 6.0;
        a.long_rows = c->adj[0].long_rows.p;
        a.n_long = c->adj[0].n_long;
        a.nb_long = (int)((a.n_long + kWarps - 1) / kWarps);
        a.D = D;
    };
    setup(a64, [&](int i) { return view(c->adj[i]); });
    if (precision == 32) setup(a32, [&](int i) { return view(c->adjf[i]); });
    int q1ch = -1;
    for (int i = 0; i < c->adj_n; ++i)
        if (c->adj_kind[i] == 1) q1ch = i;
    const unsigned grid = (unsigned)(a64.nb_long + (D + kThreads - 1) / kThreads);

    // observable weights (dense, zero off the D block)
    DBuf<double> w((size_t)D1), c0(1);
    GK_CUDA(cudaMemsetAsync(w.p, 0, sizeof(double) * D1, s));
    observable_weights(c, o_diag, w.p, c0.p);
    // trapezoid weights of the loss period
    std::vector<double> wt((size_t)S + 1, 1.0 / (double)S);
    wt[0] = wt[S] = 0.5 / (double)S;

    // buffers
    DBuf<double> v_save((size_t)D1), ckP((size_t)(period * D1));
    const long long q = std::max(1LL, (long long)std::ceil(std::sqrt((double)S)));
    const long long nseg = (S + q - 1) / q;
    DBuf<double> seg((size_t)(nseg * D1)), traj((size_t)((q + 1) * D1));
    DBuf<double> lam((size_t)D1), lacc((size_t)D1), obs((size_t)(S + 1));
    DBuf<double> part((size_t)grid * npar);
    GK_CUDA(cudaMemsetAsync(part.p, 0, sizeof(double) * grid * npar, s));
    // stage inputs and adjoint vectors in the working precision
    DBuf<double> Y2d, Y3d, Y4d, kbAd, kbBd;
    DBuf<float> Y1f, Y2f, Y3f, Y4f, kbAf, kbBf, lamf;
    // stage inputs carry the constant 1 at index D (it multiplies the K column)
    const double one = 1.0;
    const float onef = 1.0f;
    if (precision == 64) {
        Y2d.alloc((size_t)D1); Y3d.alloc((size_t)D1); Y4d.alloc((size_t)D1);
        kbAd.alloc((size_t)D1); kbBd.alloc((size_t)D1);
        for (double *p : {Y2d.p, Y3d.p, Y4d.p})
            GK_CUDA(cudaMemcpyAsync(p + D, &one, sizeof(double), cudaMemcpyHostToDevice, s));
    } else {
        Y1f.alloc((size_t)D1); Y2f.alloc((size_t)D1); Y3f.alloc((size_t)D1); Y4f.alloc((size_t)D1);
        kbAf.alloc((size_t)D1); kbBf.alloc((size_t)D1); lamf.alloc((size_t)D1);
        for (float *p : {Y1f.p, Y2f.p, Y3f.p, Y4f.p})
            GK_CUDA(cudaMemcpyAsync(p + D, &onef, sizeof(float), cudaMemcpyHostToDevice, s));
    }
    GK_CUDA(cudaStreamSynchronize(s));
    GK_CUDA(cudaMemcpyAsync(v_save.p, c->v.p, sizeof(double) * D1, cudaMemcpyDeviceToDevice, s));

    auto load_state = [&](const double *src) {
        GK_CUDA(cudaMemcpyAsync(c->v.p, src, sizeof(double) * D1, cudaMemcpyDeviceToDevice, s));
        if (precision == 32) to_f32(c->v.p, c->v32.p, D1, s);
    };
    auto save_state = [&](double *dst) {
        GK_CUDA(cudaMemcpyAsync(dst, c->v.p, sizeof(double) * D1, cudaMemcpyDeviceToDevice, s));
    };

    // 1. forward pass: period checkpoints
    load_state(v_save.p);
    for (long long p = 0; p < period; ++p) {
        save_state(ckP.p + p * D1);
        advance(c, precision, h, p * S, S);
    }
    // 2. reverse sweep
    k_fill_scaled<<<grid_for(D1, 256), 256, 0, s>>>(lam.p, w.p, wt[S], D1);
    GK_LAUNCH_CHECK();
    for (long long p = period - 1; p >= 0; --p) {
        // sqrt(S)-spaced checkpoints of this period (and the observable on the loss period)
        load_state(ckP.p + p * D1);
        const bool loss_period = (p == period - 1);
        for (long long j = 0; j < nseg; ++j) {
            save_state(seg.p + j * D1);
            long long len = std::min(q, S - j * q);
            if (loss_period) {
                for (long long i = 0; i < len; ++i) {
                    observable_apply(c, w.p, c0.p, c->v.p, 1, D1, obs.p + j * q + i);
                    advance(c, precision, h, p * S + j * q + i, 1);
                }
            } else {
                advance(c, precision, h, p * S + j * q, len);
            }
        }
        if (loss_period) observable_apply(c, w.p, c0.p, c->v.p, 1, D1, obs.p + S);
        for (long long j = nseg - 1; j >= 0; --j) {
            long long len = std::min(q, S - j * q);
            load_state(seg.p + j * D1);
            save_state(traj.p);
            for (long long i = 0; i < len; ++i) {
                advance(c, precision, h, p * S + j * q + i, 1);
                save_state(traj.p + (i + 1) * D1);
            }
            for (long long i = len - 1; i >= 0; --i) {
                const long long gstep = p * S + j * q + i;
                const double tn = t0 + (double)gstep * h;
                double th3[3];
                drive_theta(c->drive_shape, c->omega, tn, h, th3);
                const double thst[4] = {th3[0], th3[1], th3[1], th3[2]};   // theta at stages 1..4
                const long long m = gstep - first;
                const double beta = (m >= 0 && m < S) ? wt[m] : 0.0;
                double *vn = traj.p + i * D1;
                if (precision == 64) {
                    forward_stage_inputs(c, 64, h, gstep, vn, Y2d.p, Y3d.p, Y4d.p);
                    const double *Ys[4] = {vn, Y2d.p, Y3d.p, Y4d.p};
                    for (int st = 4; st >= 1; --st) {
                        double sn = thst[st - 1];
                        if (q1ch >= 0) {
                            a64.chw[q1ch] = c->E + c->A * sn;
                            a64.gfac[q1ch] = sn;
                        }
                        a64.alpha = st == 4 ? h / 6.0 : 1.0;
                        a64.beta = beta;
                        const double *xin = st == 4 ? lam.p : (st == 3 ? kbAd.p : (st == 2 ? kbBd.p : kbAd.p));
                        double *kout = st == 4 ? kbAd.p : (st == 3 ? kbBd.p : (st == 2 ? kbAd.p : nullptr));
                        const double *Y = Ys[st - 1];
                        switch (st) {
                            case 4: k_adjoint<4, double><<<grid, kThreads, 0, s>>>(a64, xin, Y, lam.p, lacc.p, kout, w.p, lam.p, part.p); break;
                            case 3: k_adjoint<3, double><<<grid, kThreads, 0, s>>>(a64, xin, Y, lam.p, lacc.p, kout, w.p, lam.p, part.p); break;
                            case 2: k_adjoint<2, double><<<grid, kThreads, 0, s>>>(a64, xin, Y, lam.p, lacc.p, kout, w.p, lam.p, part.p); break;
                            case 1: k_adjoint<1, double><<<grid, kThreads, 0, s>>>(a64, xin, Y, lam.p, lacc.p, kout, w.p, lam.p, part.p); break;
                        }
                        GK_LAUNCH_CHECK();
                    }
                } else {
                    to_f32(vn, Y1f.p, D1, s);
                    forward_stage_inputs(c, 32, h, gstep, Y1f.p, Y2f.p, Y3f.p, Y4f.p);
                    to_f32(lam.p, lamf.p, D1, s);
                    const float *Ys[4] = {Y1f.p, Y2f.p, Y3f.p, Y4f.p};
                    for (int st = 4; st >= 1; --st) {
                        double sn = thst[st - 1];
                        if (q1ch >= 0) {
                            a32.chw[q1ch] = c->E + c->A * sn;
                            a32.gfac[q1ch] = sn;
                        }
                        a32.alpha = st == 4 ? h / 6.0 : 1.0;
                        a32.beta = beta;
                        const float *xin = st == 4 ? lamf.p : (st == 3 ? kbAf.p : (st == 2 ? kbBf.p : kbAf.p));
                        float *kout = st == 4 ? kbAf.p : (st == 3 ? kbBf.p : (st == 2 ? kbAf.p : nullptr));
                        const float *Y = Ys[st - 1];
                        switch (st) {
                            case 4: k_adjoint<4, float><<<grid, kThreads, 0, s>>>(a32, xin, Y, lam.p, lacc.p, kout, w.p, lam.p, part.p); break;
                            case 3: k_adjoint<3, float><<<grid, kThreads, 0, s>>>(a32, xin, Y, lam.p, lacc.p, kout, w.p, lam.p, part.p); break;
                            case 2: k_adjoint<2, float><<<grid, kThreads, 0, s>>>(a32, xin, Y, lam.p, lacc.p, kout, w.p, lam.p, part.p); break;
                            case 1: k_adjoint<1, float><<<grid, kThreads, 0, s>>>(a32, xin, Y, lam.p, lacc.p, kout, w.p, lam.p, part.p); break;
                        }
                        GK_LAUNCH_CHECK();
                    }
                }
            }
        }
    }
    // 3. loss and gradient, reduced in a fixed order
    std::vector<double> ho((size_t)S + 1), hp((size_t)grid * npar);
    GK_CUDA(cudaMemcpyAsync(ho.data(), obs.p, sizeof(double) * (S + 1), cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaMemcpyAsync(hp.data(), part.p, sizeof(double) * grid * npar, cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaStreamSynchronize(s));
    double L = 0.0;
    for (long long m = 0; m <= S; ++m) L += wt[m] * ho[m];
    *loss = L;
    for (int k = 0; k < npar; ++k) {
        double g = 0.0;
        for (unsigned b = 0; b < grid; ++b) g += hp[(size_t)b * npar + k];
        grad[k] = g;
    }
    // restore the state
    load_state(v_save.p);
    GK_CUDA(cudaStreamSynchronize(s));
}

}  // namespace gk
