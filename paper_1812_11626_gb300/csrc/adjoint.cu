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
// Schedule: checkpoints every q steps (q ~ sqrt(S/4)) from one forward pass when they fit in
// memory, else period checkpoints and, period by period in reverse, a forward pass that sets
// the checkpoints of the period's segments; then segment by segment in reverse a CUDA graph
// that re-runs the segment's q steps forward, keeping every stage input Y1..Y4 of each step,
// and one that sweeps the same steps backwards on a second stream.  With two stage-input
// buffers the forward graph of the next segment runs while the current one is swept backwards
// (the small systems' kernels leave most of the GPU idle); events order each buffer's writer
// after its previous reader.  Every per-step scalar (the drive at the stage
// times, the loss weight of the step) is read from device tables indexed by the step, so one
// graph per segment length serves every segment.  Each state is computed twice (three times
// without room for every checkpoint); memory is periods * S/q state checkpoints (periods + S/q
// without room) plus 4 q stage inputs.
#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <vector>

#include "internal.cuh"
#include "prim.cuh"

namespace gk {

namespace {

constexpr int kThreads = 256;   // largest block; small systems launch smaller ones (adj_grid)
constexpr int kWarps = kThreads / 32;
constexpr int kMaxCh = gksl_ctx::kMaxCh;

template <typename VT>
struct AdjArgs {
    HybView<VT> ch[kMaxCh];
    double chw[kMaxCh];     // weight of channel c in A^T
    int nch;
    const double *kp[GKSL_MAX_P];   // K_p per unit rate: d b / d gamma_p
    int nkp;
    int q1ch;                  // channel of Q1 (-1: none): weight E + A theta, gradient factor theta
    double E, A;
    const double *theta;       // theta(t) at the three stage times of every step
    const long long *base;     // the step is *base + local
    long long local;
    long long first, S;        // loss period: steps [first, first + S)
    double w_edge, w_mid;      // trapezoid weights 1/(2S) and 1/S (stage 1: lam += weight * w)
    double h, h2, h3, h6;   // h, h/2, h/3, h/6 (computed on the host)
    const int *long_rows;
    long long n_long;
    int nb_long;
    long long D;
    int pipe;    // four-channel slot loads issued together (ell_rows4), for small systems
    // wide form (k_adjoint_wide): the ELL blocks of the (at most four) channels stacked into
    // one block of W_st slots, channel c's slot s at off[c] + s (off[c] = W_st past the last)
    const int *st_col;
    const VT *st_val;
    long long ld_st;
    int W_st;
    int off[4];
    int wm;   // host side: the kernel's slot capacity (0: k_adjoint)
    float chwf[4], Ef, Af;   // the channel weights and E, A in float (the wide FP32 stages)
};

// (C x)_r over the ELL slots of row r; the slot loads go out four at a time before their gathers
template <typename VT>
__device__ inline double ell_row(const HybView<VT> &H, long long r, const VT *__restrict__ x) {
    double s = 0.0;
    const int wd = H.width;
    int j = 0;
    for (; j + 4 <= wd; j += 4) {
        int cc[4];
        VT vv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            long long p = (long long)(j + u) * H.ld + r;
            cc[u] = __ldcs(H.ell_col + p);
            vv[u] = __ldcs(H.ell_val + p);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) s += (double)vv[u] * (double)__ldg(x + cc[u]);
    }
    for (; j < wd; ++j) {
        long long p = (long long)j * H.ld + r;
        s += (double)__ldcs(H.ell_val + p) * (double)__ldg(x + __ldcs(H.ell_col + p));
    }
    return s;
}

// (C_c x)_r of four channels at once: the first four ELL slots of every channel are loaded
// together (one round trip for up to 16 entries instead of one per channel), then each channel's
// remaining slots four at a time.  Each channel's sum runs over its slots in the same order as
// ell_row, so the results are the same bit for bit; it holds more registers, so it serves the
// small systems whose rows leave most warp slots of the GPU empty.
template <typename VT>
__device__ inline void ell_rows4(const HybView<VT> *H, int nch, long long r, const VT *__restrict__ x,
                                 double (&u)[4]) {
    int cc[4][4];
    VT vv[4][4];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool on = c < nch && j < H[c].width;
            const long long p = (long long)j * H[c].ld + r;
            cc[c][j] = on ? __ldcs(H[c].ell_col + p) : 0;
            vv[c][j] = on ? __ldcs(H[c].ell_val + p) : VT(0);
        }
    VT xx[4][4];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int j = 0; j < 4; ++j) xx[c][j] = (c < nch && j < H[c].width) ? __ldg(x + cc[c][j]) : VT(0);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        double s = 0.0;
        if (c < nch) {
            const int wd = H[c].width;
            if (wd >= 4) {
#pragma unroll
                for (int j = 0; j < 4; ++j) s += (double)vv[c][j] * (double)xx[c][j];
                int j = 4;
                for (; j + 4 <= wd; j += 4) {
                    int c4[4];
                    VT v4[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const long long p = (long long)(j + k) * H[c].ld + r;
                        c4[k] = __ldcs(H[c].ell_col + p);
                        v4[k] = __ldcs(H[c].ell_val + p);
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k) s += (double)v4[k] * (double)__ldg(x + c4[k]);
                }
                for (; j < wd; ++j) {
                    const long long p = (long long)j * H[c].ld + r;
                    s += (double)__ldcs(H[c].ell_val + p) * (double)__ldg(x + __ldcs(H[c].ell_col + p));
                }
            } else {
                for (int j = 0; j < wd; ++j) s += (double)vv[c][j] * (double)xx[c][j];
            }
        }
        u[c] = s;
    }
}

// (C x)_r of a long row by one warp: four entries per lane in flight, then a warp reduction
template <typename VT>
__device__ inline double tail_row(const HybView<VT> &H, long long i, int lane, const VT *__restrict__ x) {
    double s = 0.0;
    const int e1 = H.tail_ptr[i + 1];
    int e = H.tail_ptr[i] + lane;
    for (; e + 96 < e1; e += 128) {
        int cc[4];
        VT vv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            cc[u] = H.tail_col[e + 32 * u];
            vv[u] = __ldcs(H.tail_val + e + 32 * u);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) s += (double)vv[u] * (double)__ldg(x + cc[u]);
    }
    for (; e < e1; e += 32) s += (double)__ldcs(H.tail_val + e) * (double)__ldg(x + H.tail_col[e]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Warp sums of the 8 values v[0..7] of every lane in 9 shuffle-adds: each round halves the set
// a lane keeps (bits 16, 8, 4 of the lane index pick the half), the last two rounds finish the
// sum inside groups of four lanes.  Afterwards lane l holds the sum of slot
// 4 (l >> 4 & 1) + 2 (l >> 3 & 1) + (l >> 2 & 1) in v[0].
template <typename T>
__device__ inline void warp_sum8(T v[8], int lane) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const bool hi = lane & 16;
        const T send = hi ? v[k] : v[k + 4];
        const T keep = hi ? v[k + 4] : v[k];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const bool hi = lane & 8;
        const T send = hi ? v[k] : v[k + 2];
        const T keep = hi ? v[k + 2] : v[k];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    {
        const bool hi = lane & 4;
        const T send = hi ? v[0] : v[1];
        const T keep = hi ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
}

template <int STAGE, typename VT>
__device__ inline void adj_epilogue(const AdjArgs<VT> &a, long long r, double ybar, const double *__restrict__ lam,
                                    double *__restrict__ lacc, VT *__restrict__ kb_out, const double *__restrict__ w,
                                    double *lam_out, double beta) {
    if (STAGE == 4) { kb_out[r] = (VT)(a.h3 * lam[r] + a.h * ybar); lacc[r] = lam[r] + ybar; }
    if (STAGE == 3) { kb_out[r] = (VT)(a.h3 * lam[r] + a.h2 * ybar); lacc[r] = lacc[r] + ybar; }
    if (STAGE == 2) { kb_out[r] = (VT)(a.h6 * lam[r] + a.h2 * ybar); lacc[r] = lacc[r] + ybar; }
    if (STAGE == 1) { lam_out[r] = lacc[r] + ybar + beta * w[r]; }
}

// One reverse stage for NC >= nch channels.  x: the gathered vector (lam' for stage 4, kb_i
// otherwise); Y: the forward stage input Y_i (own row).  Threads walk rows with a grid stride
// (the first nb_long blocks: one warp per long row; the rest: one thread per ELL row) and keep
// their gradient partials in registers: slot c collects u_c . Y (u_c = (C_c x)_r), slot NC + q
// collects x . K_q.  The constant factors of a launch (alpha = h/6 at stage 4, theta(t) of the
// Q1 slot) are applied once per block when the partials go to this block's fixed slots of
// `part`; the host maps slots to parameters.
template <int STAGE, typename VT, int NC, bool PIPE = false>
__global__ void __launch_bounds__(kThreads) k_adjoint(AdjArgs<VT> a, const VT *__restrict__ x,
                                                     const VT *__restrict__ Y, const double *lam, double *lacc,
                                                     VT *__restrict__ kb_out, const double *__restrict__ w,
                                                     double *lam_out, double *__restrict__ part) {
    constexpr int NSLOT = 2 * NC;
    const long long step = *a.base + a.local;
    const double th = a.theta[3 * step + (STAGE == 1 ? 0 : (STAGE == 4 ? 2 : 1))];
    const double alpha = STAGE == 4 ? a.h6 : 1.0;   // kb = alpha * x
    double beta = 0.0;
    if (STAGE == 1) {
        const long long m = step - a.first;
        beta = (m >= 0 && m < a.S) ? (m == 0 ? a.w_edge : a.w_mid) : 0.0;
    }
    double chw[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) chw[c] = c == a.q1ch ? a.E + a.A * th : (c < a.nch ? a.chw[c] : 0.0);
    double g[NSLOT];
#pragma unroll
    for (int k = 0; k < NSLOT; ++k) g[k] = 0.0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nthr = blockDim.x, nwarp = nthr >> 5;
    double u[NC];
    // own-row part of the stage: the epilogue and the gradient partials of row r
    auto finish_row = [&](long long r, const double (&u)[NC]) {
        const double yr = (double)Y[r];
        double ysum = 0.0;
#pragma unroll
        for (int c = 0; c < NC; ++c)
            if (c < a.nch) {
                ysum += chw[c] * (double)u[c];
                g[c] += (double)u[c] * yr;
            }
        const double xr = (double)x[r];
#pragma unroll
        for (int q = 0; q < NC; ++q)
            if (q < a.nkp) g[NC + q] += xr * a.kp[q][r];
        adj_epilogue<STAGE, VT>(a, r, alpha * ysum, lam, lacc, kb_out, w, lam_out, beta);
    };
    if ((int)blockIdx.x < a.nb_long) {
        for (long long i = (long long)blockIdx.x * nwarp + warp; i < a.n_long; i += (long long)a.nb_long * nwarp) {
#pragma unroll
            for (int c = 0; c < NC; ++c) u[c] = c < a.nch ? tail_row<VT>(a.ch[c], i, lane, x) : 0.0;
            if (lane == 0) finish_row(a.long_rows[i], u);
        }
    } else {
        const long long stride = (long long)(gridDim.x - a.nb_long) * nthr;
        for (long long r = (long long)(blockIdx.x - a.nb_long) * nthr + threadIdx.x; r < a.D; r += stride) {
            if (__ldcs(a.ch[0].ell_col + r) < 0) continue;   // long row, handled by a warp above
            if constexpr (PIPE && NC == 4) {
                ell_rows4<VT>(a.ch, a.nch, r, x, u);
            } else {
#pragma unroll
                for (int c = 0; c < NC; ++c) u[c] = c < a.nch ? ell_row<VT>(a.ch[c], r, x) : 0.0;
            }
            finish_row(r, u);
        }
    }
    // block reduction of the partials into this block's fixed slots
    __shared__ double red[kWarps][NSLOT];
    if constexpr (NSLOT == 8) {
        warp_sum8(g, lane);
        if ((lane & 3) == 0) red[warp][4 * (lane >> 4 & 1) + 2 * (lane >> 3 & 1) + (lane >> 2 & 1)] = g[0];
    } else {
#pragma unroll
        for (int k = 0; k < NSLOT; ++k) {
            double v = g[k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp][k] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x < NSLOT) {
        const int k = threadIdx.x;
        double sum = 0.0;
        for (int ww = 0; ww < nwarp; ++ww) sum += red[ww][k];
        double f = alpha;
        if (k == a.q1ch) f *= th;
        part[(long long)blockIdx.x * NSLOT + k] += f * sum;
    }
}

// One reverse stage of a system with at most four channels whose stacked ELL slots (all
// channels' slots in one list, channel c's slot s at off[c] + s) number at most WM, one thread
// per row.  Every slot load and the row's own operands (Y_r, x_r, K_q,r, lam_r, lacc_r) go out
// at once, then every gather: two round trips to L2 per row instead of one pair per batch of four
// slots.  The channel boundaries are the same for every row, so the per-channel sums switch at
// fixed slots without divergence.  Each channel sums its slots in order in AT: double for the
// FP64 stages, float for the FP32 ones (as the FP32 forward stage does).  The FP64 stages form
// the weighted sum, the gradient partials and the stage outputs in double; the FP32 stages form
// the weighted sum, this thread's gradient partials and their warp sums in float and only the
// updates of the adjoint state, and the sums over warps and blocks, in double.  Long rows go to warps as in k_adjoint.  The FP32
// instances are held to two 256-thread blocks per SM (128 registers, a few dozen bytes spilled
// at 24 slots): at N = 1000 that takes a period-2 gradient from 754 to 609 us per step, and
// N = 200 does not move; the weighting and partials in float take it on to 504 us.
template <int STAGE, typename VT, typename AT, int WM>
__global__ void __launch_bounds__(kThreads, sizeof(VT) == 4 ? 2 : 1) k_adjoint_wide(AdjArgs<VT> a, const VT *__restrict__ x,
                                                          const VT *__restrict__ Y, const double *lam, double *lacc,
                                                          VT *__restrict__ kb_out, const double *__restrict__ w,
                                                          double *lam_out, double *__restrict__ part) {
    constexpr int NC = 4, NSLOT = 8;
    const long long step = *a.base + a.local;
    const double th = a.theta[3 * step + (STAGE == 1 ? 0 : (STAGE == 4 ? 2 : 1))];
    const double alpha = STAGE == 4 ? a.h6 : 1.0;
    double beta = 0.0;
    if (STAGE == 1) {
        const long long m = step - a.first;
        beta = (m >= 0 && m < a.S) ? (m == 0 ? a.w_edge : a.w_mid) : 0.0;
    }
    double chw[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) chw[c] = c == a.q1ch ? a.E + a.A * th : (c < a.nch ? a.chw[c] : 0.0);
    double g[NSLOT];
#pragma unroll
    for (int k = 0; k < NSLOT; ++k) g[k] = 0.0;
    // FP32 stages: the weights in float (the drive's from theta in float), and this thread's
    // partials of the ELL rows in float
    float chwf[NC], gf[NSLOT];
    if constexpr (sizeof(AT) == 4) {
        const float thf = (float)th;
#pragma unroll
        for (int c = 0; c < NC; ++c) chwf[c] = c == a.q1ch ? fmaf(a.Af, thf, a.Ef) : a.chwf[c];
    }
#pragma unroll
    for (int k = 0; k < NSLOT; ++k) gf[k] = 0.0f;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nthr = blockDim.x, nwarp = nthr >> 5;
    // own-row part: gradient partials of row r and the stage outputs
    auto finish_row = [&](long long r, const auto (&u)[NC], double yr, double xr, const double (&kr)[NC],
                          double lamr, double laccr, double wr) {
        double ysum = 0.0;
#pragma unroll
        for (int c = 0; c < NC; ++c)
            if (c < a.nch) {
                ysum += chw[c] * u[c];
                g[c] += u[c] * yr;
            }
#pragma unroll
        for (int q = 0; q < NC; ++q)
            if (q < a.nkp) g[NC + q] += xr * kr[q];
        const double ybar = alpha * ysum;
        if (STAGE == 4) { kb_out[r] = (VT)(a.h3 * lamr + a.h * ybar); lacc[r] = lamr + ybar; }
        if (STAGE == 3) { kb_out[r] = (VT)(a.h3 * lamr + a.h2 * ybar); lacc[r] = laccr + ybar; }
        if (STAGE == 2) { kb_out[r] = (VT)(a.h6 * lamr + a.h2 * ybar); lacc[r] = laccr + ybar; }
        if (STAGE == 1) lam_out[r] = laccr + ybar + beta * wr;
    };
    auto own_loads = [&](long long r, double &yr, double &xr, double (&kr)[NC], double &lamr, double &laccr,
                         double &wr) {
        yr = (double)Y[r];
        xr = (double)x[r];
#pragma unroll
        for (int q = 0; q < NC; ++q) kr[q] = q < a.nkp ? a.kp[q][r] : 0.0;
        lamr = STAGE != 1 ? lam[r] : 0.0;
        laccr = STAGE != 4 ? lacc[r] : 0.0;
        wr = STAGE == 1 ? w[r] : 0.0;
    };
    if ((int)blockIdx.x < a.nb_long) {
        for (long long i = (long long)blockIdx.x * nwarp + warp; i < a.n_long; i += (long long)a.nb_long * nwarp) {
            double u[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) u[c] = c < a.nch ? tail_row<VT>(a.ch[c], i, lane, x) : 0.0;
            if (lane == 0) {
                const long long r = a.long_rows[i];
                double yr, xr, kr[NC], lamr, laccr, wr;
                own_loads(r, yr, xr, kr, lamr, laccr, wr);
                finish_row(r, u, yr, xr, kr, lamr, laccr, wr);
            }
        }
    } else {
        const int W = a.W_st;
        const int o1 = a.off[1], o2 = a.off[2], o3 = a.off[3];
        const long long stride = (long long)(gridDim.x - a.nb_long) * nthr;
        for (long long r = (long long)(blockIdx.x - a.nb_long) * nthr + threadIdx.x; r < a.D; r += stride) {
            int cc[WM];
            VT vv[WM];
#pragma unroll
            for (int k = 0; k < WM; ++k) {
                const long long p = (long long)k * a.ld_st + r;
                cc[k] = k < W ? __ldcs(a.st_col + p) : 0;
                vv[k] = k < W ? __ldcs(a.st_val + p) : VT(0);
            }
            double yr, xr, kr[NC], lamr, laccr, wr;
            own_loads(r, yr, xr, kr, lamr, laccr, wr);
            if (cc[0] < 0) continue;   // channel 0, slot 0: -1 marks a long row, handled by a warp above
            VT xx[WM];
#pragma unroll
            for (int k = 0; k < WM; ++k) xx[k] = k < W ? __ldg(x + cc[k]) : VT(0);
            AT uc[NC] = {AT(0), AT(0), AT(0), AT(0)};
            AT s = AT(0);
            int cur = 0;
#pragma unroll
            for (int k = 0; k < WM; ++k)
                if (k < W) {
                    if (k == o1 || k == o2 || k == o3) {   // the same slots for every row
#pragma unroll
                        for (int c = 0; c < NC; ++c) uc[c] = c == cur ? s : uc[c];
                        s = AT(0);
                        ++cur;
                    }
                    s += (AT)vv[k] * (AT)xx[k];
                }
#pragma unroll
            for (int c = 0; c < NC; ++c) uc[c] = c == cur ? s : uc[c];
            if constexpr (sizeof(AT) == 8) {
                finish_row(r, uc, yr, xr, kr, lamr, laccr, wr);
            } else {
                // FP32 stages: the channel weighting and the gradient partials in float too (one
                // conversion per row for the weighted sum), only the adjoint state in double
                const float yf = Y[r], xf = x[r];
                float ys = 0.0f;
#pragma unroll
                for (int c = 0; c < NC; ++c)
                    if (c < a.nch) {
                        ys = fmaf(chwf[c], uc[c], ys);
                        gf[c] = fmaf(uc[c], yf, gf[c]);
                    }
#pragma unroll
                for (int q = 0; q < NC; ++q)
                    if (q < a.nkp) gf[NC + q] = fmaf(xf, (float)kr[q], gf[NC + q]);
                const double ybar = alpha * (double)ys;
                if (STAGE == 4) { kb_out[r] = (VT)(a.h3 * lamr + a.h * ybar); lacc[r] = lamr + ybar; }
                if (STAGE == 3) { kb_out[r] = (VT)(a.h3 * lamr + a.h2 * ybar); lacc[r] = laccr + ybar; }
                if (STAGE == 2) { kb_out[r] = (VT)(a.h6 * lamr + a.h2 * ybar); lacc[r] = laccr + ybar; }
                if (STAGE == 1) lam_out[r] = laccr + ybar + beta * wr;
            }
        }
    }
    // warp sums of the partials: in float for the ELL blocks of the FP32 stages (their partials are
    // all in gf), in double otherwise; one value per slot and warp, kept in double
    __shared__ double red[kWarps][NSLOT];
    const int slot = 4 * (lane >> 4 & 1) + 2 * (lane >> 3 & 1) + (lane >> 2 & 1);
    if (sizeof(AT) == 4 && (int)blockIdx.x >= a.nb_long) {
        warp_sum8(gf, lane);
        if ((lane & 3) == 0) red[warp][slot] = (double)gf[0];
    } else {
        warp_sum8(g, lane);
        if ((lane & 3) == 0) red[warp][slot] = g[0];
    }
    __syncthreads();
    if (threadIdx.x < NSLOT) {
        const int k = threadIdx.x;
        double sum = 0.0;
        for (int ww = 0; ww < nwarp; ++ww) sum += red[ww][k];
        double f = alpha;
        if (k == a.q1ch) f *= th;
        part[(long long)blockIdx.x * NSLOT + k] += f * sum;
    }
}

// blocks of one reverse stage: up to one per SM for the long rows (a warp each), then the ELL
// rows (a thread each), both walked with a grid stride; at most 1024 threads per SM in all (the
// register budget of the 4-channel kernel), so the whole grid is resident at once.  Blocks are
// halved (down to 64 threads) while the rows would fill fewer than four blocks per SM, so that
// a small system's rows spread evenly over every SM (N = 200: 64 threads, 4-15 % faster).
struct AdjGrid {
    int nb_long;
    unsigned total;
    int threads;
};

AdjGrid adj_grid(long long n_long, long long D, int sms) {
    int bt = kThreads;
    while (bt > 64 && (D + bt - 1) / bt < 4LL * sms) bt /= 2;
    const long long per_sm = 1024 / bt, wpb = bt / 32;
    long long nl = std::min<long long>((n_long + wpb - 1) / wpb, sms);
    long long ne = std::min<long long>((D + bt - 1) / bt, per_sm * sms - nl);
    return AdjGrid{(int)nl, (unsigned)(nl + std::max(1LL, ne)), bt};
}

__global__ void k_set_step(long long *p, long long v) { *p = v; }

__global__ void k_fill_scaled(double *__restrict__ y, const double *__restrict__ x, double a, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = a * x[i];
}

__global__ void k_fill1(void *p, long long n, int fp32) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (fp32) ((float *)p)[i] = 1.0f;
    else ((double *)p)[i] = 1.0;
}

// <O> = c0 + sum_l w_l v_{D^l} of the state at grid point m = *base + local - first of the
// loss period (nothing outside it); one block, fixed-order reduction
__global__ void k_obs_step(const double *__restrict__ w, const double *__restrict__ c0, long long P2, int N,
                           const double *__restrict__ v, const long long *base, long long local, long long first,
                           long long S, double *__restrict__ out) {
    const long long m = *base + local - first;
    if (m < 0 || m > S) return;
    double s = 0.0;
    for (int l = threadIdx.x; l < N - 1; l += blockDim.x) s += w[2 * P2 + l] * v[2 * P2 + l];
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[m] = *c0 + red[0];
}

// a stream capture that is ended (and its graph dropped) if the capturing code throws
struct Capture {
    cudaStream_t s;
    bool open = false;
    explicit Capture(cudaStream_t st) : s(st) {
        GK_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        open = true;
    }
    cudaGraphExec_t finish() {
        cudaGraph_t g;
        open = false;
        GK_CUDA(cudaStreamEndCapture(s, &g));
        cudaGraphExec_t e;
        cudaError_t err = cudaGraphInstantiate(&e, g, 0);
        cudaGraphDestroy(g);
        GK_CUDA(err);
        return e;
    }
    ~Capture() {
        if (open) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(s, &g);
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
        }
    }
};

struct ExecSet {
    struct E {
        long long len;
        int mode;
        cudaGraphExec_t exec;
    };
    std::vector<E> v;
    ~ExecSet() {
        for (auto &e : v) cudaGraphExecDestroy(e.exec);
    }
};

template <typename VT, int WM>
void rev_wide(const AdjArgs<VT> &a, unsigned grid, int bt, cudaStream_t s, const VT *lam_in, const VT *Y1,
              const VT *Y2, const VT *Y3, const VT *Y4, VT *ka, VT *kb, double *lam, double *lacc, const double *w,
              double *part) {
    using AT = VT;   // the FP32 stages sum in float, the FP64 ones in double
    k_adjoint_wide<4, VT, AT, WM><<<grid, bt, 0, s>>>(a, lam_in, Y4, lam, lacc, ka, w, lam, part);
    k_adjoint_wide<3, VT, AT, WM><<<grid, bt, 0, s>>>(a, ka, Y3, lam, lacc, kb, w, lam, part);
    k_adjoint_wide<2, VT, AT, WM><<<grid, bt, 0, s>>>(a, kb, Y2, lam, lacc, ka, w, lam, part);
    k_adjoint_wide<1, VT, AT, WM><<<grid, bt, 0, s>>>(a, ka, Y1, lam, lacc, nullptr, w, lam, part);
}

// the four reverse stages of one step: kb4 from lam', then kb3, kb2, and lam from kb1
template <typename VT, int NC>
void rev_stages_t(const AdjArgs<VT> &a, unsigned grid, int bt, cudaStream_t s, const VT *lam_in, const VT *Y1, const VT *Y2,
                  const VT *Y3, const VT *Y4, VT *ka, VT *kb, double *lam, double *lacc, const double *w,
                  double *part) {
    if constexpr (NC == 4) {
        if (a.wm) {
            switch (a.wm) {
                case 8: rev_wide<VT, 8>(a, grid, bt, s, lam_in, Y1, Y2, Y3, Y4, ka, kb, lam, lacc, w, part); break;
                case 16: rev_wide<VT, 16>(a, grid, bt, s, lam_in, Y1, Y2, Y3, Y4, ka, kb, lam, lacc, w, part); break;
                case 24: rev_wide<VT, 24>(a, grid, bt, s, lam_in, Y1, Y2, Y3, Y4, ka, kb, lam, lacc, w, part); break;
                default: rev_wide<VT, 32>(a, grid, bt, s, lam_in, Y1, Y2, Y3, Y4, ka, kb, lam, lacc, w, part); break;
            }
            return;
        }
        if (a.pipe) {
            k_adjoint<4, VT, 4, true><<<grid, bt, 0, s>>>(a, lam_in, Y4, lam, lacc, ka, w, lam, part);
            k_adjoint<3, VT, 4, true><<<grid, bt, 0, s>>>(a, ka, Y3, lam, lacc, kb, w, lam, part);
            k_adjoint<2, VT, 4, true><<<grid, bt, 0, s>>>(a, kb, Y2, lam, lacc, ka, w, lam, part);
            k_adjoint<1, VT, 4, true><<<grid, bt, 0, s>>>(a, ka, Y1, lam, lacc, nullptr, w, lam, part);
            return;
        }
    }
    k_adjoint<4, VT, NC><<<grid, bt, 0, s>>>(a, lam_in, Y4, lam, lacc, ka, w, lam, part);
    k_adjoint<3, VT, NC><<<grid, bt, 0, s>>>(a, ka, Y3, lam, lacc, kb, w, lam, part);
    k_adjoint<2, VT, NC><<<grid, bt, 0, s>>>(a, kb, Y2, lam, lacc, ka, w, lam, part);
    k_adjoint<1, VT, NC><<<grid, bt, 0, s>>>(a, ka, Y1, lam, lacc, nullptr, w, lam, part);
}

// the four reverse stages of one step: kb4 from lam', then kb3, kb2, and lam from kb1
template <typename VT>
void rev_stages(const AdjArgs<VT> &a, int NC, unsigned grid, int bt, cudaStream_t s, const VT *lam_in, const VT *Y1,
                const VT *Y2, const VT *Y3, const VT *Y4, VT *ka, VT *kb, double *lam, double *lacc, const double *w,
                double *part) {
    if (NC == 4) rev_stages_t<VT, 4>(a, grid, bt, s, lam_in, Y1, Y2, Y3, Y4, ka, kb, lam, lacc, w, part);
    else rev_stages_t<VT, kMaxCh>(a, grid, bt, s, lam_in, Y1, Y2, Y3, Y4, ka, kb, lam, lacc, w, part);
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
    const bool f32 = precision == 32;
    // parameter layout [A, gamma_p..., theta_k...]
    int nP = 0, nK = 0;
    for (int p = 0; p < GKSL_MAX_P; ++p) nP += c->has_r[p];
    for (int k = 0; k < GKSL_MAX_H0; ++k) nK += c->has_h0[k];
    const int npar = 1 + nP + nK;
    GK_REQUIRE(n_grad == npar, GKSL_ERR_ARG,
               "n_grad must equal 1 + (number of dissipators) + (number of H0 components) = " + std::to_string(npar));
    ensure_work(c, f32);
    const double T = 2.0 * M_PI / c->omega;
    const double h = T / (double)S;
    const long long nsteps = period * S, first = (period - 1) * S;
    const double t0 = c->t;
    check_drive_grid(c, S, h);
    fill_eps_table(c, t0, h, std::max(nsteps, 8LL));   // the variant timer below reads 8 steps
    // the forward passes use the stage-kernel variant the timer picks for this matrix, as
    // gksl_propagate does (a context used only for gradients would otherwise keep variant 0)
    tune_stage_variant(c, precision, h);
    DBuf<double> theta((size_t)(3 * nsteps));
    fill_theta_table(c, t0, h, nsteps, theta.p);

    // channel descriptors
    int slot_gamma[GKSL_MAX_P], slot_theta[GKSL_MAX_H0];
    {
        int q = 1;
        for (int p = 0; p < GKSL_MAX_P; ++p) slot_gamma[p] = c->has_r[p] ? q++ : -1;
        for (int k = 0; k < GKSL_MAX_H0; ++k) slot_theta[k] = c->has_h0[k] ? q++ : -1;
    }
    AdjArgs<double> a64{};
    AdjArgs<float> a32{};
    // gradient slot of each channel and of each K_p (the kernel's partials are per channel)
    int gidx[kMaxCh], kp_gidx[GKSL_MAX_P];
    auto setup = [&](auto &a, auto view_of) {
        a.nch = c->adj_n;
        a.q1ch = -1;
        for (int i = 0; i < c->adj_n; ++i) {
            a.ch[i] = view_of(i);
            int kind = c->adj_kind[i], idx = c->adj_index[i];
            if (kind == 0) { a.chw[i] = c->h0[idx].weight; gidx[i] = slot_theta[idx]; }
            if (kind == 1) { a.chw[i] = 0.0; gidx[i] = 0; a.q1ch = i; }   // E + A theta(t), on the device
            if (kind == 2) { a.chw[i] = c->diss[idx].weight; gidx[i] = slot_gamma[idx]; }
        }
        a.nkp = 0;
        for (int p = 0; p < GKSL_MAX_P; ++p)
            if (c->has_r[p]) { a.kp[a.nkp] = c->Kp[p].p; kp_gidx[a.nkp++] = slot_gamma[p]; }
        a.E = c->E;
        a.A = c->A;
        a.theta = theta.p;
        a.base = c->step_base.p;
        a.first = first;
        a.S = S;
        a.w_edge = 0.5 / (double)S;
        a.w_mid = 1.0 / (double)S;
        a.h = h;
        a.h2 = 0.5 * h;
        a.h3 = h / 3.0;
        a.h6 = h / 6.0;
        a.long_rows = c->adj[0].long_rows.p;
        a.n_long = c->adj[0].n_long;
        a.D = D;
    };
    setup(a64, [&](int i) { return view(c->adj[i]); });
    if (f32) setup(a32, [&](int i) { return view(c->adjf[i]); });
    int sms = 0;
    GK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    const AdjGrid ag = adj_grid(a64.n_long, D, sms);
    a64.nb_long = a32.nb_long = ag.nb_long;
    // small systems (blocks already shrunk to 64 threads, few warps per SM): the FP64 reverse
    // stages issue the four channels' first slots together (N = 200 period-20 gradient: 21.6 ->
    // 20.4 s; the FP32 stages measured 4 % slower with it and keep the channel-by-channel loop);
    // GKSL_ADJ_PIPE=0/1 forces it off/on in either precision
    {
        const char *env = getenv("GKSL_ADJ_PIPE");
        const bool can = c->adj_n <= 4;
        a64.pipe = (can && (env ? env[0] == '1' : ag.threads <= 64)) ? 1 : 0;
        a32.pipe = (can && env && env[0] == '1') ? 1 : 0;
    }
    unsigned grid = ag.total;
    int bt_rev = ag.threads;
    // wide reverse stages (k_adjoint_wide) for systems with at most four channels whose rows fit
    // in 32 stacked slots: the FP32 stages by default (N = 200, 300, 500: 16, 22, 12 % more
    // gradient steps per second, mostly from summing in float), not the FP64 ones (N = 200: 17 %
    // fewer; their FP64 chain, about 45 FP64 operations per row, then overlaps none of the
    // loads).  GKSL_ADJ_WIDE=0/1 forces them off/on in both precisions where they apply.
    DBuf<int> st_col;
    DBuf<double> st_val64;
    DBuf<float> st_val32;
    {
        const char *env = getenv("GKSL_ADJ_WIDE");
        const bool on64 = env ? env[0] == '1' : false;
        bool on = env ? env[0] == '1' : f32;
        long long W = 0;
        for (int i = 0; i < c->adj_n; ++i) {
            W += c->adj[i].width;
            if (c->adj[i].ld != c->adj[0].ld) on = false;
        }
        if (c->adj_n > 4 || W < 1 || W > 32) on = false;
        if (on) {
            const long long ld = c->adj[0].ld;
            st_col.alloc((size_t)(W * ld));
            if (on64) st_val64.alloc((size_t)(W * ld));
            if (f32) st_val32.alloc((size_t)(W * ld));
            int off[4];
            long long o = 0;
            for (int i = 0; i < 4; ++i) {
                off[i] = (int)o;
                if (i >= c->adj_n) continue;
                const size_t n = (size_t)(c->adj[i].width * ld);
                GK_CUDA(cudaMemcpyAsync(st_col.p + o * ld, c->adj[i].ell_col.p, sizeof(int) * n,
                                        cudaMemcpyDeviceToDevice, s));
                if (on64)
                    GK_CUDA(cudaMemcpyAsync(st_val64.p + o * ld, c->adj[i].ell_val.p, sizeof(double) * n,
                                            cudaMemcpyDeviceToDevice, s));
                if (f32)
                    GK_CUDA(cudaMemcpyAsync(st_val32.p + o * ld, c->adjf[i].ell_val.p, sizeof(float) * n,
                                            cudaMemcpyDeviceToDevice, s));
                o += c->adj[i].width;
            }
            const int wm = W <= 8 ? 8 : (W <= 16 ? 16 : (W <= 24 ? 24 : 32));
            auto fill = [&](auto &a, const auto *val) {
                a.wm = wm;
                for (int i = 0; i < 4; ++i) a.chwf[i] = i < a.nch ? (float)a.chw[i] : 0.0f;
                a.Ef = (float)a.E;
                a.Af = (float)a.A;
                a.st_col = st_col.p;
                a.st_val = val;
                a.ld_st = ld;
                a.W_st = (int)W;
                for (int i = 0; i < 4; ++i) a.off[i] = off[i];
            };
            if (on64) fill(a64, st_val64.p);
            if (f32) fill(a32, st_val32.p);
        }
    }
    // channels compiled into the kernel: 4 (one dissipator, up to two H0 components), or all
    const int NC = c->adj_n <= 4 ? 4 : kMaxCh;
    const int nslot = 2 * NC;

    // observable weights (dense, zero off the D block)
    DBuf<double> w((size_t)D1), c0(1);
    GK_CUDA(cudaMemsetAsync(w.p, 0, sizeof(double) * D1, s));
    observable_weights(c, o_diag, w.p, c0.p);
    const Basis B(c->N);

    // checkpoints every q steps.  When those of all periods fit in a quarter of the free device
    // memory, the first forward pass keeps them all and no period is run forward a second time
    // before its stage-input pass; otherwise it keeps one per period and each period, when its
    // turn comes, is run forward once more to set the checkpoints of its segments.
    const long long q = std::max(1LL, std::min(S, (long long)std::ceil(std::sqrt((double)S / 4.0))));
    const long long nseg = (S + q - 1) / q;
    size_t free_b = 0, total_b = 0;
    GK_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const bool keep_all = (double)period * nseg * D1 * sizeof(double) <= 0.25 * (double)free_b;
    DBuf<double> v_save((size_t)D1), ckP((size_t)((keep_all ? 1 : period) * D1)),
        seg((size_t)((keep_all ? period : 1) * nseg * D1));
    DBuf<double> lam((size_t)D1), lacc((size_t)D1), obs((size_t)(S + 1));
    DBuf<double> part((size_t)grid * nslot);
    GK_CUDA(cudaMemsetAsync(part.p, 0, sizeof(double) * grid * nslot, s));
    // stage inputs Y1..Y4 of the q steps of one segment, in the working precision; each vector
    // carries the constant 1 at index D (it multiplies the K column)
    const size_t esz = f32 ? sizeof(float) : sizeof(double);
    const long long ytot = 4 * q * D1;
    // two stage-input buffers when they fit in a tenth of the free memory: the forward pass of
    // the next segment (on the context stream) then overlaps the reverse sweep of the current one
    // (on a second stream, with its own step counter); otherwise one buffer and the two alternate
    GK_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const int nbuf = (double)(2 * ytot * esz) <= 0.1 * (double)free_b ? 2 : 1;
    DBuf<char> ybufs[2];
    for (int b = 0; b < nbuf; ++b) {
        ybufs[b].alloc((size_t)ytot * esz);
        k_fill1<<<grid_for(ytot, 256), 256, 0, s>>>(ybufs[b].p, ytot, f32 ? 1 : 0);
        GK_LAUNCH_CHECK();
    }
    DBuf<char> kbA((size_t)D1 * esz), kbB((size_t)D1 * esz);
    DBuf<float> lamf;
    if (f32) lamf.alloc((size_t)D1);
    DBuf<long long> rbase(1);   // step counter of the reverse stream
    a64.base = a32.base = rbase.p;
    auto Yp = [&](int b, int k, long long i) -> void * {
        return ybufs[b].p + (size_t)((k * q + i) * D1) * esz;
    };
    GK_CUDA(cudaMemcpyAsync(v_save.p, c->v.p, sizeof(double) * D1, cudaMemcpyDeviceToDevice, s));

    auto load_state = [&](const double *src) {
        GK_CUDA(cudaMemcpyAsync(c->v.p, src, sizeof(double) * D1, cudaMemcpyDeviceToDevice, s));
        if (f32) to_f32(c->v.p, c->v32.p, D1, s);
    };
    auto save_state = [&](double *dst) {
        GK_CUDA(cudaMemcpyAsync(dst, c->v.p, sizeof(double) * D1, cudaMemcpyDeviceToDevice, s));
    };

    // one reverse step (the four adjoint stages) of local step i of a segment, stage inputs in
    // buffer b, on stream st
    auto reverse_step = [&](long long i, int b, cudaStream_t st) {
        if (f32) {
            to_f32(lam.p, lamf.p, D1, st);
            AdjArgs<float> a = a32;
            a.local = i;
            const float *Y1 = (const float *)Yp(b, 0, i), *Y2 = (const float *)Yp(b, 1, i),
                        *Y3 = (const float *)Yp(b, 2, i), *Y4 = (const float *)Yp(b, 3, i);
            float *ka = (float *)kbA.p, *kb = (float *)kbB.p;
            rev_stages<float>(a, NC, grid, bt_rev, st, lamf.p, Y1, Y2, Y3, Y4, ka, kb, lam.p, lacc.p, w.p,
                              part.p);
        } else {
            AdjArgs<double> a = a64;
            a.local = i;
            const double *Y1 = (const double *)Yp(b, 0, i), *Y2 = (const double *)Yp(b, 1, i),
                         *Y3 = (const double *)Yp(b, 2, i), *Y4 = (const double *)Yp(b, 3, i);
            double *ka = (double *)kbA.p, *kb = (double *)kbB.p;
            rev_stages<double>(a, NC, grid, bt_rev, st, lam.p, Y1, Y2, Y3, Y4, ka, kb, lam.p, lacc.p, w.p,
                               part.p);
        }
        GK_LAUNCH_CHECK();
    };
    auto obs_node = [&](long long local) {
        k_obs_step<<<1, 256, 0, s>>>(w.p, c0.p, B.P2, c->N, c->v.p, c->step_base.p, local, first, S, obs.p);
        GK_LAUNCH_CHECK();
    };
    // graphs of one segment of len steps.  Forward (context stream, from the context state at step
    // *step_base): mode 0 steps only, mode 1 keeping Y1..Y4 in buffer b, mode 2 as 1 with the
    // observable at every grid point (the loss period).  Reverse (mode 3, second stream, from
    // step *rbase): the reverse sweep over buffer b.
    cudaStream_t s2 = nullptr;
    GK_CUDA(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
    struct StreamGuard {
        cudaStream_t st;
        ~StreamGuard() { if (st) cudaStreamDestroy(st); }
    } s2guard{s2};
    ExecSet execs;
    auto segment_graph = [&](long long len, int mode, int b) -> cudaGraphExec_t {
        for (auto &e : execs.v)
            if (e.len == len && e.mode == mode + 4 * b) return e.exec;
        Capture cap(mode == 3 ? s2 : s);
        if (mode == 3) {
            for (long long i = len - 1; i >= 0; --i) reverse_step(i, b, s2);
        } else {
            for (long long i = 0; i < len; ++i) {
                if (mode > 0) {
                    if (f32) GK_CUDA(cudaMemcpyAsync(Yp(b, 0, i), c->v32.p, sizeof(float) * D1, cudaMemcpyDeviceToDevice, s));
                    else GK_CUDA(cudaMemcpyAsync(Yp(b, 0, i), c->v.p, sizeof(double) * D1, cudaMemcpyDeviceToDevice, s));
                }
                if (mode == 2) obs_node(i);
                if (mode > 0) step_into(c, precision, h, i, Yp(b, 1, i), Yp(b, 2, i), Yp(b, 3, i));
                else step_into(c, precision, h, i, nullptr, nullptr, nullptr);
            }
            if (mode == 2) obs_node(len);
        }
        cudaGraphExec_t e = cap.finish();
        execs.v.push_back({len, mode + 4 * b, e});
        return e;
    };
    struct EventPair {
        cudaEvent_t ev[2] = {nullptr, nullptr};
        ~EventPair() {
            for (auto e : ev)
                if (e) cudaEventDestroy(e);
        }
    } evF, evR;   // forward pass into buffer b done / reverse sweep over buffer b done
    for (int b = 0; b < 2; ++b) {
        GK_CUDA(cudaEventCreateWithFlags(&evF.ev[b], cudaEventDisableTiming));
        GK_CUDA(cudaEventCreateWithFlags(&evR.ev[b], cudaEventDisableTiming));
    }

    // 1. forward pass: the checkpoints of every segment (keep_all) or of every period; the end
    // state of the last period is not needed
    load_state(v_save.p);
    if (keep_all) {
        for (long long p = 0; p < period; ++p)
            for (long long j = 0; j < nseg; ++j) {
                save_state(seg.p + (p * nseg + j) * D1);
                if (p + 1 == period && j + 1 == nseg) break;
                set_step_base(c, p * S + j * q);
                GK_CUDA(cudaGraphLaunch(segment_graph(std::min(q, S - j * q), 0, 0), s));
            }
    } else {
        for (long long p = 0; p < period; ++p) {
            save_state(ckP.p + p * D1);
            if (p + 1 < period) advance(c, precision, h, p * S, S);
        }
    }
    // 2. reverse sweep; lam starts as dL/dv at the last grid point.  Segment k (in reverse order)
    // runs forward into buffer k % nbuf on the context stream, once the reverse sweep that last
    // read that buffer has finished, and then backwards on the second stream; the forward pass of
    // segment k + 1 overlaps the reverse sweep of segment k.
    k_fill_scaled<<<grid_for(D1, 256), 256, 0, s>>>(lam.p, w.p, 0.5 / (double)S, D1);
    GK_LAUNCH_CHECK();
    GK_CUDA(cudaEventRecord(evF.ev[0], s));
    GK_CUDA(cudaStreamWaitEvent(s2, evF.ev[0], 0));   // lam, the tables and the buffers are ready
    long long k = 0;
    for (long long p = period - 1; p >= 0; --p) {
        const int mode = (p == period - 1) ? 2 : 1;
        const double *segp = seg.p + (keep_all ? p * nseg * D1 : 0);
        if (!keep_all) {
            load_state(ckP.p + p * D1);
            for (long long j = 0; j < nseg; ++j) {
                save_state(seg.p + j * D1);
                if (j + 1 == nseg) break;   // the last segment starts from this checkpoint
                set_step_base(c, p * S + j * q);
                GK_CUDA(cudaGraphLaunch(segment_graph(q, 0, 0), s));
            }
        }
        for (long long j = nseg - 1; j >= 0; --j, ++k) {
            const long long len = std::min(q, S - j * q);
            const int b = (int)(k % nbuf);
            if (k >= nbuf) GK_CUDA(cudaStreamWaitEvent(s, evR.ev[b], 0));
            load_state(segp + j * D1);
            set_step_base(c, p * S + j * q);
            GK_CUDA(cudaGraphLaunch(segment_graph(len, mode, b), s));
            GK_CUDA(cudaEventRecord(evF.ev[b], s));
            GK_CUDA(cudaStreamWaitEvent(s2, evF.ev[b], 0));
            k_set_step<<<1, 1, 0, s2>>>(rbase.p, p * S + j * q);
            GK_LAUNCH_CHECK();
            GK_CUDA(cudaGraphLaunch(segment_graph(len, 3, b), s2));
            GK_CUDA(cudaEventRecord(evR.ev[b], s2));
        }
    }
    GK_CUDA(cudaStreamSynchronize(s2));
    // 3. loss and gradient, reduced in a fixed order
    std::vector<double> ho((size_t)S + 1), hp((size_t)grid * nslot);
    GK_CUDA(cudaMemcpyAsync(ho.data(), obs.p, sizeof(double) * (S + 1), cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaMemcpyAsync(hp.data(), part.p, sizeof(double) * grid * nslot, cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaStreamSynchronize(s));
    double L = 0.0;
    for (long long m = 0; m <= S; ++m) L += (m == 0 || m == S ? 0.5 / (double)S : 1.0 / (double)S) * ho[m];
    *loss = L;
    auto slot_sum = [&](int k) {
        double g = 0.0;
        for (unsigned b = 0; b < grid; ++b) g += hp[(size_t)b * nslot + k];
        return g;
    };
    for (int k = 0; k < npar; ++k) grad[k] = 0.0;
    for (int i = 0; i < c->adj_n; ++i) grad[gidx[i]] += slot_sum(i);
    for (int q = 0; q < a64.nkp; ++q) grad[kp_gidx[q]] += slot_sum(NC + q);
    // restore the state
    load_state(v_save.p);
    GK_CUDA(cudaStreamSynchronize(s));
}

}  // namespace gk
