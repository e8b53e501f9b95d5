// Classical RK4 on dv/dt = (Q0 + eps(t) Q1) v + K (Sec. IV step 3.1, Eq. 8).
//
// One fused kernel per stage: every row r computes k_r = (Q0E y)_r + (eps_s - E) (Q1 y)_r,
// where Q0E = Q0 + E Q1 carries K as an extra column that multiplies the constant 1 stored
// at index D of every state-sized vector, and immediately applies the stage's update:
//   stage 1: y2 = v + h/2 k1, acc = k1          stage 2: y3 = v + h/2 k2, acc += 2 k2
//   stage 3: y4 = v + h k3,   acc += 2 k3       stage 4: v += h/6 (acc + k4)
// The stage times are t_n, t_n + h/2 (twice), t_n + h with t_n = t0 + n h; the drive values
// eps(t) - E = A sin(omega t) for a whole run are tabulated once per call, so no thread
// evaluates a sine.  Matrix streams are loaded with the evict-first hint (__ldcs) so the
// state-sized vectors stay in L2; the gather of y goes through the read-only path.  Columns come
// from the 32-bit ELL array or, where the variant timer keeps it, from its 16-bit relative copy
// (Hyb::ell_c16), whose escaped rows get threads of their own at the front of the grid.
//
// FP32 bulk form: the same kernels on FP32 values and vectors, with the FP32 increment
// h/6 (acc + k4) added to an FP64 master state every step, and (optionally) one full FP64
// step every `corr_every` steps.
#include <cmath>

#include "internal.cuh"
#include "prim.cuh"
#include "stage.cuh"

namespace gk {

namespace {

constexpr int kThreads = 256;
constexpr int kWarpsPerBlock = kThreads / 32;
constexpr int kGraphSteps = 64;

__global__ void k_eps_table(double t0, double h, double A, double omega, int shape, long long n,
                            double *__restrict__ tab) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double th[3];
    drive_theta(shape, omega, t0 + (double)i * h, h, th);
    tab[3 * i + 0] = A * th[0];
    tab[3 * i + 1] = A * th[1];
    tab[3 * i + 2] = A * th[2];
}

__global__ void k_set_ll(long long *p, long long v) { *p = v; }

template <typename VT>
__device__ inline VT ldcs(const VT *p) { return __ldcs(p); }

// column of a 16-bit ELL entry e of row r whose S/J partner is pr (Hyb::ell_c16)
__device__ inline int c16_col(int e, int r, int pr) { return ((e & 1) ? pr : r) + (e >> 1); }

// column of ELL slot position p of row r: from the 16-bit form (C) or the 32-bit one
template <bool C, typename VT>
__device__ inline int ell_c(const HybView<VT> &H, long long p, long long r, int pr) {
    if constexpr (C) return c16_col(ldcs(H.ell_c16 + p), (int)r, pr);
    else return ldcs(H.ell_col + p);
}

// all W columns of row r; c[0] = -1 for a row handled elsewhere (a long row, or with C a row
// escaped from the 16-bit form)
template <bool C, int W, typename VT>
__device__ inline void ell_cols(const HybView<VT> &H, long long r, int (&c)[W]) {
    if constexpr (C) {
        const int e0 = ldcs(H.ell_c16 + r);
        if (e0 == kC16Esc) {
            c[0] = -1;
            return;
        }
        const int pr = (int)c16_partner(r, H.c16_pairs);
        c[0] = c16_col(e0, (int)r, pr);
#pragma unroll
        for (int j = 1; j < W; ++j) c[j] = ell_c<true>(H, (long long)j * H.ld + r, r, pr);
    } else {
#pragma unroll
        for (int j = 0; j < W; ++j) c[j] = ldcs(H.ell_col + (long long)j * H.ld + r);
    }
}

// sum over the ELL slots of row r (slot 0 already loaded as c0/a0; pr: r's S/J partner for C)
template <typename VT, typename AT, int W, bool C>
__device__ inline AT ell_dot(const HybView<VT> &H, long long r, int pr, int c0, VT a0, const VT *__restrict__ y) {
    AT s = (AT)a0 * (AT)__ldg(y + c0);
    if (W > 0) {
#pragma unroll
        for (int j = 1; j < W; ++j) {
            long long p = (long long)j * H.ld + r;
            s += (AT)ldcs(H.ell_val + p) * (AT)__ldg(y + ell_c<C>(H, p, r, pr));
        }
    } else {
#pragma unroll 4
        for (int j = 1; j < H.width; ++j) {
            long long p = (long long)j * H.ld + r;
            s += (AT)ldcs(H.ell_val + p) * (AT)__ldg(y + ell_c<C>(H, p, r, pr));
        }
    }
    return s;
}

// slot 0 of row r: its column (c0) and, for C, its S/J partner (pr); false for a row handled
// elsewhere (a long row, or with C a row escaped from the 16-bit form)
template <bool C, typename VT>
__device__ inline bool ell_slot0(const HybView<VT> &H, long long r, int &c0, int &pr) {
    pr = 0;
    if constexpr (C) {
        const int e0 = ldcs(H.ell_c16 + r);
        if (e0 == kC16Esc) return false;
        pr = (int)c16_partner(r, H.c16_pairs);
        c0 = c16_col(e0, (int)r, pr);
        return true;
    } else {
        c0 = ldcs(H.ell_col + r);
        return c0 >= 0;
    }
}

template <typename VT, typename AT>
__device__ inline AT ell_dot_full(const HybView<VT> &H, long long r, const VT *__restrict__ y) {
    AT s = AT(0);
#pragma unroll 2
    for (int j = 0; j < H.width; ++j) {
        long long p = (long long)j * H.ld + r;
        s += (AT)ldcs(H.ell_val + p) * (AT)__ldg(y + ldcs(H.ell_col + p));
    }
    return s;
}

// (C y)_i of long row i by one warp: each lane sums its entries e, e + 32, ... in order, eight of
// them in flight at a time (the sums are those of a one-at-a-time loop bit for bit), then a warp
// reduction.  Eight in flight matter where long rows are most of the matrix (a dense L).
template <typename VT, typename AT>
__device__ inline AT tail_dot(const HybView<VT> &H, long long i, int lane, const VT *__restrict__ y) {
    AT s = AT(0);
    const int e1 = H.tail_ptr[i + 1];
    int e = H.tail_ptr[i] + lane;
    for (; e + 224 < e1; e += 256) {
        int cc[8];
        VT vv[8], yy[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            cc[u] = H.tail_col[e + 32 * u];
            vv[u] = ldcs(H.tail_val + e + 32 * u);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) yy[u] = __ldg(y + cc[u]);
#pragma unroll
        for (int u = 0; u < 8; ++u) s += (AT)vv[u] * (AT)yy[u];
    }
    for (; e < e1; e += 32) s += (AT)ldcs(H.tail_val + e) * (AT)__ldg(y + H.tail_col[e]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

struct StepArgs {
    const int *long_rows;
    long long n_long;
    long long D;
    int nb_long;
    const double *eps_tab;
    const long long *base;
    long long local;
    HConst hc;
    const double *q1v;    // Q1 folded into slot 0 (M kernels): its value per row
    const float *q1vf;
    const int *esc_rows;  // rows escaped from the 16-bit column form (C kernels), one thread each
    long long n_esc;
    int nb_esc;           // blocks of escaped rows, after the nb_long blocks of long rows
};

template <typename VT>
__device__ inline const VT *q1_of(const StepArgs &a);
template <>
__device__ inline const double *q1_of<double>(const StepArgs &a) { return a.q1v; }
template <>
__device__ inline const float *q1_of<float>(const StepArgs &a) { return a.q1vf; }

// One ELL row of the stage: k_r from slot 0 (plus the folded Q1 value for M) and the other
// slots, then the stage update; nothing for a row handled elsewhere.
template <int STAGE, int W, typename VT, bool M, bool C>
__device__ inline void ell_row(const HybView<VT> &A0, const HybView<VT> &A1, const StepArgs &a, VT eps, long long r,
                               const VT *__restrict__ y, VT *v, double *v64, VT *__restrict__ yn,
                               VT *__restrict__ acc) {
    int c0, pr;
    if (!ell_slot0<C>(A0, r, c0, pr)) return;
    VT a0 = ldcs(A0.ell_val + r);
    if (M) a0 = fma(eps, ldcs(q1_of<VT>(a) + r), a0);
    VT s0 = ell_dot<VT, VT, W, C>(A0, r, pr, c0, a0, y);
    if (!M) s0 = s0 + eps * ell_dot_full<VT, VT>(A1, r, y);
    epi<STAGE, VT>(r, s0, v, v64, yn, acc, a.hc);
}

// Blocks [nb_long, nb_long + nb_esc) of a C launch: the rows escaped from the 16-bit column form,
// one thread each, through the 32-bit columns.  Returns whether this block is one of them.
template <int STAGE, int W, typename VT, bool M, bool C>
__device__ inline bool esc_rows_part(const HybView<VT> &A0, const HybView<VT> &A1, const StepArgs &a, VT eps,
                                     const VT *__restrict__ y, VT *v, double *v64, VT *yn, VT *acc) {
    if (!C || (int)blockIdx.x >= a.nb_long + a.nb_esc) return false;
    const long long i = (long long)(blockIdx.x - a.nb_long) * kThreads + threadIdx.x;
    if (i < a.n_esc) ell_row<STAGE, W, VT, M, false>(A0, A1, a, eps, a.esc_rows[i], y, v, v64, yn, acc);
    return true;
}

// M: Q1 folded into slot 0 (slot 0 holds q0 + (eps - E) q1, no Q1 ELL is read)
// C: columns from the 16-bit form (Hyb::ell_c16), with M only
template <int STAGE, int W, bool M, bool C>
__global__ void __launch_bounds__(kThreads) k_stage64(HybView<double> A0, HybView<double> A1, StepArgs a,
                                                      const double *__restrict__ y, double *v, double *__restrict__ yn,
                                                      double *__restrict__ acc) {
    __shared__ double s_eps;
    if (threadIdx.x == 0) s_eps = a.eps_tab[3 * (*a.base + a.local) + eps_slot<STAGE>()];
    __syncthreads();
    const double eps = s_eps;
    if ((int)blockIdx.x < a.nb_long) {
        int lane = threadIdx.x & 31;
        long long i = (long long)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
        if (i >= a.n_long) return;
        double s0 = tail_dot<double, double>(A0, i, lane, y);
        double s1 = tail_dot<double, double>(A1, i, lane, y);
        if (lane == 0) epi64<STAGE>(a.long_rows[i], s0 + eps * s1, v, yn, acc, a.hc);
        return;
    }
    if (esc_rows_part<STAGE, W, double, M, C>(A0, A1, a, eps, y, v, nullptr, yn, acc)) return;
    long long r = (long long)(blockIdx.x - a.nb_long - a.nb_esc) * kThreads + threadIdx.x;
    if (r < a.D) ell_row<STAGE, W, double, M, C>(A0, A1, a, eps, r, y, v, nullptr, yn, acc);
}

template <int STAGE, int W, bool M, bool C>
__global__ void __launch_bounds__(kThreads) k_stage32(HybView<float> A0, HybView<float> A1, StepArgs a,
                                                      const float *__restrict__ y, float *v32, double *v64,
                                                      float *__restrict__ yn, float *__restrict__ acc) {
    __shared__ float s_eps;
    if (threadIdx.x == 0) s_eps = (float)a.eps_tab[3 * (*a.base + a.local) + eps_slot<STAGE>()];
    __syncthreads();
    const float eps = s_eps;
    if ((int)blockIdx.x < a.nb_long) {
        int lane = threadIdx.x & 31;
        long long i = (long long)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
        if (i >= a.n_long) return;
        float s0 = tail_dot<float, float>(A0, i, lane, y);
        float s1 = tail_dot<float, float>(A1, i, lane, y);
        if (lane == 0) epi32<STAGE>(a.long_rows[i], s0 + eps * s1, v32, v64, yn, acc, a.hc);
        return;
    }
    if (esc_rows_part<STAGE, W, float, M, C>(A0, A1, a, eps, y, v32, v64, yn, acc)) return;
    long long r = (long long)(blockIdx.x - a.nb_long - a.nb_esc) * kThreads + threadIdx.x;
    if (r < a.D) ell_row<STAGE, W, float, M, C>(A0, A1, a, eps, r, y, v32, v64, yn, acc);
}

// ---- variants of the ELL part (same arithmetic, same summation order per row)

template <int STAGE, typename VT>
__device__ inline bool long_rows_part(const HybView<VT> &A0, const HybView<VT> &A1, const StepArgs &a, VT eps,
                                      const VT *__restrict__ y, VT *v, double *v64, VT *yn, VT *acc) {
    if ((int)blockIdx.x >= a.nb_long) return false;
    int lane = threadIdx.x & 31;
    long long i = (long long)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (i < a.n_long) {
        VT s0 = tail_dot<VT, VT>(A0, i, lane, y);
        VT s1 = tail_dot<VT, VT>(A1, i, lane, y);
        if (lane == 0) epi<STAGE, VT>(a.long_rows[i], s0 + eps * s1, v, v64, yn, acc, a.hc);
    }
    return true;
}

// Variant 1: the whole ELL row is loaded into registers (all columns, then all values, then
// all gathers) before the products, with a larger register budget for the loads in flight.
template <int STAGE, int W, typename VT, bool M, bool C>
__global__ void __launch_bounds__(kThreads, 3) k_stage_pf(HybView<VT> A0, HybView<VT> A1, StepArgs a,
                                                          const VT *__restrict__ y, VT *v, double *v64,
                                                          VT *__restrict__ yn, VT *__restrict__ acc) {
    __shared__ VT s_eps;
    if (threadIdx.x == 0) s_eps = (VT)a.eps_tab[3 * (*a.base + a.local) + eps_slot<STAGE>()];
    __syncthreads();
    const VT eps = s_eps;
    if (long_rows_part<STAGE, VT>(A0, A1, a, eps, y, v, v64, yn, acc)) return;
    if (esc_rows_part<STAGE, W, VT, M, C>(A0, A1, a, eps, y, v, v64, yn, acc)) return;
    long long r = (long long)(blockIdx.x - a.nb_long - a.nb_esc) * kThreads + threadIdx.x;
    if (r >= a.D) return;
    int c[W];
    VT x[W], m[W];
    ell_cols<C, W>(A0, r, c);
    if (c[0] < 0) return;
#pragma unroll
    for (int j = 0; j < W; ++j) m[j] = ldcs(A0.ell_val + (long long)j * A0.ld + r);
    if (M) m[0] = eps * ldcs(q1_of<VT>(a) + r) + m[0];
#pragma unroll
    for (int j = 0; j < W; ++j) x[j] = __ldg(y + c[j]);
    VT s0 = m[0] * x[0];
#pragma unroll
    for (int j = 1; j < W; ++j) s0 += m[j] * x[j];
    if (!M) s0 = s0 + eps * ell_dot_full<VT, VT>(A1, r, y);
    epi<STAGE, VT>(r, s0, v, v64, yn, acc, a.hc);
}

// Variant 3: variant 1 with programmatic dependent launch.  Each block lets the next stage's
// launch begin as soon as it starts, loads its rows' matrix columns and values (no stage writes
// them), and only then waits for the previous stage to complete (griddepcontrol.wait) before it
// reads the drive table, the step base or a state vector, or writes anything.  The next stage's
// blocks thus take the SMs the previous stage frees in its last wave and stream their matrix
// slots meanwhile.
template <int STAGE, int W, typename VT, bool M, bool C>
__global__ void __launch_bounds__(kThreads, 3) k_stage_pdl(HybView<VT> A0, HybView<VT> A1, StepArgs a,
                                                           const VT *__restrict__ y, VT *v, double *v64,
                                                           VT *__restrict__ yn, VT *__restrict__ acc) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if ((int)blockIdx.x < a.nb_long) {
        asm volatile("griddepcontrol.wait;" ::: "memory");
        const VT eps = (VT)a.eps_tab[3 * (*a.base + a.local) + eps_slot<STAGE>()];
        const int lane = threadIdx.x & 31;
        const long long i = (long long)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
        if (i < a.n_long) {
            VT s0 = tail_dot<VT, VT>(A0, i, lane, y);
            VT s1 = tail_dot<VT, VT>(A1, i, lane, y);
            if (lane == 0) epi<STAGE, VT>(a.long_rows[i], s0 + eps * s1, v, v64, yn, acc, a.hc);
        }
        return;
    }
    if (C && (int)blockIdx.x < a.nb_long + a.nb_esc) {
        asm volatile("griddepcontrol.wait;" ::: "memory");
        const VT eps = (VT)a.eps_tab[3 * (*a.base + a.local) + eps_slot<STAGE>()];
        esc_rows_part<STAGE, W, VT, M, C>(A0, A1, a, eps, y, v, v64, yn, acc);
        return;
    }
    const long long r = (long long)(blockIdx.x - a.nb_long - a.nb_esc) * kThreads + threadIdx.x;
    const bool in = r < a.D;
    int c[W];
    VT m[W];
    VT q = VT(0);
    if (in) {
        ell_cols<C, W>(A0, r, c);
#pragma unroll
        for (int j = 0; j < W; ++j) m[j] = ldcs(A0.ell_val + (long long)j * A0.ld + r);
        if (M) q = ldcs(q1_of<VT>(a) + r);
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (!in || c[0] < 0) return;   // past the end, or a row handled above (long or escaped)
    const VT eps = (VT)a.eps_tab[3 * (*a.base + a.local) + eps_slot<STAGE>()];
    if (M) m[0] = eps * q + m[0];
    VT x[W];
#pragma unroll
    for (int j = 0; j < W; ++j) x[j] = __ldg(y + c[j]);
    VT s0 = m[0] * x[0];
#pragma unroll
    for (int j = 1; j < W; ++j) s0 += m[j] * x[j];
    if (!M) s0 = s0 + eps * ell_dot_full<VT, VT>(A1, r, y);
    epi<STAGE, VT>(r, s0, v, v64, yn, acc, a.hc);
}

// Variant 2: two consecutive rows per thread with 2-wide vector loads of the slot-major ELL
// arrays (ld is a multiple of 32 and r is even, so every vector access is aligned).
template <int STAGE, int W, typename VT, bool M>
__global__ void __launch_bounds__(kThreads) k_stage_r2(HybView<VT> A0, HybView<VT> A1, StepArgs a,
                                                       const VT *__restrict__ y, VT *v, double *v64,
                                                       VT *__restrict__ yn, VT *__restrict__ acc) {
    using V2 = typename Vec2<VT>::T;
    __shared__ VT s_eps;
    if (threadIdx.x == 0) s_eps = (VT)a.eps_tab[3 * (*a.base + a.local) + eps_slot<STAGE>()];
    __syncthreads();
    const VT eps = s_eps;
    if (long_rows_part<STAGE, VT>(A0, A1, a, eps, y, v, v64, yn, acc)) return;
    long long r = ((long long)(blockIdx.x - a.nb_long) * kThreads + threadIdx.x) * 2;
    if (r >= a.D) return;
    const int w0 = W > 0 ? W : A0.width;
    int2 c = ldcs((const int2 *)(A0.ell_col + r));
    V2 m = ldcs((const V2 *)(A0.ell_val + r));
    if (M) {
        const V2 q = ldcs((const V2 *)(q1_of<VT>(a) + r));
        m.x = eps * q.x + m.x;
        m.y = eps * q.y + m.y;
    }
    const bool live0 = c.x >= 0, live1 = (r + 1 < a.D) && c.y >= 0;
    VT sa = m.x * __ldg(y + (c.x < 0 ? 0 : c.x));
    VT sb = m.y * __ldg(y + (c.y < 0 ? 0 : c.y));
#pragma unroll
    for (int j = 1; j < (W > 0 ? W : 64); ++j) {
        if (W == 0 && j >= w0) break;
        long long p = (long long)j * A0.ld + r;
        int2 cj = ldcs((const int2 *)(A0.ell_col + p));
        V2 mj = ldcs((const V2 *)(A0.ell_val + p));
        sa += mj.x * __ldg(y + cj.x);
        sb += mj.y * __ldg(y + cj.y);
    }
    if (!M) {
        VT ta = VT(0), tb = VT(0);
        for (int j = 0; j < A1.width; ++j) {
            long long p = (long long)j * A1.ld + r;
            int2 cj = ldcs((const int2 *)(A1.ell_col + p));
            V2 mj = ldcs((const V2 *)(A1.ell_val + p));
            ta += mj.x * __ldg(y + cj.x);
            tb += mj.y * __ldg(y + cj.y);
        }
        sa = sa + eps * ta;
        sb = sb + eps * tb;
    }
    if (live0) epi<STAGE, VT>(r, sa, v, v64, yn, acc, a.hc);
    if (live1) epi<STAGE, VT>(r + 1, sb, v, v64, yn, acc, a.hc);
}

__global__ void k_to_f32(const double *__restrict__ v, float *__restrict__ o, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) o[i] = (float)v[i];
}

__global__ void k_fill(double *p, long long n, double x) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = x;
}

__global__ void k_fill_f(float *p, long long n, float x) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = x;
}

__global__ void k_check_finite(const double *__restrict__ v, long long n, int *__restrict__ flag) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !isfinite(v[i])) atomicOr(flag, 1);
}

struct Launch {
    unsigned grid;
    StepArgs a;
};

Launch make_launch(gksl_ctx *c, const Hyb<double> &h0, double h, const double *tab, long long local) {
    Launch L;
    L.a.long_rows = h0.long_rows.p;
    L.a.n_long = h0.n_long;
    L.a.D = c->D;
    L.a.nb_long = (int)((h0.n_long + kWarpsPerBlock - 1) / kWarpsPerBlock);
    L.a.eps_tab = tab;
    L.a.base = c->step_base.p;
    L.a.local = local;
    L.a.hc.h = h;
    L.a.hc.h2 = 0.5 * h;
    L.a.hc.h6 = h / 6.0;
    L.a.hc.hf = (float)h;
    L.a.hc.h2f = 0.5f * (float)h;
    L.a.hc.h6f = (float)(h / 6.0);
    L.a.q1v = c->q1_folded ? c->q1v.p : nullptr;
    L.a.q1vf = c->q1_folded ? c->q1vf.p : nullptr;
    L.a.esc_rows = nullptr;
    L.a.n_esc = 0;
    L.a.nb_esc = 0;
    L.grid = (unsigned)(L.a.nb_long + (c->D + kThreads - 1) / kThreads);
    return L;
}

// One RK4 step; the stage inputs go to y2, y3, y4 (y4 may alias y2: the default buffers are
// yA, yB, yA).
// launch with programmatic stream serialization (the kernel waits on its predecessor itself)
template <typename... P, typename... A>
void launch_pdl(void (*kernel)(P...), unsigned grid, cudaStream_t s, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    GK_CUDA(cudaLaunchKernelEx(&cfg, kernel, args...));
}

template <int W, bool M, bool C>
void step64_w(gksl_ctx *c, const Launch &L, double *y2, double *y3, double *y4) {
    auto A0 = view(c->hyb0), A1 = view(c->hyb1);
    cudaStream_t s = c->stream;
    k_stage64<1, W, M, C><<<L.grid, kThreads, 0, s>>>(A0, A1, L.a, c->v.p, c->v.p, y2, c->acc.p);
    k_stage64<2, W, M, C><<<L.grid, kThreads, 0, s>>>(A0, A1, L.a, y2, c->v.p, y3, c->acc.p);
    k_stage64<3, W, M, C><<<L.grid, kThreads, 0, s>>>(A0, A1, L.a, y3, c->v.p, y4, c->acc.p);
    k_stage64<4, W, M, C><<<L.grid, kThreads, 0, s>>>(A0, A1, L.a, y4, c->v.p, nullptr, c->acc.p);
}

template <int W, bool M, bool C>
void step32_w(gksl_ctx *c, const Launch &L, float *y2, float *y3, float *y4) {
    auto A0 = view(c->hyb0f), A1 = view(c->hyb1f);
    cudaStream_t s = c->stream;
    k_stage32<1, W, M, C><<<L.grid, kThreads, 0, s>>>(A0, A1, L.a, c->v32.p, c->v32.p, c->v.p, y2, c->acc32.p);
    k_stage32<2, W, M, C><<<L.grid, kThreads, 0, s>>>(A0, A1, L.a, y2, c->v32.p, c->v.p, y3, c->acc32.p);
    k_stage32<3, W, M, C><<<L.grid, kThreads, 0, s>>>(A0, A1, L.a, y3, c->v32.p, c->v.p, y4, c->acc32.p);
    k_stage32<4, W, M, C><<<L.grid, kThreads, 0, s>>>(A0, A1, L.a, y4, c->v32.p, c->v.p, nullptr, c->acc32.p);
}

// variants 1, 2 and 3 on either precision (variant 2 reads 32-bit columns only)
template <int VAR, int W, typename VT, bool M, bool C>
void step_var(gksl_ctx *c, const Launch &L0, const Hyb<VT> &h0, const Hyb<VT> &h1, VT *v, double *v64, VT *y2, VT *y3,
              VT *y4, VT *acc) {
    auto A0 = view(h0), A1 = view(h1);
    cudaStream_t s = c->stream;
    Launch L = L0;
    if (VAR == 2) L.grid = (unsigned)(L.a.nb_long + (c->D + 2 * kThreads - 1) / (2 * kThreads));
    if constexpr (VAR == 3) {
        launch_pdl(k_stage_pdl<1, W, VT, M, C>, L.grid, s, A0, A1, L.a, (const VT *)v, v, v64, y2, acc);
        launch_pdl(k_stage_pdl<2, W, VT, M, C>, L.grid, s, A0, A1, L.a, (const VT *)y2, v, v64, y3, acc);
        launch_pdl(k_stage_pdl<3, W, VT, M, C>, L.grid, s, A0, A1, L.a, (const VT *)y3, v, v64, y4, acc);
        launch_pdl(k_stage_pdl<4, W, VT, M, C>, L.grid, s, A0, A1, L.a, (const VT *)y4, v, v64, (VT *)nullptr,
                   acc);
    } else if constexpr (VAR == 1) {
        k_stage_pf<1, W, VT, M, C><<<L.grid, kThreads, 0, s>>>(A0, A1, L.a, v, v, v64, y2, acc);
        k_stage_pf<2, W, VT, M, C><<<L.grid, kThreads, 0, s>>>(A0, A1, L.a, y2, v, v64, y3, acc);
        k_stage_pf<3, W, VT, M, C><<<L.grid, kThreads, 0, s>>>(A0, A1, L.a, y3, v, v64, y4, acc);
        k_stage_pf<4, W, VT, M, C><<<L.grid, kThreads, 0, s>>>(A0, A1, L.a, y4, v, v64, nullptr, acc);
    } else {
        k_stage_r2<1, W, VT, M><<<L.grid, kThreads, 0, s>>>(A0, A1, L.a, v, v, v64, y2, acc);
        k_stage_r2<2, W, VT, M><<<L.grid, kThreads, 0, s>>>(A0, A1, L.a, y2, v, v64, y3, acc);
        k_stage_r2<3, W, VT, M><<<L.grid, kThreads, 0, s>>>(A0, A1, L.a, y3, v, v64, y4, acc);
        k_stage_r2<4, W, VT, M><<<L.grid, kThreads, 0, s>>>(A0, A1, L.a, y4, v, v64, nullptr, acc);
    }
}

// CSR-form step with explicit stage-input buffers (null: the context's yA, yB, yA)
template <bool M, bool C>
void launch_step_csr_t(gksl_ctx *c, int precision, double h, const double *tab, long long local, void *Y2, void *Y3,
                       void *Y4) {
    Launch L = make_launch(c, c->hyb0, h, tab, local);
    int W = c->hyb0.width;
    int var = c->rk4_var[precision == 64 ? 0 : 1];
    if ((var == 1 || var == 3) && W != 18) var = 0;   // the register-prefetch variants exist for 18 slots only
    if (C && var != 2) {   // blocks for the rows escaped from the 16-bit columns
        const long long n_esc = precision == 64 ? c->hyb0.n_esc : c->hyb0f.n_esc;
        L.a.esc_rows = precision == 64 ? c->hyb0.c16_esc.p : c->hyb0f.c16_esc.p;
        L.a.n_esc = n_esc;
        L.a.nb_esc = (int)((n_esc + kThreads - 1) / kThreads);
        L.grid += (unsigned)L.a.nb_esc;
    }
    if (precision == 64) {
        double *y2 = Y2 ? (double *)Y2 : c->yA.p, *y3 = Y3 ? (double *)Y3 : c->yB.p, *y4 = Y4 ? (double *)Y4 : c->yA.p;
        const Hyb<double> &h0 = c->hyb0, &h1 = c->hyb1;
        double *v = c->v.p, *acc = c->acc.p;
        if (var == 3) step_var<3, 18, double, M, C>(c, L, h0, h1, v, nullptr, y2, y3, y4, acc);
        else if (var == 1) step_var<1, 18, double, M, C>(c, L, h0, h1, v, nullptr, y2, y3, y4, acc);
        else if (var == 2 && W == 18) step_var<2, 18, double, M, false>(c, L, h0, h1, v, nullptr, y2, y3, y4, acc);
        else if (var == 2) step_var<2, 0, double, M, false>(c, L, h0, h1, v, nullptr, y2, y3, y4, acc);
        else if (W == 18) step64_w<18, M, C>(c, L, y2, y3, y4);
        else step64_w<0, M, C>(c, L, y2, y3, y4);
    } else {
        float *y2 = Y2 ? (float *)Y2 : c->yA32.p, *y3 = Y3 ? (float *)Y3 : c->yB32.p, *y4 = Y4 ? (float *)Y4 : c->yA32.p;
        const Hyb<float> &h0 = c->hyb0f, &h1 = c->hyb1f;
        float *v = c->v32.p, *acc = c->acc32.p;
        double *v64 = c->v.p;
        if (var == 3) step_var<3, 18, float, M, C>(c, L, h0, h1, v, v64, y2, y3, y4, acc);
        else if (var == 1) step_var<1, 18, float, M, C>(c, L, h0, h1, v, v64, y2, y3, y4, acc);
        else if (var == 2 && W == 18) step_var<2, 18, float, M, false>(c, L, h0, h1, v, v64, y2, y3, y4, acc);
        else if (var == 2) step_var<2, 0, float, M, false>(c, L, h0, h1, v, v64, y2, y3, y4, acc);
        else if (W == 18) step32_w<18, M, C>(c, L, y2, y3, y4);
        else step32_w<0, M, C>(c, L, y2, y3, y4);
    }
    GK_LAUNCH_CHECK();
}

void launch_step_csr(gksl_ctx *c, int precision, double h, const double *tab, long long local, void *Y2, void *Y3,
                     void *Y4) {
    const int pi = precision == 64 ? 0 : 1;
    const bool cmp = (pi == 0 ? c->hyb0.ell_c16.p : c->hyb0f.ell_c16.p) != nullptr && c->rk4_c16[pi];
    if (c->q1_folded && cmp) launch_step_csr_t<true, true>(c, precision, h, tab, local, Y2, Y3, Y4);
    else if (c->q1_folded) launch_step_csr_t<true, false>(c, precision, h, tab, local, Y2, Y3, Y4);
    else launch_step_csr_t<false, false>(c, precision, h, tab, local, Y2, Y3, Y4);
}

void launch_step(gksl_ctx *c, int precision, double h, const double *tab, long long local) {
    if (c->asm_flags & GKSL_ASM_MATRIX_FREE) {
        mf_step(c, precision, h, tab, local);
        return;
    }
    launch_step_csr(c, precision, h, tab, local, nullptr, nullptr, nullptr);
}

cudaGraphExec_t graph_for(gksl_ctx *c, long long steps, int precision, double h, const double *tab);

// Time the stage-kernel variants on this context's matrix, each with 32-bit and (where built)
// 16-bit columns, as a CUDA graph of 8 steps as propagation replays them (from a saved copy of
// the state, which is restored afterwards; best of two timed replays), and keep the fastest; the
// 16-bit columns only when they beat the best 32-bit variant by 2 % (where the FP64 pipe, not
// the matrix stream, bounds the stage the two tie, and the 32-bit form has no escaped rows).
// Systems below D = 1024 keep variant 0 (16-bit columns where built).  GKSL_RK4_VARIANT=0..3
// forces a variant, GKSL_RK4_COLUMNS=32 the 32-bit columns.
void tune_variant(gksl_ctx *c, int precision, double h, const double *tab) {
    constexpr int kSteps = 8;
    int pi = precision == 64 ? 0 : 1;
    if (c->rk4_tuned[pi]) return;
    c->rk4_tuned[pi] = true;
    if (c->asm_flags & GKSL_ASM_MATRIX_FREE) return;   // one matrix-free kernel per stage
    const char *envc = getenv("GKSL_RK4_COLUMNS");
    const bool have16 = (pi == 0 ? c->hyb0.ell_c16.p : c->hyb0f.ell_c16.p) != nullptr &&
                        !(envc && envc[0] == '3' && envc[1] == '2');
    c->rk4_c16[pi] = have16;
    for (int var = 0; var < 4; ++var) c->rk4_var_us[pi][var] = c->rk4_var_us_c16[pi][var] = 0.0;
    const char *env = getenv("GKSL_RK4_VARIANT");
    if (env && env[0] >= '0' && env[0] <= '3') {
        c->rk4_var[pi] = env[0] - '0';
        return;
    }
    c->rk4_var[pi] = 0;
    if (c->D < 1024) return;
    long long D1 = c->D + 1;
    DBuf<double> save((size_t)D1);
    GK_CUDA(cudaMemcpyAsync(save.p, c->v.p, sizeof(double) * D1, cudaMemcpyDeviceToDevice, c->stream));
    cudaEvent_t e0, e1;
    GK_CUDA(cudaEventCreate(&e0));
    GK_CUDA(cudaEventCreate(&e1));
    float best[2] = {1e30f, 1e30f};   // [column form]: 32-bit, 16-bit
    int best_v[2] = {0, 0};
    for (int k = 0; k < 8; ++k) {
        const int var = k >> 1;
        const bool c16 = k & 1;
        if ((var == 1 || var == 3) && c->hyb0.width != 18) continue;   // 18-slot layouts only
        if (c16 && (!have16 || var == 2)) continue;                     // variant 2 reads 32-bit columns
        c->rk4_var[pi] = var;
        c->rk4_c16[pi] = c16;
        cudaGraphExec_t g = graph_for(c, kSteps, precision, h, tab);
        k_set_ll<<<1, 1, 0, c->stream>>>(c->step_base.p, 0);
        GK_LAUNCH_CHECK();
        GK_CUDA(cudaGraphLaunch(g, c->stream));   // warm-up
        float ms = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            k_set_ll<<<1, 1, 0, c->stream>>>(c->step_base.p, 0);
            GK_LAUNCH_CHECK();
            GK_CUDA(cudaEventRecord(e0, c->stream));
            GK_CUDA(cudaGraphLaunch(g, c->stream));
            GK_CUDA(cudaEventRecord(e1, c->stream));
            GK_CUDA(cudaEventSynchronize(e1));
            float t = 0;
            GK_CUDA(cudaEventElapsedTime(&t, e0, e1));
            ms = std::min(ms, t);
        }
        (c16 ? c->rk4_var_us_c16 : c->rk4_var_us)[pi][var] = 1000.0 * ms / kSteps;
        if (ms < best[c16]) {
            best[c16] = ms;
            best_v[c16] = var;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const bool use16 = best[1] < 0.98f * best[0];
    c->rk4_var[pi] = best_v[use16];
    c->rk4_c16[pi] = use16;
    GK_CUDA(cudaMemcpyAsync(c->v.p, save.p, sizeof(double) * D1, cudaMemcpyDeviceToDevice, c->stream));
    if (precision == 32) {
        k_to_f32<<<grid_for(D1, 256), 256, 0, c->stream>>>(c->v.p, c->v32.p, D1);
        GK_LAUNCH_CHECK();
    }
    GK_CUDA(cudaStreamSynchronize(c->stream));
}

// one CUDA graph per (chunk length, precision, h); replayed with the step base set before
cudaGraphExec_t graph_for(gksl_ctx *c, long long steps, int precision, double h, const double *tab) {
    const int pi = precision == 64 ? 0 : 1;
    const int var = c->rk4_var[pi] + (c->rk4_c16[pi] ? 4 : 0);
    for (auto &g : c->graphs)
        if (g.steps == steps && g.precision == precision && g.h == h && g.variant == var) return g.exec;
    cudaGraph_t graph;
    const bool mf = (c->asm_flags & GKSL_ASM_MATRIX_FREE) != 0;
    GK_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    if (mf) mf_prep(c, precision);
    for (long long i = 0; i < steps; ++i) launch_step(c, precision, h, tab, i);
    if (mf) mf_post(c, precision);
    GK_CUDA(cudaStreamEndCapture(c->stream, &graph));
    cudaGraphExec_t exec;
    GK_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    GK_CUDA(cudaGraphDestroy(graph));
    c->graphs.push_back({steps, precision, h, exec, var});
    return exec;
}

void run_steps(gksl_ctx *c, int precision, double h, const double *tab, long long first, long long count) {
    if (rk4_block_applies(c, precision)) {   // a small system: the whole chunk in one launch
        rk4_block_run(c, precision, h, tab, first, count);
        return;
    }
    long long n = first, end = first + count;
    while (end - n >= kGraphSteps) {
        k_set_ll<<<1, 1, 0, c->stream>>>(c->step_base.p, n);
        GK_LAUNCH_CHECK();
        GK_CUDA(cudaGraphLaunch(graph_for(c, kGraphSteps, precision, h, tab), c->stream));
        n += kGraphSteps;
    }
    if (n < end) {
        k_set_ll<<<1, 1, 0, c->stream>>>(c->step_base.p, n);
        GK_LAUNCH_CHECK();
        const bool mf = (c->asm_flags & GKSL_ASM_MATRIX_FREE) != 0;
        if (mf) mf_prep(c, precision);
        for (long long i = 0; n + i < end; ++i) launch_step(c, precision, h, tab, i);
        if (mf) mf_post(c, precision);
        n = end;
    }
}

}  // namespace

void tune_stage_variant(gksl_ctx *c, int precision, double h) { tune_variant(c, precision, h, c->eps_tab.p); }

void clear_graphs(gksl_ctx *c) {
    for (auto &g : c->graphs) cudaGraphExecDestroy(g.exec);
    c->graphs.clear();
}

void ensure_work(gksl_ctx *c, bool fp32) {
    long long n = c->D + 1;
    if (c->yA.n < (size_t)n) {
        c->yA.alloc((size_t)n);
        c->yB.alloc((size_t)n);
        c->acc.alloc((size_t)n);
        k_fill<<<grid_for(n, 256), 256, 0, c->stream>>>(c->yA.p, n, 1.0);
        k_fill<<<grid_for(n, 256), 256, 0, c->stream>>>(c->yB.p, n, 1.0);
        k_fill<<<grid_for(n, 256), 256, 0, c->stream>>>(c->acc.p, n, 0.0);
        GK_LAUNCH_CHECK();
        clear_graphs(c);
    }
    if (fp32 && c->v32.n < (size_t)n) {
        c->v32.alloc((size_t)n);
        c->yA32.alloc((size_t)n);
        c->yB32.alloc((size_t)n);
        c->acc32.alloc((size_t)n);
        k_fill_f<<<grid_for(n, 256), 256, 0, c->stream>>>(c->yA32.p, n, 1.0f);
        k_fill_f<<<grid_for(n, 256), 256, 0, c->stream>>>(c->yB32.p, n, 1.0f);
        k_fill_f<<<grid_for(n, 256), 256, 0, c->stream>>>(c->acc32.p, n, 0.0f);
        GK_LAUNCH_CHECK();
        clear_graphs(c);
    }
    if (c->step_base.n == 0) c->step_base.alloc(1);
    if (c->flag.n == 0) c->flag.alloc(1);
}

bool state_finite(gksl_ctx *c) {
    GK_CUDA(cudaMemsetAsync(c->flag.p, 0, sizeof(int), c->stream));
    k_check_finite<<<grid_for(c->D, 256), 256, 0, c->stream>>>(c->v.p, c->D, c->flag.p);
    GK_LAUNCH_CHECK();
    int f = 0;
    GK_CUDA(cudaMemcpyAsync(&f, c->flag.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    GK_CUDA(cudaStreamSynchronize(c->stream));
    return f == 0;
}

void fill_eps_table(gksl_ctx *c, double t0, double h, long long n) {
    size_t need = (size_t)(3 * (n > 0 ? n : 1));
    if (c->eps_tab.n < need) {
        clear_graphs(c);   // graphs bake the table pointer
        c->eps_tab.alloc(need);
    }
    if (n > 0) {
        k_eps_table<<<grid_for(n, 256), 256, 0, c->stream>>>(t0, h, c->A, c->omega, c->drive_shape, n,
                                                              c->eps_tab.p);
        GK_LAUNCH_CHECK();
    }
}

void check_drive_grid(const gksl_ctx *c, long long spp, double h) {
    if (c->drive_shape != GKSL_DRIVE_SQUARE) return;
    GK_REQUIRE(spp % 2 == 0, GKSL_ERR_ARG, "the square drive needs an even steps_per_period (jumps at T/2)");
    double k = c->t / h;
    GK_REQUIRE(std::fabs(k - std::nearbyint(k)) <= 1e-6 * std::max(1.0, std::fabs(k)), GKSL_ERR_ARG,
               "the square drive needs the current time on the step grid");
}

void advance(gksl_ctx *c, int precision, double h, long long first, long long count) {
    run_steps(c, precision, h, c->eps_tab.p, first, count);
}

void to_f32(const double *v, float *o, long long n, cudaStream_t s) {
    k_to_f32<<<grid_for(n, 256), 256, 0, s>>>(v, o, n);
    GK_LAUNCH_CHECK();
}

void step_into(gksl_ctx *c, int precision, double h, long long local, void *Y2, void *Y3, void *Y4) {
    GK_REQUIRE(!(c->asm_flags & GKSL_ASM_MATRIX_FREE), GKSL_ERR_STATE, "stage inputs need the CSR form");
    launch_step_csr(c, precision, h, c->eps_tab.p, local, Y2, Y3, Y4);
}

void set_step_base(gksl_ctx *c, long long g) {
    k_set_ll<<<1, 1, 0, c->stream>>>(c->step_base.p, g);
    GK_LAUNCH_CHECK();
}

void fill_theta_table(gksl_ctx *c, double t0, double h, long long n, double *tab) {
    if (n > 0) {
        k_eps_table<<<grid_for(n, 256), 256, 0, c->stream>>>(t0, h, 1.0, c->omega, c->drive_shape, n, tab);
        GK_LAUNCH_CHECK();
    }
}

void propagate(gksl_ctx *c, long long spp, long long n_steps, int precision, long long corr_every,
               long long emit_every, double *v_out, bool out_on_device) {
    GK_REQUIRE(c->assembled, GKSL_ERR_STATE, "gksl_assemble must be called before gksl_propagate");
    GK_REQUIRE(c->state_set, GKSL_ERR_STATE, "no state: call gksl_set_rho0 or gksl_set_state first");
    GK_REQUIRE(precision == 64 || precision == 32, GKSL_ERR_ARG, "precision must be 64 or 32");
    GK_REQUIRE(spp > 0 && n_steps >= 0, GKSL_ERR_ARG, "steps_per_period must be > 0 and n_steps >= 0");
    if (precision == 32)
        GK_REQUIRE(c->asm_flags & GKSL_ASM_FP32, GKSL_ERR_STATE, "precision 32 needs gksl_assemble with GKSL_ASM_FP32");
    ensure_work(c, precision == 32);
    const double T = 2.0 * M_PI / c->omega;
    const double h = T / (double)spp;
    check_drive_grid(c, spp, h);
    fill_eps_table(c, c->t, h, std::max(n_steps, 8LL));   // the variant timing below uses 8 steps
    DBuf<double> &tab = c->eps_tab;
    if (precision == 32) {
        k_to_f32<<<grid_for(c->D + 1, 256), 256, 0, c->stream>>>(c->v.p, c->v32.p, c->D + 1);
        GK_LAUNCH_CHECK();
    }
    if (n_steps > 0) tune_variant(c, precision, h, tab.p);
    long long n = 0, emitted = 0;
    while (n < n_steps) {
        long long stop = n_steps;
        if (emit_every > 0) stop = std::min(stop, (n / emit_every + 1) * emit_every);
        long long corr_step = -1;   // 0-based index of the next FP64 step of the FP32 form
        if (precision == 32 && corr_every > 0) corr_step = (n / corr_every + 1) * corr_every - 1;
        if (corr_step >= 0 && corr_step < stop) {
            if (corr_step > n) run_steps(c, 32, h, tab.p, n, corr_step - n);
            run_steps(c, 64, h, tab.p, corr_step, 1);
            k_to_f32<<<grid_for(c->D + 1, 256), 256, 0, c->stream>>>(c->v.p, c->v32.p, c->D + 1);
            GK_LAUNCH_CHECK();
            n = corr_step + 1;
        } else {
            run_steps(c, precision, h, tab.p, n, stop - n);
            n = stop;
        }
        if (emit_every > 0 && n % emit_every == 0 && v_out) {
            double *dst = v_out + emitted * c->D;
            GK_CUDA(cudaMemcpyAsync(dst, c->v.p, sizeof(double) * c->D,
                                    out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
            ++emitted;
        }
    }
    GK_CUDA(cudaStreamSynchronize(c->stream));
    c->t = c->t + (double)n_steps * h;
    GK_REQUIRE(state_finite(c), GKSL_ERR_DIVERGED, "state became non-finite during propagation");
}

}  // namespace gk
