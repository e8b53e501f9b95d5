// RK4 propagation of a small system by one thread block (Sec. IV step 3.1, as rk4.cu).
//
// For small systems a stage of the fused stage kernels is too short to fill the GPU: each of the
// four launches of an RK4 step costs a few microseconds of launch and drain, whatever the size
// (about 15 us per step from N = 10 to N = 50 with CUDA graphs).  Here one block runs a whole
// chunk of steps in one launch, used up to D + 1 = 256 rows in FP64 and 576 in FP32, where it
// measured faster.  The state-sized vectors (v, the two stage-input buffers and acc,
// and in the FP32 form the FP64 master state) live in shared memory; the matrix streams through
// L1 from the same hybrid format; a block barrier separates the stages.  Each row is summed as
// in the stage kernels (slot 0 with the folded Q1 value, then the other slots in order; long rows
// by a warp, each lane in order, then the same shuffle tree), and the stage updates are the same
// functions, so the states equal those of the stage kernels bit for bit.
#include <cstdlib>

#include "internal.cuh"
#include "stage.cuh"

namespace gk {

namespace {

constexpr int kBlockThreads = 512;
constexpr long long kBlockMaxRows = 4096;   // D + 1 rows: 128 KB of FP64 vectors in shared memory
// where one block beats the stage kernels (measured, us per RK4 step, block against stages):
// FP64 N = 6: 4.6 / 27.3, N = 10: 9.5 / 14.7, N = 16: 13.4 / 14.3, N = 24: 32.6 / 15.3 (the one
// SM's FP64 pipe binds); FP32 N = 6: 3.2 / 27.0, N = 16: 5.5 / 12.9, N = 24: 10.4 / 13.0,
// N = 32: 16.4 / 12.7.  A cluster of up to 16 CTAs sharing the vectors through distributed shared
// memory was measured too and lost everywhere: its barrier between stages costs about 1.5 us more
// than the block's (N = 6 FP64: 10.4 us per step even as one CTA; N = 64: 22.8 against 14.9).
constexpr long long kBlockRows64 = 256, kBlockRows32 = 576;

// (C y)_r over the ELL slots of row r, y in shared memory; slot 0 given (c0, a0)
template <typename VT, int W>
__device__ inline VT row_dot(const HybView<VT> &H, long long r, int c0, VT a0, const VT *y) {
    VT s = a0 * y[c0];
    if constexpr (W > 0) {
#pragma unroll
        for (int j = 1; j < W; ++j) {
            const long long p = (long long)j * H.ld + r;
            s += __ldg(H.ell_val + p) * y[__ldg(H.ell_col + p)];
        }
    } else {
        for (int j = 1; j < H.width; ++j) {
            const long long p = (long long)j * H.ld + r;
            s += __ldg(H.ell_val + p) * y[__ldg(H.ell_col + p)];
        }
    }
    return s;
}

template <typename VT>
__device__ inline VT row_dot_full(const HybView<VT> &H, long long r, const VT *y) {
    VT s = VT(0);
    for (int j = 0; j < H.width; ++j) {
        const long long p = (long long)j * H.ld + r;
        s += __ldg(H.ell_val + p) * y[__ldg(H.ell_col + p)];
    }
    return s;
}

// (C y)_i of long row i by one warp, y in shared memory: lane sums in order, eight in flight,
// then the xor shuffle tree (the order of the stage kernels' long rows)
template <typename VT>
__device__ inline VT tail_dot_s(const HybView<VT> &H, long long i, int lane, const VT *y) {
    VT s = VT(0);
    const int e1 = H.tail_ptr[i + 1];
    int e = H.tail_ptr[i] + lane;
    for (; e + 224 < e1; e += 256) {
        int cc[8];
        VT vv[8], yy[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            cc[u] = __ldg(H.tail_col + e + 32 * u);
            vv[u] = __ldg(H.tail_val + e + 32 * u);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) yy[u] = y[cc[u]];
#pragma unroll
        for (int u = 0; u < 8; ++u) s += vv[u] * yy[u];
    }
    for (; e < e1; e += 32) s += __ldg(H.tail_val + e) * y[__ldg(H.tail_col + e)];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

struct BlockArgs {
    const int *long_rows;
    int n_long;
    long long D;
    const double *eps_tab;   // eps(t) - E at the three stage times of every step of the run
    long long first;         // the chunk's first step
    long long nsteps;
    HConst hc;
};

// one stage: every row's derivative from y, then the stage update into yn / acc / v
template <int STAGE, typename VT, int W, bool M>
__device__ inline void block_stage(const HybView<VT> &A0, const HybView<VT> &A1, const VT *q1, const BlockArgs &a,
                                   VT eps, const VT *y, VT *v, double *v64, VT *yn, VT *acc) {
    for (long long r = threadIdx.x; r < a.D; r += blockDim.x) {
        const int c0 = __ldg(A0.ell_col + r);
        if (c0 < 0) continue;   // a long row, summed by a warp below
        VT a0 = __ldg(A0.ell_val + r);
        if (M) a0 = fma(eps, __ldg(q1 + r), a0);
        VT s = row_dot<VT, W>(A0, r, c0, a0, y);
        if (!M) s = s + eps * row_dot_full<VT>(A1, r, y);
        epi<STAGE, VT>(r, s, v, v64, yn, acc, a.hc);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = warp; i < a.n_long; i += nw) {
        const VT s0 = tail_dot_s<VT>(A0, i, lane, y);
        const VT s1 = tail_dot_s<VT>(A1, i, lane, y);
        if (lane == 0) epi<STAGE, VT>(a.long_rows[i], s0 + eps * s1, v, v64, yn, acc, a.hc);
    }
    __syncthreads();
}

// The whole chunk: vectors into shared memory (index D holds the constant 1 that multiplies the
// K column), nsteps RK4 steps, the state back to global memory.  FP64 form: v_g is the state;
// FP32 form: v_g the FP64 master, v32_g its FP32 mirror.
template <typename VT, int W, bool M>
__global__ void __launch_bounds__(kBlockThreads) k_rk4_block(HybView<VT> A0, HybView<VT> A1, const VT *q1, BlockArgs a,
                                                             double *v_g, float *v32_g) {
    extern __shared__ __align__(16) unsigned char sm[];
    constexpr bool F64 = sizeof(VT) == 8;
    const long long n = a.D + 1;
    double *v64 = reinterpret_cast<double *>(sm);   // FP32 form only
    VT *base = reinterpret_cast<VT *>(sm + (F64 ? 0 : sizeof(double) * n));
    VT *v = base, *yA = base + n, *yB = base + 2 * n, *acc = base + 3 * n;
    for (long long r = threadIdx.x; r < n; r += blockDim.x) {
        if constexpr (F64) {
            v[r] = (VT)v_g[r];
        } else {
            v64[r] = v_g[r];
            v[r] = (VT)v32_g[r];
        }
        yA[r] = VT(1);
        yB[r] = VT(1);
        acc[r] = VT(0);
    }
    __syncthreads();
    for (long long s = 0; s < a.nsteps; ++s) {
        const double *e = a.eps_tab + 3 * (a.first + s);
        block_stage<1, VT, W, M>(A0, A1, q1, a, (VT)e[0], v, v, v64, yA, acc);
        block_stage<2, VT, W, M>(A0, A1, q1, a, (VT)e[1], yA, v, v64, yB, acc);
        block_stage<3, VT, W, M>(A0, A1, q1, a, (VT)e[1], yB, v, v64, yA, acc);
        block_stage<4, VT, W, M>(A0, A1, q1, a, (VT)e[2], yA, v, v64, nullptr, acc);
    }
    for (long long r = threadIdx.x; r < a.D; r += blockDim.x) {
        if constexpr (F64) {
            v_g[r] = (double)v[r];
        } else {
            v_g[r] = v64[r];
            v32_g[r] = (float)v[r];
        }
    }
}

template <typename VT, int W, bool M>
void launch_block(gksl_ctx *c, const Hyb<VT> &h0, const Hyb<VT> &h1, const VT *q1, const BlockArgs &a) {
    constexpr bool F64 = sizeof(VT) == 8;
    const size_t smem = (size_t)(a.D + 1) * (4 * sizeof(VT) + (F64 ? 0 : sizeof(double)));
    GK_CUDA(cudaFuncSetAttribute(k_rk4_block<VT, W, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_rk4_block<VT, W, M><<<1, kBlockThreads, smem, c->stream>>>(view(h0), view(h1), q1, a, c->v.p,
                                                                   F64 ? nullptr : c->v32.p);
    GK_LAUNCH_CHECK();
}

}  // namespace

bool rk4_block_applies(const gksl_ctx *c, int precision) {
    if (c->asm_flags & GKSL_ASM_MATRIX_FREE) return false;
    if (c->D + 1 > kBlockMaxRows) return false;
    const char *env = getenv("GKSL_RK4_BLOCK");
    if (env) return env[0] == '1';
    return c->D + 1 <= (precision == 64 ? kBlockRows64 : kBlockRows32);
}

void rk4_block_run(gksl_ctx *c, int precision, double h, const double *tab, long long first, long long count) {
    if (count <= 0) return;
    BlockArgs a;
    a.long_rows = c->hyb0.long_rows.p;
    a.n_long = (int)c->hyb0.n_long;
    a.D = c->D;
    a.eps_tab = tab;
    a.first = first;
    a.nsteps = count;
    a.hc.h = h;
    a.hc.h2 = 0.5 * h;
    a.hc.h6 = h / 6.0;
    a.hc.hf = (float)h;
    a.hc.h2f = 0.5f * (float)h;
    a.hc.h6f = (float)(h / 6.0);
    // the same instances as the stage kernels: the 18-slot one for 18-slot matrices, folded or not
    const bool M = c->q1_folded;
    const bool w18 = c->hyb0.width == 18;
    if (precision == 64) {
        const double *q1 = M ? c->q1v.p : nullptr;
        if (M && w18) launch_block<double, 18, true>(c, c->hyb0, c->hyb1, q1, a);
        else if (M) launch_block<double, 0, true>(c, c->hyb0, c->hyb1, q1, a);
        else if (w18) launch_block<double, 18, false>(c, c->hyb0, c->hyb1, q1, a);
        else launch_block<double, 0, false>(c, c->hyb0, c->hyb1, q1, a);
    } else {
        const float *q1 = M ? c->q1vf.p : nullptr;
        if (M && w18) launch_block<float, 18, true>(c, c->hyb0f, c->hyb1f, q1, a);
        else if (M) launch_block<float, 0, true>(c, c->hyb0f, c->hyb1f, q1, a);
        else if (w18) launch_block<float, 18, false>(c, c->hyb0f, c->hyb1f, q1, a);
        else launch_block<float, 0, false>(c, c->hyb0f, c->hyb1f, q1, a);
    }
}

}  // namespace gk
