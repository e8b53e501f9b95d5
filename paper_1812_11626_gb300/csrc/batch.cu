// Batched propagation: many instances of Eq. 8 that share the unfolded components and differ
// in the drive amplitude A_b and a dissipation scale g_b,
//     dv_b/dt = (QH + A_b sin(omega t) Q1 + g_b R) v_b + g_b K,
// with QH = sum_k theta_k Q(H0_k) + E Q1 and R, K the gamma-weighted dissipator terms of a
// group's context.  The state of a group is a (D+1) x B matrix V (instance index fastest,
// row D = 1 so that K rides as an extra column of R), and every RK4 stage is a sparse-matrix
// times dense-matrix product with three value channels.
//
// One persistent launch per stage covers every group (mixed N): each CTA walks the tile list
// (group, 8-row block, instance chunk); a warp owns one row and its 32 lanes own consecutive
// instances, so each matrix entry is loaded once per chunk and the gathers V[col, b] are
// coalesced.  Chunks are 32 * ipl instances wide (ipl instances per lane), chosen per group by
// timing the candidates (autotuner).  Groups with fewer steps drop out of the tile walk when
// they finish.  The FP32 bulk updates an FP64 master state every step; every
// `correction_every` steps one FP64 step replaces an FP32 one.  Chunks of steps are captured
// in CUDA graphs.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"
#include "prim.cuh"

namespace gk {
namespace {

constexpr int kBThreads = 256;
constexpr int kRowsPerTile = kBThreads / 32;
constexpr int kMaxIpl = 4;
constexpr int kMaxGroups = 8;
constexpr int kBatchGraphSteps = 32;

constexpr int kMaxCh = 4;   // QH, Q1, [R | K], and optionally one scanned Hamiltonian component

struct GroupDev {
    // pair units (FP32 path): unit u < P2 holds the rows u and P2 + u (the S and J generators of
    // one pair, which couple to nearly the same columns), units u >= P2 the D rows one each; per
    // unit the union of its rows' columns over all channels, with both rows' channel values
    const int *pptr;
    const int *pcol;
    const float4 *pval;   // 2 per entry: row a {QH, Q1, R|K, scan}, row b (0 for a D unit)
    long long P2, nunits;
    int pairs;            // FP32 steps use the pair units
    const int *ptr[kMaxCh];
    const int *col[kMaxCh];
    const float *vf[kMaxCh];
    const double *vd[kMaxCh];
    int nch;                  // 3, or 4 with a scanned component
    const double *S;          // per-instance coefficient of channel 3 (theta_b - theta_k)
    const float *Sf;
    long long D;
    int B, ipl, nchunks;
    long long Bs;   // row stride of the state matrices: B rounded up to 4 (16-byte rows)
    int vec4;       // FP32 steps use the 4-instances-per-lane path
    long long nsteps;
    double h, h2, h6;   // h, h/2, h/6 (computed on the host)
    float hf, h2f, h6f;
    const double *sin_tab;   // sin(omega t) at the 3 stage times of each step
    const float *sin_tab_f;  // the same in FP32 (FP32 steps use no FP64 arithmetic)
    const double *A, *g;
    const float *Af, *gf;
    double *V64;
    float *V32, *Y32[2], *ACC32;
    double *Y64[2], *ACC64;
    long long tile_begin, ntiles;
};

struct BatchArgs {
    GroupDev gr[kMaxGroups];
    int ng;
    long long ntiles;
    const long long *base;
    long long local;
};

// Stage update of element o = r * Bs + b (instance b of row r) from k.
template <int STAGE, bool F64>
__device__ inline void stage_update(const GroupDev &G, long long o, double kd, float kf) {
    if (F64) {
        double *yn = STAGE == 1 ? G.Y64[0] : (STAGE == 2 ? G.Y64[1] : G.Y64[0]);
        if (STAGE == 1) { yn[o] = G.V64[o] + G.h2 * kd; G.ACC64[o] = kd; }
        if (STAGE == 2) { yn[o] = G.V64[o] + G.h2 * kd; G.ACC64[o] += 2.0 * kd; }
        if (STAGE == 3) { yn[o] = G.V64[o] + G.h * kd; G.ACC64[o] += 2.0 * kd; }
        if (STAGE == 4) { G.V64[o] = G.V64[o] + G.h6 * (G.ACC64[o] + kd); G.V32[o] = (float)G.V64[o]; }
    } else {
        float *yn = STAGE == 1 ? G.Y32[0] : (STAGE == 2 ? G.Y32[1] : G.Y32[0]);
        if (STAGE == 1) { yn[o] = G.V32[o] + G.h2f * kf; G.ACC32[o] = kf; }
        if (STAGE == 2) { yn[o] = G.V32[o] + G.h2f * kf; G.ACC32[o] += 2.0f * kf; }
        if (STAGE == 3) { yn[o] = G.V32[o] + G.hf * kf; G.ACC32[o] += 2.0f * kf; }
        if (STAGE == 4) {
            float inc = G.h6f * (G.ACC32[o] + kf);
            double nv = G.V64[o] + (double)inc;
            G.V64[o] = nv;
            G.V32[o] = (float)nv;
        }
    }
}

// Row r for the instances b0 + 32 k, k < ipl, of this lane (scalar gathers).
template <int STAGE, bool F64>
__device__ inline void row_scalar(const GroupDev &G, long long r, int ch, int lane, long long step) {
    using VT = typename std::conditional<F64, double, float>::type;
    const int B = G.B;
    const long long Bs = G.Bs;
    const VT *X;
    if (F64) X = (const VT *)(STAGE == 1 ? (void *)G.V64 : (STAGE == 3 ? (void *)G.Y64[1] : (void *)G.Y64[0]));
    else X = (const VT *)(STAGE == 1 ? (void *)G.V32 : (STAGE == 3 ? (void *)G.Y32[1] : (void *)G.Y32[0]));
    VT acc[kMaxCh][kMaxIpl];
#pragma unroll
    for (int c = 0; c < kMaxCh; ++c)
#pragma unroll
        for (int k = 0; k < kMaxIpl; ++k) acc[c][k] = VT(0);
    const int b0 = ch * 32 * G.ipl + lane;
    // entries in groups of 4: load their columns and values, then issue every gather of the
    // group before the products, so each warp keeps several loads in flight
    constexpr int U = 4;
#pragma unroll
    for (int c = 0; c < kMaxCh; ++c) {
        if (c >= G.nch) break;
        const int e1 = G.ptr[c][r + 1];
        int e = G.ptr[c][r];
        for (; e + U <= e1; e += U) {
            int col[U];
            VT v[U], x[U][kMaxIpl];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                col[u] = G.col[c][e + u];
                v[u] = F64 ? (VT)G.vd[c][e + u] : (VT)G.vf[c][e + u];
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int k = 0; k < kMaxIpl; ++k) {
                    int b = b0 + 32 * k;
                    x[u][k] = (k < G.ipl && b < B) ? __ldg(X + (long long)col[u] * Bs + b) : VT(0);
                }
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int k = 0; k < kMaxIpl; ++k) acc[c][k] += v[u] * x[u][k];
        }
        for (; e < e1; ++e) {
            const int col = G.col[c][e];
            const VT v = F64 ? (VT)G.vd[c][e] : (VT)G.vf[c][e];
            const VT *xr = X + (long long)col * Bs;
#pragma unroll
            for (int k = 0; k < kMaxIpl; ++k) {
                int b = b0 + 32 * k;
                if (k < G.ipl && b < B) acc[c][k] += v * __ldg(xr + b);
            }
        }
    }
    const int slot = STAGE == 1 ? 0 : (STAGE == 4 ? 2 : 1);
    const long long ts = 3 * step + slot;
#pragma unroll
    for (int k = 0; k < kMaxIpl; ++k) {
        int b = b0 + 32 * k;
        if (k >= G.ipl || b >= B) continue;
        long long o = r * Bs + b;
        if (F64) {
            double kd = acc[0][k] + (G.A[b] * G.sin_tab[ts]) * acc[1][k] + G.g[b] * acc[2][k];
            if (G.nch > 3) kd += G.S[b] * acc[3][k];
            stage_update<STAGE, true>(G, o, kd, 0.0f);
        } else {
            float kf = (float)(acc[0][k] + (G.Af[b] * G.sin_tab_f[ts]) * acc[1][k] + G.gf[b] * acc[2][k]);
            if (G.nch > 3) kf += G.Sf[b] * (float)acc[3][k];
            stage_update<STAGE, false>(G, o, 0.0, kf);
        }
    }
}

// Row r for 4 consecutive instances per lane (128 per warp), one 16-byte gather per entry.
template <int STAGE>
__device__ inline void row_vec4(const GroupDev &G, long long r, int ch, int lane, long long step) {
    const int bq = ch * 128 + 4 * lane;
    if (bq >= G.B) return;
    const long long Bs = G.Bs;
    const float *X = STAGE == 1 ? G.V32 : (STAGE == 3 ? G.Y32[1] : G.Y32[0]);
    float4 acc[kMaxCh];
#pragma unroll
    for (int c = 0; c < kMaxCh; ++c) acc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    constexpr int U = 4;
#pragma unroll
    for (int c = 0; c < kMaxCh; ++c) {
        if (c >= G.nch) break;
        const int e1 = G.ptr[c][r + 1];
        int e = G.ptr[c][r];
        for (; e + U <= e1; e += U) {
            int col[U];
            float v[U];
            float4 x[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                col[u] = G.col[c][e + u];
                v[u] = G.vf[c][e + u];
            }
#pragma unroll
            for (int u = 0; u < U; ++u) x[u] = __ldg((const float4 *)(X + (long long)col[u] * Bs + bq));
#pragma unroll
            for (int u = 0; u < U; ++u) {
                acc[c].x += v[u] * x[u].x;
                acc[c].y += v[u] * x[u].y;
                acc[c].z += v[u] * x[u].z;
                acc[c].w += v[u] * x[u].w;
            }
        }
        for (; e < e1; ++e) {
            const float v = G.vf[c][e];
            const float4 x = __ldg((const float4 *)(X + (long long)G.col[c][e] * Bs + bq));
            acc[c].x += v * x.x;
            acc[c].y += v * x.y;
            acc[c].z += v * x.z;
            acc[c].w += v * x.w;
        }
    }
    const int slot = STAGE == 1 ? 0 : (STAGE == 4 ? 2 : 1);
    const float sn = G.sin_tab_f[3 * step + slot];
    const float a0[4] = {acc[0].x, acc[0].y, acc[0].z, acc[0].w};
    const float a1[4] = {acc[1].x, acc[1].y, acc[1].z, acc[1].w};
    const float a2[4] = {acc[2].x, acc[2].y, acc[2].z, acc[2].w};
    const float a3[4] = {acc[3].x, acc[3].y, acc[3].z, acc[3].w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int b = bq + k;
        if (b >= G.B) break;
        float kf = a0[k] + (G.Af[b] * sn) * a1[k] + G.gf[b] * a2[k];
        if (G.nch > 3) kf += G.Sf[b] * a3[k];
        stage_update<STAGE, false>(G, r * Bs + b, 0.0, kf);
    }
}

// Unit u of the pair form for the instances b0 + 32 k, k < ipl, of this lane: every entry's
// column is gathered once and serves both rows of the unit (scalar 4-byte gathers, coalesced
// across lanes), then the two rows' stage updates.
template <int STAGE>
__device__ inline void unit_pair(const GroupDev &G, long long u, int ch, int lane, long long step) {
    const int B = G.B;
    const long long Bs = G.Bs;
    const float *X = STAGE == 1 ? G.V32 : (STAGE == 3 ? G.Y32[1] : G.Y32[0]);
    const bool scan = G.nch > 3;
    float acc[2][kMaxCh][kMaxIpl];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int c = 0; c < kMaxCh; ++c)
#pragma unroll
            for (int k = 0; k < kMaxIpl; ++k) acc[q][c][k] = 0.f;
    const int b0 = ch * 32 * G.ipl + lane;
    const int e1 = G.pptr[u + 1];
    constexpr int U = 2;
    int e = G.pptr[u];
    for (; e + U <= e1; e += U) {
        int col[U];
        float x[U][kMaxIpl];
#pragma unroll
        for (int v = 0; v < U; ++v) col[v] = G.pcol[e + v];
#pragma unroll
        for (int v = 0; v < U; ++v)
#pragma unroll
            for (int k = 0; k < kMaxIpl; ++k) {
                const int b = b0 + 32 * k;
                x[v][k] = (k < G.ipl && b < B) ? __ldg(X + (long long)col[v] * Bs + b) : 0.f;
            }
#pragma unroll
        for (int v = 0; v < U; ++v) {
            const float4 wa = G.pval[2 * (e + v)], wb = G.pval[2 * (e + v) + 1];
#pragma unroll
            for (int k = 0; k < kMaxIpl; ++k) {
                acc[0][0][k] += wa.x * x[v][k]; acc[0][1][k] += wa.y * x[v][k]; acc[0][2][k] += wa.z * x[v][k];
                acc[1][0][k] += wb.x * x[v][k]; acc[1][1][k] += wb.y * x[v][k]; acc[1][2][k] += wb.z * x[v][k];
                if (scan) { acc[0][3][k] += wa.w * x[v][k]; acc[1][3][k] += wb.w * x[v][k]; }
            }
        }
    }
    for (; e < e1; ++e) {
        const int col = G.pcol[e];
        const float4 wa = G.pval[2 * e], wb = G.pval[2 * e + 1];
#pragma unroll
        for (int k = 0; k < kMaxIpl; ++k) {
            const int b = b0 + 32 * k;
            const float x = (k < G.ipl && b < B) ? __ldg(X + (long long)col * Bs + b) : 0.f;
            acc[0][0][k] += wa.x * x; acc[0][1][k] += wa.y * x; acc[0][2][k] += wa.z * x;
            acc[1][0][k] += wb.x * x; acc[1][1][k] += wb.y * x; acc[1][2][k] += wb.z * x;
            if (scan) { acc[0][3][k] += wa.w * x; acc[1][3][k] += wb.w * x; }
        }
    }
    const int slot = STAGE == 1 ? 0 : (STAGE == 4 ? 2 : 1);
    const float sn = G.sin_tab_f[3 * step + slot];
    const long long ra = u < G.P2 ? u : G.P2 + u;   // D units: row 2 P2 + (u - P2)
    const int nrows = u < G.P2 ? 2 : 1;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        if (q >= nrows) break;
        const long long r = q == 0 ? ra : u + G.P2;
#pragma unroll
        for (int k = 0; k < kMaxIpl; ++k) {
            const int b = b0 + 32 * k;
            if (k >= G.ipl || b >= B) continue;
            float kf = acc[q][0][k] + (G.Af[b] * sn) * acc[q][1][k] + G.gf[b] * acc[q][2][k];
            if (scan) kf += G.Sf[b] * acc[q][3][k];
            stage_update<STAGE, false>(G, r * Bs + b, 0.0, kf);
        }
    }
}

// PAIRS: the instance with the pair path, launched (FP32 steps) when some group uses it; its
// accumulators for two rows take more registers, so the row-only instance stays separate
template <int STAGE, bool F64, bool PAIRS>
__global__ void __launch_bounds__(kBThreads) k_batch_stage(BatchArgs a) {
    const long long step = *a.base + a.local;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (long long t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        int gi = 0;
        while (gi + 1 < a.ng && t >= a.gr[gi + 1].tile_begin) ++gi;
        const GroupDev &G = a.gr[gi];
        if (step >= G.nsteps) continue;
        long long tl = t - G.tile_begin;
        int ch = (int)(tl % G.nchunks);
        if constexpr (PAIRS && !F64) {
            if (G.pairs) {
                const long long u = (tl / G.nchunks) * kRowsPerTile + warp;
                if (u < G.nunits) unit_pair<STAGE>(G, u, ch, lane, step);
                continue;
            }
        }
        long long r = (tl / G.nchunks) * kRowsPerTile + warp;
        if (r >= G.D) continue;
        if (!F64 && G.vec4) row_vec4<STAGE>(G, r, ch, lane, step);
        else row_scalar<STAGE, F64>(G, r, ch, lane, step);
    }
}

// theta of the drive (sin or square, see drive_theta) at the 3 stage times of each step
__global__ void k_sin_table(double t0, double h, double omega, int shape, long long n, double *__restrict__ tab,
                            float *__restrict__ tabf) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double th[3];
    drive_theta(shape, omega, t0 + (double)i * h, h, th);
    double s0 = th[0], s1 = th[1], s2 = th[2];
    tab[3 * i + 0] = s0;
    tab[3 * i + 1] = s1;
    tab[3 * i + 2] = s2;
    tabf[3 * i + 0] = (float)s0;
    tabf[3 * i + 1] = (float)s1;
    tabf[3 * i + 2] = (float)s2;
}

__global__ void k_replicate(const double *__restrict__ v, long long rows, int B, double *__restrict__ V64,
                            float *__restrict__ V32) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * B) return;
    double x = v[i / B];
    V64[i] = x;
    V32[i] = (float)x;
}

__global__ void k_fill_row(double *V64, float *V32, float *Ya, float *Yb, double *Y64a, double *Y64b, long long row,
                           int B) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    long long o = row * B + b;
    V64[o] = 1.0;
    V32[o] = 1.0f;
    Ya[o] = 1.0f;
    Yb[o] = 1.0f;
    Y64a[o] = 1.0;
    Y64b[o] = 1.0;
}

__global__ void k_column(const double *__restrict__ V, long long rows, int B, int b, double *__restrict__ out) {
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < rows) out[r] = V[r * B + b];
}

__global__ void k_set_base(long long *p, long long v) { *p = v; }

struct Group {
    gksl_ctx *ctx = nullptr;
    long long D = 0;
    int B = 0;
    long long Bs = 0;     // B rounded up to 4: the row stride of every state matrix
    int ipl = 1;          // instances per lane of the scalar FP32 path
    bool vec4 = true;     // FP32 steps: 4 instances per lane with 16-byte gathers
    int ipl64 = 1;        // instances per lane of the FP64 steps
    CsrR m[kMaxCh];       // QH (E folded), Q1, [R | K], scanned component Q(H0_k)
    DBuf<float> mf[kMaxCh];  // FP32 values
    int nch = 3;
    DBuf<double> S;       // per-instance coefficient of the scanned component (theta_b - theta_k)
    DBuf<float> Sf;
    DBuf<double> A, g, V64, Y64a, Y64b, ACC64, sin_tab;
    DBuf<float> Af, gf, sin_tab_f;
    DBuf<float> V32, Ya, Yb, ACC32;
    long long nsteps = 0;
    double h = 0.0;
    double t = 0.0;   // time of the group's states
    double tuned_us = 0.0;
    DBuf<int> pptr, pcol;               // pair units of the FP32 path (see GroupDev)
    DBuf<float4> pval;
    long long P2 = 0, nunits = 0, pnnz = 0;
    bool pairs = false;
    DBuf<double> Vprev;                 // state one period earlier (gksl_batch_asymptotic)
    DBuf<unsigned long long> resid;     // per-instance period-map residual, as double bit patterns
};

}  // namespace
}  // namespace gk

struct gksl_batch {
    std::vector<gk::Group> groups;
    cudaStream_t stream = nullptr;
    int device = 0;
    std::string err;
    gk::DBuf<long long> base;
    std::vector<int> first_instance;   // global instance index of each group's first instance
    int n_instances = 0;
    struct Graph {
        int f64;
        cudaGraphExec_t exec;
    };
    std::vector<Graph> graphs;
    bool tuned = false;
    ~gksl_batch() {
        for (auto &g : graphs) cudaGraphExecDestroy(g.exec);
        if (stream) cudaStreamDestroy(stream);
    }
};

namespace gk {
namespace {

__global__ void k_f2(const double *__restrict__ v, float *__restrict__ o, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) o[i] = (float)v[i];
}

// Pair units of a group: unit u < P2 merges the sorted column lists of rows u and P2 + u over
// every channel, unit u >= P2 those of row P2 + u; pass 1 counts a unit's distinct columns, pass 2
// writes them with both rows' FP32 channel values (0 where a row or channel has no entry).
struct ChanCsr {
    const int *ptr[kMaxCh];
    const int *col[kMaxCh];
    const float *val[kMaxCh];
    int nch;
};

template <bool FILL>
__global__ void k_pair_units(ChanCsr m, long long P2, long long nunits, long long *__restrict__ cnt,
                             const int *__restrict__ pptr, int *__restrict__ pcol, float4 *__restrict__ pval) {
    const long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= nunits) return;
    const int nr = u < P2 ? 2 : 1;
    const long long row[2] = {u < P2 ? u : P2 + u, u + P2};
    int e[2][kMaxCh], end[2][kMaxCh];
    for (int q = 0; q < 2; ++q)
        for (int c = 0; c < kMaxCh; ++c) {
            const bool on = q < nr && c < m.nch;
            e[q][c] = on ? m.ptr[c][row[q]] : 0;
            end[q][c] = on ? m.ptr[c][row[q] + 1] : 0;
        }
    long long n = 0, o = FILL ? pptr[u] : 0;
    for (;;) {
        int cmin = 0x7fffffff;
        for (int q = 0; q < 2; ++q)
            for (int c = 0; c < kMaxCh; ++c)
                if (e[q][c] < end[q][c] && m.col[c][e[q][c]] < cmin) cmin = m.col[c][e[q][c]];
        if (cmin == 0x7fffffff) break;
        float v[2][kMaxCh] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
        for (int q = 0; q < 2; ++q)
            for (int c = 0; c < kMaxCh; ++c)
                if (e[q][c] < end[q][c] && m.col[c][e[q][c]] == cmin) {
                    if (FILL) v[q][c] = m.val[c][e[q][c]];
                    ++e[q][c];
                }
        if (FILL) {
            pcol[o] = cmin;
            pval[2 * o] = make_float4(v[0][0], v[0][1], v[0][2], v[0][3]);
            pval[2 * o + 1] = make_float4(v[1][0], v[1][1], v[1][2], v[1][3]);
            ++o;
        }
        ++n;
    }
    if (!FILL) cnt[u] = n;
}

__global__ void k_ll_to_i32(const long long *__restrict__ in, long long n, int *__restrict__ out) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (int)in[i];
}

void build_pairs(Group &G, cudaStream_t s) {
    ChanCsr m{};
    m.nch = G.nch;
    for (int c = 0; c < G.nch; ++c) {
        m.ptr[c] = G.m[c].rowptr.p;
        m.col[c] = G.m[c].col.p;
        m.val[c] = G.mf[c].p;
    }
    G.P2 = G.ctx->P2;
    G.nunits = G.D - G.P2;
    const long long nu = G.nunits;
    DBuf<long long> cnt((size_t)nu), off((size_t)nu + 1);
    k_pair_units<false><<<grid_for(nu, 256), 256, 0, s>>>(m, G.P2, nu, cnt.p, nullptr, nullptr, nullptr);
    GK_LAUNCH_CHECK();
    const long long nnz = scan_ll(cnt.p, off.p, nu, true, true, s);
    GK_REQUIRE(nnz < (1LL << 30), GKSL_ERR_ARG, "batched group too large for the pair form");
    G.pptr.alloc((size_t)nu + 1);
    G.pcol.alloc((size_t)std::max(1LL, nnz));
    G.pval.alloc((size_t)std::max(1LL, 2 * nnz));
    k_ll_to_i32<<<grid_for(nu + 1, 256), 256, 0, s>>>(off.p, nu + 1, G.pptr.p);
    GK_LAUNCH_CHECK();
    k_pair_units<true><<<grid_for(nu, 256), 256, 0, s>>>(m, G.P2, nu, nullptr, G.pptr.p, G.pcol.p, G.pval.p);
    GK_LAUNCH_CHECK();
    G.pnnz = nnz;
    GK_CUDA(cudaStreamSynchronize(s));
}

BatchArgs make_args(gksl_batch *b, bool f64, long long local) {
    BatchArgs a{};
    a.ng = (int)b->groups.size();
    long long tb = 0;
    for (int i = 0; i < a.ng; ++i) {
        Group &G = b->groups[i];
        GroupDev &d = a.gr[i];
        for (int c = 0; c < kMaxCh; ++c) {
            d.ptr[c] = G.m[c].rowptr.p;
            d.col[c] = G.m[c].col.p;
            d.vf[c] = G.mf[c].p;
            d.vd[c] = G.m[c].val.p;
        }
        d.nch = G.nch;
        d.pptr = G.pptr.p;
        d.pcol = G.pcol.p;
        d.pval = G.pval.p;
        d.P2 = G.P2;
        d.nunits = G.nunits;
        d.pairs = (!f64 && G.pairs) ? 1 : 0;
        d.S = G.S.p;
        d.Sf = G.Sf.p;
        d.D = G.D;
        d.B = G.B;
        d.Bs = G.Bs;
        d.vec4 = (!f64 && G.vec4) ? 1 : 0;
        d.ipl = f64 ? G.ipl64 : G.ipl;
        d.nchunks = d.vec4 ? (G.B + 127) / 128 : (G.B + 32 * d.ipl - 1) / (32 * d.ipl);
        d.nsteps = G.nsteps;
        d.h = G.h;
        d.h2 = 0.5 * G.h;
        d.h6 = G.h / 6.0;
        d.hf = (float)G.h;
        d.h2f = (float)(0.5 * G.h);
        d.h6f = (float)(G.h / 6.0);
        d.sin_tab = G.sin_tab.p;
        d.sin_tab_f = G.sin_tab_f.p;
        d.A = G.A.p;
        d.g = G.g.p;
        d.Af = G.Af.p;
        d.gf = G.gf.p;
        d.V64 = G.V64.p;
        d.V32 = G.V32.p;
        d.Y32[0] = G.Ya.p;
        d.Y32[1] = G.Yb.p;
        d.ACC32 = G.ACC32.p;
        d.Y64[0] = G.Y64a.p;
        d.Y64[1] = G.Y64b.p;
        d.ACC64 = G.ACC64.p;
        d.tile_begin = tb;
        const long long units = d.pairs ? G.nunits : G.D;   // warps' work items: pair units or rows
        d.ntiles = ((units + kRowsPerTile - 1) / kRowsPerTile) * d.nchunks;
        tb += d.ntiles;
    }
    a.ntiles = tb;
    a.base = b->base.p;
    a.local = local;
    return a;
}

unsigned batch_grid(long long ntiles) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long g = (long long)sms * 8;
    if (g > ntiles) g = ntiles;
    return (unsigned)(g < 1 ? 1 : g);
}

void launch_batch_step(gksl_batch *b, bool f64, long long local) {
    BatchArgs a = make_args(b, f64, local);
    unsigned grid = batch_grid(a.ntiles);
    cudaStream_t s = b->stream;
    bool pairs = false;
    for (int i = 0; i < a.ng; ++i) pairs = pairs || a.gr[i].pairs;
    if (f64) {
        k_batch_stage<1, true, false><<<grid, kBThreads, 0, s>>>(a);
        k_batch_stage<2, true, false><<<grid, kBThreads, 0, s>>>(a);
        k_batch_stage<3, true, false><<<grid, kBThreads, 0, s>>>(a);
        k_batch_stage<4, true, false><<<grid, kBThreads, 0, s>>>(a);
    } else if (pairs) {
        k_batch_stage<1, false, true><<<grid, kBThreads, 0, s>>>(a);
        k_batch_stage<2, false, true><<<grid, kBThreads, 0, s>>>(a);
        k_batch_stage<3, false, true><<<grid, kBThreads, 0, s>>>(a);
        k_batch_stage<4, false, true><<<grid, kBThreads, 0, s>>>(a);
    } else {
        k_batch_stage<1, false, false><<<grid, kBThreads, 0, s>>>(a);
        k_batch_stage<2, false, false><<<grid, kBThreads, 0, s>>>(a);
        k_batch_stage<3, false, false><<<grid, kBThreads, 0, s>>>(a);
        k_batch_stage<4, false, false><<<grid, kBThreads, 0, s>>>(a);
    }
    GK_LAUNCH_CHECK();
}

void clear_batch_graphs(gksl_batch *b) {
    for (auto &g : b->graphs) cudaGraphExecDestroy(g.exec);
    b->graphs.clear();
}

cudaGraphExec_t batch_graph(gksl_batch *b, bool f64) {
    for (auto &g : b->graphs)
        if (g.f64 == (int)f64) return g.exec;
    cudaGraph_t graph;
    GK_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < kBatchGraphSteps; ++i) launch_batch_step(b, f64, i);
    GK_CUDA(cudaStreamEndCapture(b->stream, &graph));
    cudaGraphExec_t exec;
    GK_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    GK_CUDA(cudaGraphDestroy(graph));
    b->graphs.push_back({(int)f64, exec});
    return exec;
}

void run_batch_steps(gksl_batch *b, bool f64, long long first, long long count) {
    long long n = first, end = first + count;
    while (end - n >= kBatchGraphSteps) {
        k_set_base<<<1, 1, 0, b->stream>>>(b->base.p, n);
        GK_LAUNCH_CHECK();
        GK_CUDA(cudaGraphLaunch(batch_graph(b, f64), b->stream));
        n += kBatchGraphSteps;
    }
    if (n < end) {
        k_set_base<<<1, 1, 0, b->stream>>>(b->base.p, n);
        GK_LAUNCH_CHECK();
        for (long long i = 0; n + i < end; ++i) launch_batch_step(b, f64, i);
    }
}

void reset_batch(gksl_batch *b) {
    for (auto &G : b->groups) {
        gksl_ctx *c = G.ctx;
        GK_REQUIRE(c->state_set, GKSL_ERR_STATE, "a group context has no state");
        G.t = 0.0;
        long long rows = G.D + 1;
        // every stride slot (padding instances included) gets a finite copy of the state
        k_replicate<<<grid_for(rows * G.Bs, 256), 256, 0, b->stream>>>(c->v.p, rows, (int)G.Bs, G.V64.p, G.V32.p);
        GK_LAUNCH_CHECK();
        k_fill_row<<<grid_for(G.Bs, 128), 128, 0, b->stream>>>(G.V64.p, G.V32.p, G.Ya.p, G.Yb.p, G.Y64a.p, G.Y64b.p,
                                                                G.D, (int)G.Bs);
        GK_LAUNCH_CHECK();
    }
    GK_CUDA(cudaStreamSynchronize(b->stream));
}

// Time every candidate chunk width on a few FP32 steps of the group alone; keep the fastest.
void autotune(gksl_batch *b) {
    std::vector<Group *> all;
    for (auto &G : b->groups) all.push_back(&G);
    // GKSL_BATCH_TILE=0 forces the 16-byte-gather path, 1..4 the scalar row path with that many
    // instances per lane, p1..p4 the pair path (for tests of each path; normally chosen by timing)
    const char *env = getenv("GKSL_BATCH_TILE");
    if (env) {
        const bool pr = env[0] == 'p';
        const char *d = pr ? env + 1 : env;
        if (d[0] >= (pr ? '1' : '0') && d[0] <= '0' + kMaxIpl && d[1] == 0) {
            const int f = d[0] - '0';
            for (auto *G : all) {
                G->pairs = pr;
                G->vec4 = !pr && f == 0;
                G->ipl = f == 0 ? 1 : f;
                G->tuned_us = 0.0;
            }
            clear_batch_graphs(b);
            b->tuned = true;
            return;
        }
    }
    cudaEvent_t e0, e1;
    GK_CUDA(cudaEventCreate(&e0));
    GK_CUDA(cudaEventCreate(&e1));
    for (auto *G : all) {
        // run this group alone: other groups get nsteps = 0 for the trial
        std::vector<long long> saved;
        for (auto *H : all) saved.push_back(H->nsteps);
        for (auto *H : all) H->nsteps = (H == G) ? 1LL << 40 : 0;
        std::vector<double> tab_saved;
        if (G->sin_tab.n < 3 * 64) {
            G->sin_tab.alloc(3 * 64);
            G->sin_tab_f.alloc(3 * 64);
        }
        k_sin_table<<<1, 64, 0, b->stream>>>(0.0, 1e-6, 1.0, 0, 16, G->sin_tab.p, G->sin_tab_f.p);
        GK_LAUNCH_CHECK();
        double best = 1e300;
        int best_ipl = 1;
        bool best_vec4 = false, best_pairs = false;
        // candidates: the 16-byte gather path (ipl = 0 below), 1..4 scalar instances per lane on
        // rows, then the same on pair units
        for (int cand = 0; cand <= 2 * kMaxIpl; ++cand) {
            const bool pr = cand > kMaxIpl;
            const int ipl = pr ? cand - kMaxIpl : cand;
            if (ipl > 0 && 32 * (ipl - 1) >= G->B) continue;   // wider chunks than the batch add nothing
            G->pairs = pr;
            G->vec4 = (ipl == 0);
            G->ipl = ipl == 0 ? 1 : ipl;
            G->h = 1e-6;   // tiny step: the trial leaves the state essentially unchanged
            k_set_base<<<1, 1, 0, b->stream>>>(b->base.p, 0);
            for (int w = 0; w < 2; ++w) launch_batch_step(b, false, w);
            GK_CUDA(cudaEventRecord(e0, b->stream));
            for (int w = 0; w < 8; ++w) launch_batch_step(b, false, w);
            GK_CUDA(cudaEventRecord(e1, b->stream));
            GK_CUDA(cudaEventSynchronize(e1));
            float ms = 0;
            GK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) { best = ms; best_ipl = G->ipl; best_vec4 = G->vec4; best_pairs = G->pairs; }
        }
        G->ipl = best_ipl;
        G->vec4 = best_vec4;
        G->pairs = best_pairs;
        G->tuned_us = best * 1000.0 / 8.0;
        for (size_t i = 0; i < all.size(); ++i) all[i]->nsteps = saved[i];
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    reset_batch(b);   // the trials touched the states
    clear_batch_graphs(b);
    b->tuned = true;
}

}  // namespace
}  // namespace gk

using namespace gk;

namespace {
template <typename F>
gksl_status bguarded(gksl_batch *b, F &&f) {
    if (!b) return GKSL_ERR_ARG;
    try {
        int prev = -1;
        cudaGetDevice(&prev);
        if (prev != b->device) cudaSetDevice(b->device);
        b->err.clear();
        f();
        return GKSL_OK;
    } catch (const Error &e) {
        b->err = e.msg;
        return e.st;
    } catch (const std::exception &e) {
        b->err = e.what();
        return GKSL_ERR_ARG;
    }
}
}  // namespace

static thread_local std::string g_create_error;

extern "C" gksl_status gksl_batch_create(int n_groups, gksl_ctx *const *groups, const int *n_inst, const double *A,
                                         const double *g, gksl_batch **out) {
    if (!out || n_groups < 1 || n_groups > kMaxGroups || !groups || !n_inst || !A || !g) return GKSL_ERR_ARG;
    *out = nullptr;
    gksl_batch *b = new (std::nothrow) gksl_batch();
    if (!b) return GKSL_ERR_OOM;
    b->device = groups[0] ? groups[0]->device : 0;
    gksl_status st = bguarded(b, [&] {
        GK_CUDA(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
        b->base.alloc(1);
        int total = 0;
        for (int i = 0; i < n_groups; ++i) {
            GK_REQUIRE(groups[i] && n_inst[i] > 0, GKSL_ERR_ARG, "every group needs a context and >= 1 instance");
            GK_REQUIRE(groups[i]->assembled, GKSL_ERR_STATE, "group contexts must be assembled");
            GK_REQUIRE(!(groups[i]->asm_flags & GKSL_ASM_MATRIX_FREE), GKSL_ERR_STATE,
                       "group contexts must be assembled with CSR matrices");
            GK_REQUIRE(groups[i]->device == b->device, GKSL_ERR_ARG, "all groups must live on one device");
            total += n_inst[i];
        }
        std::vector<double> hA(A, A + total), hg(g, g + total);
        for (int i = 0; i < total; ++i)
            GK_REQUIRE(std::isfinite(hA[i]) && std::isfinite(hg[i]) && hg[i] >= 0.0, GKSL_ERR_ARG,
                       "instance parameters must be finite with g >= 0");
        b->groups.resize((size_t)n_groups);
        int off = 0;
        for (int i = 0; i < n_groups; ++i) {
            gksl_ctx *c = groups[i];
            Group &G = b->groups[i];
            G.ctx = c;
            G.D = c->D;
            G.B = n_inst[i];
            b->first_instance.push_back(off);
            cudaStream_t s = c->stream;
            // channels from the group's components: QH = sum theta Q(H0_k) + E Q1, Q1, [R | K]
            std::vector<std::pair<const CsrR *, double>> th, rr;
            for (int k = 0; k < GKSL_MAX_H0; ++k)
                if (c->has_h0[k]) th.push_back({&c->QH0[k], c->h0[k].weight});
            th.push_back({&c->Q1, c->E});
            for (int p = 0; p < GKSL_MAX_P; ++p)
                if (c->has_r[p]) rr.push_back({&c->R[p], c->diss[p].weight});
            // merged on the device by the assembly's COO reduction (exact zeros dropped)
            merge_terms(c, th, nullptr, G.m[0]);
            merge_terms(c, {{&c->Q1, 1.0}}, nullptr, G.m[1]);
            merge_terms(c, rr, c->K.p, G.m[2]);
            for (int ch = 0; ch < 3; ++ch) {
                G.mf[ch].alloc((size_t)std::max(1LL, G.m[ch].nnz));
                if (G.m[ch].nnz > 0) {
                    k_f2<<<grid_for(G.m[ch].nnz, 256), 256, 0, s>>>(G.m[ch].val.p, G.mf[ch].p, G.m[ch].nnz);
                    GK_LAUNCH_CHECK();
                }
            }
            GK_CUDA(cudaStreamSynchronize(s));
            build_pairs(G, s);
            G.A.alloc((size_t)G.B);
            G.g.alloc((size_t)G.B);
            G.Af.alloc((size_t)G.B);
            G.gf.alloc((size_t)G.B);
            GK_CUDA(cudaMemcpy(G.A.p, hA.data() + off, sizeof(double) * G.B, cudaMemcpyHostToDevice));
            GK_CUDA(cudaMemcpy(G.g.p, hg.data() + off, sizeof(double) * G.B, cudaMemcpyHostToDevice));
            std::vector<float> fa(hA.begin() + off, hA.begin() + off + G.B), fg(hg.begin() + off, hg.begin() + off + G.B);
            GK_CUDA(cudaMemcpy(G.Af.p, fa.data(), sizeof(float) * G.B, cudaMemcpyHostToDevice));
            GK_CUDA(cudaMemcpy(G.gf.p, fg.data(), sizeof(float) * G.B, cudaMemcpyHostToDevice));
            G.Bs = (G.B + 3) / 4 * 4;
            G.ipl64 = std::min(kMaxIpl, (G.B + 31) / 32);
            long long n = (G.D + 1) * G.Bs;
            G.V64.alloc((size_t)n);
            G.Y64a.alloc((size_t)n);
            G.Y64b.alloc((size_t)n);
            G.ACC64.alloc((size_t)n);
            G.V32.alloc((size_t)n);
            G.Ya.alloc((size_t)n);
            G.Yb.alloc((size_t)n);
            G.ACC32.alloc((size_t)n);
            off += G.B;
        }
        b->n_instances = total;
        reset_batch(b);
    });
    if (st != GKSL_OK) {
        g_create_error = b->err;
        delete b;
        return st;
    }
    g_create_error.clear();
    *out = b;
    return GKSL_OK;
}

extern "C" void gksl_batch_destroy(gksl_batch *b) {
    if (!b) return;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    delete b;
}

extern "C" const char *gksl_batch_last_error(const gksl_batch *b) {
    return b ? b->err.c_str() : g_create_error.c_str();
}

extern "C" gksl_status gksl_batch_reset(gksl_batch *b) {
    return bguarded(b, [&] { reset_batch(b); });
}

namespace gk {
namespace {

// n_steps[g] RK4 steps of every group g at h = T / steps_per_period[g] (FP32 bulk, an FP64 step
// every correction_every steps); returns the device time in milliseconds
double batch_advance(gksl_batch *b, const long long *spp, const long long *n_steps, long long correction_every) {
    GK_REQUIRE(spp && n_steps, GKSL_ERR_ARG, "steps_per_period and n_steps arrays required");
    if (!b->tuned) autotune(b);
    long long maxsteps = 0;
    for (size_t i = 0; i < b->groups.size(); ++i) {
        Group &G = b->groups[i];
        GK_REQUIRE(spp[i] > 0 && n_steps[i] >= 0, GKSL_ERR_ARG, "steps_per_period > 0 and n_steps >= 0 required");
        double T = 2.0 * M_PI / G.ctx->omega;
        double h = T / (double)spp[i];
        long long n = n_steps[i];
        if (G.ctx->drive_shape == GKSL_DRIVE_SQUARE) {
            double k = G.t / h;
            GK_REQUIRE(spp[i] % 2 == 0 && std::fabs(k - std::nearbyint(k)) <= 1e-6 * std::max(1.0, std::fabs(k)),
                       GKSL_ERR_ARG, "the square drive needs an even steps_per_period and times on the step grid");
        }
        if (G.h != h || G.nsteps != n) clear_batch_graphs(b);
        G.h = h;
        G.nsteps = n;
        if (G.sin_tab.n < (size_t)(3 * std::max(1LL, n))) {
            G.sin_tab.alloc((size_t)(3 * std::max(1LL, n)));
            G.sin_tab_f.alloc((size_t)(3 * std::max(1LL, n)));
            clear_batch_graphs(b);
        }
        if (n > 0) {
            k_sin_table<<<grid_for(n, 256), 256, 0, b->stream>>>(G.t, h, G.ctx->omega, G.ctx->drive_shape, n,
                                                                 G.sin_tab.p, G.sin_tab_f.p);
            GK_LAUNCH_CHECK();
        }
        G.t += (double)n * h;
        maxsteps = std::max(maxsteps, n);
    }
    cudaEvent_t e0, e1;
    GK_CUDA(cudaEventCreate(&e0));
    GK_CUDA(cudaEventCreate(&e1));
    GK_CUDA(cudaEventRecord(e0, b->stream));
    long long n = 0;
    while (n < maxsteps) {
        long long stop = maxsteps;
        long long corr = -1;
        if (correction_every > 0) corr = (n / correction_every + 1) * correction_every - 1;
        if (corr >= 0 && corr < stop) {
            if (corr > n) run_batch_steps(b, false, n, corr - n);
            run_batch_steps(b, true, corr, 1);
            n = corr + 1;
        } else {
            run_batch_steps(b, false, n, stop - n);
            n = stop;
        }
    }
    GK_CUDA(cudaEventRecord(e1, b->stream));
    GK_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    GK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return (double)ms;
}

// r_b = max_{r < D} |V[r, b] - P[r, b]| for every instance b, as the bit pattern of a non-negative
// double (the unsigned order of those patterns is the order of the values); a non-finite
// difference counts as +inf.  Block (32, 8): 32 consecutive instances, rows strided over y.
__global__ void k_period_residual(const double *__restrict__ V, const double *__restrict__ P, long long D,
                                  long long Bs, int B, unsigned long long *__restrict__ out) {
    const int b = blockIdx.x * 32 + threadIdx.x;
    if (b >= B) return;
    double m = 0.0;
    for (long long r = (long long)blockIdx.y * blockDim.y + threadIdx.y; r < D; r += (long long)gridDim.y * blockDim.y) {
        double d = fabs(V[r * Bs + b] - P[r * Bs + b]);
        if (d != d) d = INFINITY;
        m = d > m ? d : m;
    }
    if (m > 0.0) atomicMax(out + b, (unsigned long long)__double_as_longlong(m));
}

}  // namespace
}  // namespace gk

extern "C" gksl_status gksl_batch_propagate(gksl_batch *b, const long long *spp, const long long *n_steps,
                                            long long correction_every, double *seconds) {
    return bguarded(b, [&] {
        NvtxRange r("gksl_batch_propagate");
        double ms = batch_advance(b, spp, n_steps, correction_every);
        if (seconds) *seconds = ms * 1e-3;
    });
}

extern "C" gksl_status gksl_batch_asymptotic(gksl_batch *b, const long long *spp, long long transient,
                                             long long max_periods, double tol, long long correction_every,
                                             double *residual, long long *periods) {
    return bguarded(b, [&] {
        NvtxRange r("gksl_batch_asymptotic");
        GK_REQUIRE(spp && residual && transient >= 0 && max_periods >= 1 && tol >= 0.0, GKSL_ERR_ARG,
                   "steps_per_period and residual required, transient >= 0, max_periods >= 1, tol >= 0");
        const size_t ng = b->groups.size();
        std::vector<long long> per(spp, spp + ng), none(ng, 0);
        for (size_t g = 0; g < ng; ++g) GK_REQUIRE(per[g] > 0, GKSL_ERR_ARG, "steps_per_period > 0 required");
        if (transient > 0) {
            std::vector<long long> n(ng);
            for (size_t g = 0; g < ng; ++g) n[g] = per[g] * transient;
            batch_advance(b, per.data(), n.data(), correction_every);
        }
        std::vector<double> res((size_t)b->n_instances, 0.0);
        long long k = 0;
        for (;;) {
            for (auto &G : b->groups) {
                const size_t n = (size_t)((G.D + 1) * G.Bs);
                if (G.Vprev.n < n) G.Vprev.alloc(n);
                if (G.resid.n < (size_t)G.B) G.resid.alloc((size_t)G.B);
                GK_CUDA(cudaMemcpyAsync(G.Vprev.p, G.V64.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, b->stream));
                GK_CUDA(cudaMemsetAsync(G.resid.p, 0, sizeof(unsigned long long) * G.B, b->stream));
            }
            batch_advance(b, per.data(), per.data(), correction_every);
            ++k;
            double worst = 0.0;
            for (size_t g = 0; g < ng; ++g) {
                Group &G = b->groups[g];
                const long long ry = std::min<long long>((G.D + 7) / 8, 1024);
                k_period_residual<<<dim3((unsigned)((G.B + 31) / 32), (unsigned)ry), dim3(32, 8), 0, b->stream>>>(
                    G.V64.p, G.Vprev.p, G.D, G.Bs, G.B, G.resid.p);
                GK_LAUNCH_CHECK();
                std::vector<unsigned long long> bits((size_t)G.B);
                GK_CUDA(cudaMemcpyAsync(bits.data(), G.resid.p, sizeof(unsigned long long) * G.B,
                                        cudaMemcpyDeviceToHost, b->stream));
                GK_CUDA(cudaStreamSynchronize(b->stream));
                for (int i = 0; i < G.B; ++i) {
                    double x;
                    std::memcpy(&x, &bits[(size_t)i], sizeof(double));
                    res[(size_t)(b->first_instance[g] + i)] = x;
                    worst = std::max(worst, x);
                }
            }
            if (worst <= tol || k >= max_periods) break;
        }
        std::memcpy(residual, res.data(), sizeof(double) * res.size());
        if (periods) *periods = transient + k;
    });
}

extern "C" gksl_status gksl_batch_get_state(gksl_batch *b, int instance, double *v) {
    return bguarded(b, [&] {
        GK_REQUIRE(v && instance >= 0 && instance < b->n_instances, GKSL_ERR_ARG, "bad instance or null v");
        size_t gi = 0;
        while (gi + 1 < b->groups.size() && instance >= b->first_instance[gi + 1]) ++gi;
        Group &G = b->groups[gi];
        DBuf<double> col((size_t)G.D);
        k_column<<<grid_for(G.D, 256), 256, 0, b->stream>>>(G.V64.p, G.D, (int)G.Bs, instance - b->first_instance[gi],
                                                            col.p);
        GK_LAUNCH_CHECK();
        copy_out(v, col.p, sizeof(double) * G.D, b->stream);
        GK_CUDA(cudaStreamSynchronize(b->stream));
    });
}

extern "C" gksl_status gksl_batch_set_scan(gksl_batch *b, int component, const double *theta_b) {
    return bguarded(b, [&] {
        GK_REQUIRE(component >= 0 && component < GKSL_MAX_H0 && theta_b, GKSL_ERR_ARG,
                   "component index out of range or null theta_b");
        std::vector<double> th((size_t)b->n_instances);
        GK_CUDA(cudaMemcpy(th.data(), theta_b, sizeof(double) * th.size(), cudaMemcpyDefault));
        for (double x : th) GK_REQUIRE(std::isfinite(x), GKSL_ERR_ARG, "theta_b must be finite");
        for (size_t gi = 0; gi < b->groups.size(); ++gi) {
            Group &G = b->groups[gi];
            gksl_ctx *c = G.ctx;
            GK_REQUIRE(c->has_h0[component], GKSL_ERR_ARG, "the scanned component is not set in every group");
            const CsrR &q = c->QH0[component];
            CsrR &m = G.m[3];
            m.rows = q.rows;
            m.cols = q.cols;
            m.nnz = q.nnz;
            m.rowptr.alloc((size_t)q.rows + 1);
            m.col.alloc((size_t)std::max(1LL, q.nnz));
            m.val.alloc((size_t)std::max(1LL, q.nnz));
            GK_CUDA(cudaMemcpyAsync(m.rowptr.p, q.rowptr.p, sizeof(int) * (q.rows + 1), cudaMemcpyDeviceToDevice,
                                    b->stream));
            if (q.nnz > 0) {
                GK_CUDA(cudaMemcpyAsync(m.col.p, q.col.p, sizeof(int) * q.nnz, cudaMemcpyDeviceToDevice, b->stream));
                GK_CUDA(cudaMemcpyAsync(m.val.p, q.val.p, sizeof(double) * q.nnz, cudaMemcpyDeviceToDevice, b->stream));
            }
            G.mf[3].alloc((size_t)std::max(1LL, q.nnz));
            if (q.nnz > 0) {
                k_f2<<<grid_for(q.nnz, 256), 256, 0, b->stream>>>(m.val.p, G.mf[3].p, q.nnz);
                GK_LAUNCH_CHECK();
            }
            // instance b uses theta_b in place of the context's theta_k: coefficient theta_b - theta_k
            std::vector<double> s((size_t)G.B);
            std::vector<float> sf((size_t)G.B);
            for (int i = 0; i < G.B; ++i) {
                s[i] = th[b->first_instance[gi] + i] - c->h0[component].weight;
                sf[i] = (float)s[i];
            }
            G.S.alloc((size_t)G.B);
            G.Sf.alloc((size_t)G.B);
            GK_CUDA(cudaMemcpy(G.S.p, s.data(), sizeof(double) * G.B, cudaMemcpyHostToDevice));
            GK_CUDA(cudaMemcpy(G.Sf.p, sf.data(), sizeof(float) * G.B, cudaMemcpyHostToDevice));
            G.nch = 4;
            build_pairs(G, b->stream);
        }
        GK_CUDA(cudaStreamSynchronize(b->stream));
        clear_batch_graphs(b);
        b->tuned = false;
    });
}

extern "C" gksl_status gksl_batch_group_stats(gksl_batch *b, int group, long long *rows, int *instances,
                                              long long *channel_entries, long long *pair_entries, int *path) {
    return bguarded(b, [&] {
        GK_REQUIRE(group >= 0 && group < (int)b->groups.size(), GKSL_ERR_ARG, "bad group");
        const Group &G = b->groups[group];
        if (rows) *rows = G.D;
        if (instances) *instances = G.B;
        if (pair_entries) *pair_entries = G.pnnz;
        if (path) *path = G.pairs ? 2 : (G.vec4 ? 0 : 1);
        if (channel_entries) {
            long long n = 0;
            for (int c = 0; c < G.nch; ++c) n += G.m[c].nnz;
            *channel_entries = n;
        }
    });
}

extern "C" gksl_status gksl_batch_info(gksl_batch *b, int group, int *instances_per_lane, double *tuned_us_per_step) {
    return bguarded(b, [&] {
        GK_REQUIRE(group >= 0 && group < (int)b->groups.size(), GKSL_ERR_ARG, "bad group");
        // 4 for the 16-byte gather path (4 consecutive instances per lane)
        if (instances_per_lane) *instances_per_lane = b->groups[group].vec4 ? 4 : b->groups[group].ipl;
        if (tuned_us_per_step) *tuned_us_per_step = b->groups[group].tuned_us;
    });
}
