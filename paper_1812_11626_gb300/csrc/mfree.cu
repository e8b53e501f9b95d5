// Matrix-free RK4 stages: Q(t) v + K applied without an assembled Q.
//
// By Eq. 6 and Eq. 8 the unfolded right-hand side is the Lindbladian read in the generator
// basis, w_s = Tr(F_s L_t(rho)) with rho = 1/N + sum_m v_m F_m, and Eq. 1 gives
//   L_t(rho) = -i[H(t), rho] - {Gamma, rho} + sum_p L'_p rho L'_p^+,
//   H(t) = H0 + (eps(t) - E) H1,  Gamma = 1/2 sum_p gamma_p L_p^+ L_p,  L'_p = sqrt(gamma_p) L_p,
// where H0 already holds sum_k theta_k H0_k + E H1.  For banded operators every term is a short
// stencil on rho, so a stage needs only O(N) operator data (the operators' diagonals) and the
// state: the structure constants of Eq. 5 are applied implicitly, entry by entry, which is the
// paper's "compute the tensor elements on the fly" (Sec. IV step 2.2) carried through to the
// propagation.
//
// Scaled variables: rho' = sqrt(2) rho has rho'_ab = v_S(a,b) - i v_J(a,b) for a < b, and the
// outputs are w_S = Re X'_jk, w_J = -Im X'_jk with X' = L_t(rho') (L_t is linear).  The
// diagonal generators D^l mix all diagonal entries (the D^l reading of the Sec. II list):
//   rho_jj = 1/N + sum_l v_{D^l} (D^l)_jj,   w_{D^l} = sum_j (D^l)_jj X_jj.
// Both maps are linear and the RK4 updates are linear, so during a run of steps the D part of
// every state-sized vector y is carried as its diagonal image g_j = sqrt(2) sum_l y_l (D^l)_jj
// (rho'_jj = sqrt(2)/N + g_j) and updated entry by entry with X'_jj, the image of the stage
// derivative (Tr L_t(rho) = 0, so the image of w is X'_jj itself).  Prefix sums over the N
// diagonal entries convert the D coefficients of v to the image at the start of a run of steps
// (k_mf_prep) and back at its end (k_mf_post), which also removes the rounding drift of the
// image's trace.
//
// FP32 stages.  The dimer's diagonals are large (U n(n-1)/2 ~ 2.5e3 in H, n1 - n2 ~ 1e2 in L)
// and, term by term, -i[H, rho] and L rho L^+ - 1/2{L^+L, rho} cancel them against each other
// for j ~ k; in FP32 that loses ~6 bits.  The FP32 kernel therefore evaluates the same X' in a
// rearranged form where every such cancellation is an explicit difference of diagonal entries
// taken from hi/lo-split values, and the remaining couplings are combined in FP64 on the host:
//   X_jk = C_jk rho_jk + sum_{d!=0} R_(j,j+d) rho_(j+d,k) + sum_{d!=0} rho_(j,k+d) conj(R_(k,k+d))
//        + sum_p [ conj(delta_p) U_p - delta_p T_p(j,k) + sum_{d!=0} L'_(j,j+d) T_p(j+d,k) ],
//   R_(j,a) = -i H(t)_(j,a) + sum_p [ L'_(j,a) conj(L'_jj) - 1/2 (L'^+ L')_(j,a) ],   a != j,
//   delta_p = L'_kk - L'_jj,  U_p = sum_{a!=j} L'_(j,a) rho_(a,k),  T_p(a,k) = sum_{b!=k} rho_(a,b) conj(L'_(k,b)),
//   C_jk = -i (H_jj - H_kk) - 1/2 sum_p (off_pj + off_pk) + sum_p [ -1/2 |delta_p|^2 + i Im(L'_jj conj(delta_p)) ],
// with off_pj = sum_{i!=j} |L'_(i,j)|^2.  Expanding the right-hand side term by term gives back
// L_t(rho)_jk exactly.
//
// One stage is one launch over the tiles of the upper triangle j <= k of rho (32 x 32 outputs
// each, 256 threads, 4 rows of one column per thread).  A block first issues every global load
// it needs (the rho' tile with its halo, the band coefficients of its rows and columns, and the
// operands of its own stage updates), then evaluates X' from shared memory and applies the RK4
// stage update to the two generators of every pair (j < k) and to the diagonal image (j = k).
#include <algorithm>
#include <cmath>
#include <complex>

#include "internal.cuh"
#include "stage.cuh"

namespace gk {

namespace {

constexpr int kTJ = 32, kTK = 32;               // tile rows (j) and columns (k)
constexpr int kThreads = 256;
constexpr int kRJ = kTJ / (kThreads / 32);      // output rows per thread (one column each)

template <typename T>
struct Cx;
template <>
struct Cx<double> { using t = double2; };
template <>
struct Cx<float> { using t = float2; };

struct MfArgs {
    int N;
    long long P2;
    int P;
    const int *tiles;
    const double *eps_tab;
    const long long *base;
    long long local;
    HConst hc;
    double diag0;   // sqrt(2)/N: the F0/N part of rho on the diagonal image (computed on the host)
    float diag0f;
};

// the vectors of one stage: input y, state v (FP64 master v64), next input yn, accumulator, and
// the diagonal images of the same four (gi: image of y)
template <typename T>
struct MfVec {
    const T *y;
    T *v;
    double *v64;
    T *yn, *acc;
    const T *gi;
    T *gv;
    double *gv64;
    T *gyn, *gacc;
};

// lexicographic index of the pair a < b in 32-bit arithmetic (the matrix-free form keeps
// N <= 32768, so D < 2^30)
__device__ inline int pair_start(int N, int a) { return a * N - ((a * (a + 1)) >> 1) - a - 1; }
__device__ inline int pair_of(int N, int a, int b) { return pair_start(N, a) + b; }

// block-wide inclusive prefix sum of one value per thread; *total receives the block sum
__device__ inline double block_incl_scan(double x, double *sh, double *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        double t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    double before = 0.0, all = 0.0;
    for (int i = 0; i < kThreads / 32; ++i) {
        double s = sh[i];
        if (i < w) before += s;
        all += s;
    }
    __syncthreads();
    *total = all;
    return x + before;
}

// image g_j = sqrt(2) (sum_{l>j} v_l c_l - j v_j c_j) of the D coefficients of v (one block);
// g32 (may be null) receives an FP32 copy
__global__ void __launch_bounds__(kThreads) k_mf_prep(int N, long long P2, const double *__restrict__ v,
                                                       double *__restrict__ g, float *__restrict__ g32) {
    __shared__ double sh[kThreads / 32];
    const int S = (N + kThreads - 1) / kThreads;
    const int lo = min(N, (int)threadIdx.x * S), hi = min(N, lo + S);
    double usum = 0.0;
    for (int j = lo; j < hi; ++j) usum += j >= 1 ? v[2 * P2 + j - 1] * cl(j) : 0.0;
    double total;
    const double incl = block_incl_scan(usum, sh, &total);
    double carry = total - incl;   // sum over later segments
    for (int j = hi - 1; j >= lo; --j) {
        const double u = j >= 1 ? v[2 * P2 + j - 1] * cl(j) : 0.0;
        const double x = M_SQRT2 * (carry - (double)j * u);
        g[j] = x;
        if (g32) g32[j] = (float)x;
        carry += u;
    }
}

// D coefficients v_l = (sum_{j<l} g_j - l g_l) c_l / sqrt(2) back from the image (one block);
// v32 (may be null) receives the FP32 mirror
__global__ void __launch_bounds__(kThreads) k_mf_post(int N, long long P2, const double *__restrict__ g,
                                                       double *__restrict__ v, float *__restrict__ v32) {
    __shared__ double sh[kThreads / 32];
    const int S = (N + kThreads - 1) / kThreads;
    const int lo = min(N, (int)threadIdx.x * S), hi = min(N, lo + S);
    double loc = 0.0;
    for (int j = lo; j < hi; ++j) loc += g[j];
    double total;
    double run = block_incl_scan(loc, sh, &total) - loc;
    for (int j = lo; j < hi; ++j) {
        const double x = g[j];
        if (j >= 1) {
            const double w = (run - (double)j * x) * cl(j) * M_SQRT1_2;
            v[2 * P2 + j - 1] = w;
            if (v32) v32[2 * P2 + j - 1] = (float)w;
        }
        run += x;
    }
}

// rho' on a tile and its halo of BT rows and columns: all loads first, then the stores.  The
// 32 central columns of every tile row go one per lane, with the pair index advancing by one
// along the row; the 2 BT halo columns of all rows are a second, flat pass.
template <int BT, typename T>
__device__ inline typename Cx<T>::t rho_entry(const MfArgs &a, const MfVec<T> &q, int ai, int bi, int rowstart,
                                              T diag0) {
    typename Cx<T>::t val;
    val.x = T(0);
    val.y = T(0);
    const int N = a.N;
    if (ai >= 0 && ai < N && bi >= 0 && bi < N) {
        if (ai < bi) {
            const int p = rowstart + bi;
            val.x = q.y[p];
            val.y = -q.y[a.P2 + p];
        } else if (ai > bi) {
            const int p = pair_of(N, bi, ai);
            val.x = q.y[p];
            val.y = q.y[a.P2 + p];
        } else {
            val.x = diag0 + q.gi[ai];
        }
    }
    return val;
}

template <int BT, typename T>
__device__ inline void load_rho(typename Cx<T>::t *rho, const MfArgs &a, const MfVec<T> &q, int j0, int k0) {
    using C = typename Cx<T>::t;
    constexpr int RW = kTK + 2 * BT, RH = kTJ + 2 * BT;
    constexpr int IT = (RH + kThreads / 32 - 1) / (kThreads / 32);     // central part, rows per warp
    constexpr int nh = RH * 2 * BT, IH = (nh + kThreads - 1) / kThreads;  // halo columns
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const T diag0 = sizeof(T) == 8 ? (T)a.diag0 : (T)a.diag0f;
    C val[IT], hal[IH];
#pragma unroll
    for (int it = 0; it < IT; ++it) {
        const int ra = w + it * (kThreads / 32);
        const int ai = j0 - BT + ra;
        val[it].x = T(0);
        val[it].y = T(0);
        if (ra < RH) val[it] = rho_entry<BT, T>(a, q, ai, k0 + lane, pair_start(a.N, ai), diag0);
    }
#pragma unroll
    for (int it = 0; it < IH; ++it) {
        const int e = threadIdx.x + it * kThreads;
        const int ra = e / (2 * BT), h = e - ra * (2 * BT);
        const int cb = h < BT ? h : kTK + h;       // columns [0, BT) and [BT + 32, RW)
        const int ai = j0 - BT + ra;
        hal[it].x = T(0);
        hal[it].y = T(0);
        if (e < nh) hal[it] = rho_entry<BT, T>(a, q, ai, k0 - BT + cb, pair_start(a.N, ai), diag0);
    }
#pragma unroll
    for (int it = 0; it < IT; ++it) {
        const int ra = w + it * (kThreads / 32);
        if (ra < RH) rho[ra * RW + BT + lane] = val[it];
    }
#pragma unroll
    for (int it = 0; it < IH; ++it) {
        const int e = threadIdx.x + it * kThreads;
        const int ra = e / (2 * BT), h = e - ra * (2 * BT);
        const int cb = h < BT ? h : kTK + h;
        if (e < nh) rho[ra * RW + cb] = hal[it];
    }
}

// the thread's outputs (rows i0 + i of column c): pair generators for j < k, the diagonal image
// for j = k; operands loaded up front
template <int STAGE, typename T>
struct TileOut {
    int r[kRJ];           // pair index, or -2 - j for the diagonal j, or -1
    EpIn<T> s[kRJ], jv[kRJ];
    __device__ void prepare(const MfArgs &a, const MfVec<T> &q, int j0, int k0, int i0, int c) {
        const int k = k0 + c;
#pragma unroll
        for (int i = 0; i < kRJ; ++i) {
            const int j = j0 + i0 + i;
            r[i] = -1;
            if (j >= a.N || k >= a.N || j > k) continue;
            if (j < k) {
                r[i] = pair_of(a.N, j, k);
                epi_load<STAGE, T>(r[i], q.v, q.v64, q.acc, s[i]);
                epi_load<STAGE, T>(a.P2 + r[i], q.v, q.v64, q.acc, jv[i]);
            } else {
                r[i] = -2 - j;
                epi_load<STAGE, T>(j, q.gv, q.gv64, q.gacc, s[i]);
            }
        }
    }
    template <typename C>
    __device__ void store(const MfArgs &a, const MfVec<T> &q, const C (&X)[kRJ]) const {
#pragma unroll
        for (int i = 0; i < kRJ; ++i) {
            if (r[i] >= 0) {
                epi_store<STAGE, T>(r[i], X[i].x, s[i], q.v, q.v64, q.yn, q.acc, a.hc);
                epi_store<STAGE, T>(a.P2 + r[i], -X[i].y, jv[i], q.v, q.v64, q.yn, q.acc, a.hc);
            } else if (r[i] <= -2) {
                epi_store<STAGE, T>(-2 - r[i], X[i].x, s[i], q.gv, q.gv64, q.gyn, q.gacc, a.hc);
            }
        }
    }
};

// ------------------------------------------------------------------ FP64 stages

template <typename T>
struct MfOps {
    const T *h0, *h1, *g, *l;   // interleaved complex diagonals
};

// shared-memory geometry of one instantiation (half-bandwidths of H, Gamma, L)
template <int BH, int BG, int BL>
struct Geo {
    static constexpr int BR = BH > BG ? BH : BG;          // reach of the H and Gamma terms
    static constexpr int BT = BR > BL ? BR : BL;          // halo of the rho tile
    static constexpr int RW = kTK + 2 * BT, RH = kTJ + 2 * BT;
    static constexpr int TH = kTJ + 2 * BL;               // rows of rho L'^+ kept
    static constexpr int WH = 2 * BH + 1, WG = 2 * BG + 1, WL = 2 * BL + 1;
    static constexpr int n_rho = RH * RW, n_t = TH * kTK;
    static constexpr int n_coef = (kTJ + kTK) * (WH + WG + WL);
    static constexpr int total = n_rho + n_t + n_coef;    // complex entries
};

// c += coef * p for the H term of a row (-i h p), the Gamma term of a row (-g p), and the
// column forms (p * i conj(h)) and (-p * conj(g)); REAL skips the imaginary coefficient parts.
template <bool REAL, typename C>
__device__ inline void row_h(C &x, const C &h, const C &p) {
    x.x += h.x * p.y;
    x.y -= h.x * p.x;
    if (!REAL) { x.x += h.y * p.x; x.y += h.y * p.y; }
}
template <bool REAL, typename C>
__device__ inline void row_g(C &x, const C &g, const C &p) {
    x.x -= g.x * p.x;
    x.y -= g.x * p.y;
    if (!REAL) { x.x += g.y * p.y; x.y -= g.y * p.x; }
}
template <bool REAL, typename C>
__device__ inline void col_h(C &x, const C &h, const C &p) {
    x.x -= p.y * h.x;
    x.y += p.x * h.x;
    if (!REAL) { x.x += p.x * h.y; x.y += p.y * h.y; }
}
template <bool REAL, typename C>
__device__ inline void col_g(C &x, const C &g, const C &p) {
    x.x -= p.x * g.x;
    x.y -= p.y * g.x;
    if (!REAL) { x.x -= p.y * g.y; x.y += p.x * g.y; }
}

// stage the coefficient rows (tile rows then tile columns) of a band array of width W, plus
// alpha * src_t (ROT: -i alpha * src_t) when src_t is given
template <int W, bool ROT, typename T>
__device__ inline void load_band(typename Cx<T>::t *dst, const T *src, const T *src_t, T alpha, int N, int j0,
                                 int k0, long long chan_off) {
    using C = typename Cx<T>::t;
    constexpr int n = (kTJ + kTK) * W;
    constexpr int IT = (n + kThreads - 1) / kThreads;
    C val[IT];
#pragma unroll
    for (int it = 0; it < IT; ++it) {
        const int e = threadIdx.x + it * kThreads;
        const int i = e / W, d = e - i * W;
        const int row = i < kTJ ? j0 + i : k0 + (i - kTJ);
        val[it].x = T(0);
        val[it].y = T(0);
        if (e < n && row < N) {
            const long long o = 2 * ((chan_off + row) * W + d);
            val[it].x = src[o];
            val[it].y = src[o + 1];
            if (src_t) {
                if (ROT) {
                    val[it].x += alpha * src_t[o + 1];
                    val[it].y -= alpha * src_t[o];
                } else {
                    val[it].x += alpha * src_t[o];
                    val[it].y += alpha * src_t[o + 1];
                }
            }
        }
    }
#pragma unroll
    for (int it = 0; it < IT; ++it) {
        const int e = threadIdx.x + it * kThreads;
        if (e < n) dst[e] = val[it];
    }
}

template <int STAGE, int BH, int BG, int BL, bool REAL, typename T>
__global__ void __launch_bounds__(kThreads, BL == 1 ? 3 : 2) k_mf_stage(MfArgs a, MfOps<T> op, MfVec<T> q) {
    using G = Geo<BH, BG, BL>;
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *rho = reinterpret_cast<C *>(smem_raw);
    C *Tb = rho + G::n_rho;
    C *hrow = Tb + G::n_t;
    C *hcol = hrow + kTJ * G::WH;
    C *grow = hcol + kTK * G::WH;
    C *gcol = grow + kTJ * G::WG;
    C *lrow = gcol + kTK * G::WG;
    C *lcol = lrow + kTJ * G::WL;

    const int N = a.N, tid = threadIdx.x;
    const int tj = a.tiles[2 * blockIdx.x], tk = a.tiles[2 * blockIdx.x + 1];
    const int j0 = tj * kTJ, k0 = tk * kTK;
    const int c = tid & 31, i0 = (tid >> 5) * kRJ;
    const T alpha = (T)a.eps_tab[3 * (*a.base + a.local) + eps_slot<STAGE>()];

    TileOut<STAGE, T> out;
    out.prepare(a, q, j0, k0, i0, c);
    load_rho<G::BT, T>(rho, a, q, j0, k0);
    load_band<G::WH, false, T>(hrow, op.h0, op.h1, alpha, N, j0, k0, 0);
    load_band<G::WG, false, T>(grow, op.g, nullptr, T(0), N, j0, k0, 0);
    if (a.P > 0) load_band<G::WL, false, T>(lrow, op.l, nullptr, T(0), N, j0, k0, 0);
    __syncthreads();

    C X[kRJ];
#pragma unroll
    for (int i = 0; i < kRJ; ++i) { X[i].x = T(0); X[i].y = T(0); }

    // row terms -i H rho - Gamma rho down the column c, and column terms i rho H - rho Gamma
    // along the rows of this thread.  The row and column taps at offset 0 act on the same
    // entry rho_jk, so they are applied once with the merged coefficients
    // (h_jj - conj(h_kk)) and (g_jj + conj(g_kk)) (as row taps).
    {
        C hc[G::WH], gc[G::WG];
#pragma unroll
        for (int d = 0; d < G::WH; ++d) hc[d] = hcol[c * G::WH + d];
#pragma unroll
        for (int d = 0; d < G::WG; ++d) gc[d] = gcol[c * G::WG + d];
        C p[kRJ + 2 * G::BR];
#pragma unroll
        for (int t = 0; t < kRJ + 2 * G::BR; ++t) p[t] = rho[(i0 + G::BT - G::BR + t) * G::RW + c + G::BT];
#pragma unroll
        for (int i = 0; i < kRJ; ++i) {
#pragma unroll
            for (int d = -BH; d <= BH; ++d) {
                C h = hrow[(i0 + i) * G::WH + d + BH];
                if (d == 0) {
                    h.x -= hc[BH].x;
                    if (!REAL) h.y += hc[BH].y;
                }
                row_h<REAL>(X[i], h, p[i + G::BR + d]);
            }
#pragma unroll
            for (int d = -BG; d <= BG; ++d) {
                C g = grow[(i0 + i) * G::WG + d + BG];
                if (d == 0) {
                    g.x += gc[BG].x;
                    if (!REAL) g.y -= gc[BG].y;
                }
                row_g<REAL>(X[i], g, p[i + G::BR + d]);
            }
        }
#pragma unroll
        for (int i = 0; i < kRJ; ++i) {
            const C *rr = rho + (i0 + i + G::BT) * G::RW + c + G::BT;
#pragma unroll
            for (int d = -G::BR; d <= G::BR; ++d) {
                if (d == 0) continue;   // merged into the row taps above
                const C pv = rr[d];
                if (d >= -BH && d <= BH) col_h<REAL>(X[i], hc[d + BH], pv);
                if (d >= -BG && d <= BG) col_g<REAL>(X[i], gc[d + BG], pv);
            }
        }
    }
    // jump terms: L' rho L'^+ per channel, as L' (rho L'^+)
    for (int ch = 0; ch < a.P; ++ch) {
        if (ch > 0) {
            __syncthreads();   // previous channel done with lrow, lcol, Tb
            load_band<G::WL, false, T>(lrow, op.l, nullptr, T(0), N, j0, k0, (long long)ch * N);
            __syncthreads();
        }
        // Tb[ta][c] = sum_d rho'_(a, k+d) conj(L'_(k, k+d)), rows a = j0 - BL + ta
        for (int e = tid; e < G::n_t; e += kThreads) {
            const int ta = e / kTK, cc = e - ta * kTK;
            const C *rr = rho + (ta + G::BT - BL) * G::RW + cc + G::BT;
            C t;
            t.x = T(0);
            t.y = T(0);
#pragma unroll
            for (int d = -BL; d <= BL; ++d) {
                const C pv = rr[d];
                const C lv = lcol[cc * G::WL + d + BL];
                t.x += pv.x * lv.x;
                t.y += pv.y * lv.x;
                if (!REAL) { t.x += pv.y * lv.y; t.y -= pv.x * lv.y; }
            }
            Tb[e] = t;
        }
        __syncthreads();
        C qv[kRJ + 2 * BL];
#pragma unroll
        for (int t = 0; t < kRJ + 2 * BL; ++t) qv[t] = Tb[(i0 + t) * kTK + c];
#pragma unroll
        for (int i = 0; i < kRJ; ++i) {
#pragma unroll
            for (int d = -BL; d <= BL; ++d) {
                const C lv = lrow[(i0 + i) * G::WL + d + BL];
                const C tv = qv[i + BL + d];
                X[i].x += lv.x * tv.x;
                X[i].y += lv.x * tv.y;
                if (!REAL) { X[i].x -= lv.y * tv.y; X[i].y += lv.y * tv.x; }
            }
        }
    }
    out.store(a, q, X);
}

// ------------------------------------------------------------------ FP32 stages

struct MfOps32 {
    const float *r;     // [N][WR] complex: R_(j, j+d) without the drive term, centre 0
    const float *h1o;   // [N][WR] complex: H1_(j, j+d) off the diagonal, centre 0
    const float *dg;    // [N][8]: H0_jj hi, lo, H1_jj hi, lo, 1/2 sum_p off_pj
    const float *lo;    // [P][N][WL] complex: L'_p off the diagonal, centre 0
    const float *ld;    // [P][N][4]: L'_p,jj: re hi, re lo, im hi, im lo
};

template <int BR, int BL>
struct Geo32 {
    static constexpr int BT = BR > BL ? BR : BL;
    static constexpr int RW = kTK + 2 * BT, RH = kTJ + 2 * BT, TH = kTJ + 2 * BL;
    static constexpr int WR = 2 * BR + 1, WL = 2 * BL + 1;
    static constexpr int n_rho = RH * RW, n_t = TH * kTK;
    static constexpr int n_r = (kTJ + kTK) * WR, n_l = (kTJ + kTK) * WL;
    static constexpr int n_dg = (kTJ + kTK) * 3, n_ld = (kTJ + kTK) * 2;   // float2 units (6 and 4 floats a row)
    static constexpr int total = n_rho + n_t + n_r + n_l + n_dg + n_ld;
};

__device__ inline float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ inline float2 cmulc(float2 a, float2 b) { return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); }
__device__ inline void cadd(float2 &x, float2 v) { x.x += v.x; x.y += v.y; }

// stage `W` floats per row (tile rows then columns) from a [N][S] float array
template <int W, int S>
__device__ inline void load_rows(float *dst, const float *src, int N, int j0, int k0, long long chan_off) {
    constexpr int n = (kTJ + kTK) * W;
    constexpr int IT = (n + kThreads - 1) / kThreads;
    float val[IT];
#pragma unroll
    for (int it = 0; it < IT; ++it) {
        const int e = threadIdx.x + it * kThreads;
        const int i = e / W, f = e - i * W;
        const int row = i < kTJ ? j0 + i : k0 + (i - kTJ);
        val[it] = (e < n && row < N && f < S) ? src[(chan_off + row) * S + f] : 0.f;
    }
#pragma unroll
    for (int it = 0; it < IT; ++it) {
        const int e = threadIdx.x + it * kThreads;
        if (e < n) dst[e] = val[it];
    }
}

template <int STAGE, int BR, int BL>
__global__ void __launch_bounds__(kThreads, BL == 1 ? 4 : 2) k_mf_stage32(MfArgs a, MfOps32 op, MfVec<float> q) {
    using G = Geo32<BR, BL>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *rho = reinterpret_cast<float2 *>(smem_raw);
    float2 *Tb = rho + G::n_rho;
    float2 *rr = Tb + G::n_t;                                    // R(t) of the tile rows, then columns
    float2 *ll = rr + G::n_r;                                    // L'_p off-diagonal, rows then columns
    float *dg = reinterpret_cast<float *>(ll + G::n_l);          // [64][6]
    float *ld = dg + 6 * (kTJ + kTK);                            // [64][4]

    const int N = a.N, tid = threadIdx.x;
    const int tj = a.tiles[2 * blockIdx.x], tk = a.tiles[2 * blockIdx.x + 1];
    const int j0 = tj * kTJ, k0 = tk * kTK;
    const int c = tid & 31, i0 = (tid >> 5) * kRJ;
    const float alpha = (float)a.eps_tab[3 * (*a.base + a.local) + eps_slot<STAGE>()];

    TileOut<STAGE, float> out;
    out.prepare(a, q, j0, k0, i0, c);
    load_rho<G::BT, float>(rho, a, q, j0, k0);
    load_band<G::WR, true, float>(rr, op.r, op.h1o, alpha, N, j0, k0, 0);
    load_rows<6, 8>(dg, op.dg, N, j0, k0, 0);
    if (a.P > 0) {
        load_band<G::WL, false, float>(ll, op.lo, nullptr, 0.f, N, j0, k0, 0);
        load_rows<4, 4>(ld, op.ld, N, j0, k0, 0);
    }
    __syncthreads();
    // T(a, k) = sum_{b != k} rho'_(a,b) conj(L'_(k,b)) of channel 0, rows a = j0 - BL + ta
    auto build_t = [&]() {
        for (int e = tid; e < G::n_t; e += kThreads) {
            const int ta = e / kTK, cc = e - ta * kTK;
            const float2 *rw = rho + (ta + G::BT - BL) * G::RW + cc + G::BT;
            const float2 *lc = ll + (kTJ + cc) * G::WL;
            float2 t = make_float2(0.f, 0.f);
#pragma unroll
            for (int d = -BL; d <= BL; ++d) {
                if (d == 0) continue;
                cadd(t, cmulc(rw[d], lc[d + BL]));
            }
            Tb[e] = t;
        }
    };
    if (a.P > 0) {
        build_t();
        __syncthreads();
    }

    float2 X[kRJ];
#pragma unroll
    for (int i = 0; i < kRJ; ++i) X[i] = make_float2(0.f, 0.f);
    float2 p[kRJ + 2 * BR];   // rho' down column c
#pragma unroll
    for (int t = 0; t < kRJ + 2 * BR; ++t) p[t] = rho[(i0 + G::BT - BR + t) * G::RW + c + G::BT];

    // centre: -i (H_jj - H_kk) - 1/2 sum_p (off_pj + off_pk), differences of split values
    const float *dk = dg + 6 * (kTJ + c);
#pragma unroll
    for (int i = 0; i < kRJ; ++i) {
        const float *dj = dg + 6 * (i0 + i);
        const float dh = ((dj[0] - dk[0]) + (dj[1] - dk[1])) + alpha * ((dj[2] - dk[2]) + (dj[3] - dk[3]));
        cadd(X[i], cmul(make_float2(-(dj[4] + dk[4]), -dh), p[i + BR]));
    }
    // couplings off the centre: R down the column, conj(R) along the row
    const float2 *rc = rr + (kTJ + c) * G::WR;
#pragma unroll
    for (int i = 0; i < kRJ; ++i) {
        const float2 *rj = rr + (i0 + i) * G::WR;
        const float2 *rowp = rho + (i0 + i + G::BT) * G::RW + c + G::BT;
#pragma unroll
        for (int d = -BR; d <= BR; ++d) {
            if (d == 0) continue;
            cadd(X[i], cmul(rj[d + BR], p[i + BR + d]));
            cadd(X[i], cmulc(rowp[d], rc[d + BR]));
        }
    }
    // jump terms per channel
    for (int ch = 0; ch < a.P; ++ch) {
        if (ch > 0) {
            __syncthreads();
            load_band<G::WL, false, float>(ll, op.lo, nullptr, 0.f, N, j0, k0, (long long)ch * N);
            load_rows<4, 4>(ld, op.ld, N, j0, k0, (long long)ch * N);
            __syncthreads();
            build_t();
            __syncthreads();
        }
        float2 qv[kRJ + 2 * BL];
#pragma unroll
        for (int t = 0; t < kRJ + 2 * BL; ++t) qv[t] = Tb[(i0 + t) * kTK + c];
        const float *lk = ld + 4 * (kTJ + c);
#pragma unroll
        for (int i = 0; i < kRJ; ++i) {
            const float *lj = ld + 4 * (i0 + i);
            const float2 del = make_float2((lk[0] - lj[0]) + (lk[1] - lj[1]), (lk[2] - lj[2]) + (lk[3] - lj[3]));
            // centre: -1/2 |delta|^2 + i Im(L'_jj conj(delta))
            const float2 cj = make_float2(-0.5f * (del.x * del.x + del.y * del.y), lj[2] * del.x - lj[0] * del.y);
            cadd(X[i], cmul(cj, p[i + BR]));
            const float2 *lr = ll + (i0 + i) * G::WL;
            float2 U = make_float2(0.f, 0.f);
#pragma unroll
            for (int d = -BL; d <= BL; ++d) {
                if (d == 0) continue;
                cadd(U, cmul(lr[d + BL], p[i + BR + d]));
                cadd(X[i], cmul(lr[d + BL], qv[i + BL + d]));
            }
            cadd(X[i], cmulc(U, del));                                   // conj(delta) U
            const float2 dt = cmul(del, qv[i + BL]);                     // delta T(j,k)
            X[i].x -= dt.x;
            X[i].y -= dt.y;
        }
    }
    out.store(a, q, X);
}

// ------------------------------------------------------------------ dispatch

// the four stage launches of one step; images: 0 v, 1 yA, 2 yB, 3 acc
template <typename T, typename K1, typename K2, typename K3, typename K4, typename Ops>
void four_stages(K1 k1, K2 k2, K3 k3, K4 k4, const MfArgs &a, const Ops &op, unsigned grid, size_t sm,
                 cudaStream_t s, T *v, double *v64, T *ya, T *yb, T *acc, T *const *g, double *g64) {
    MfVec<T> q{v, v, v64, ya, acc, g[0], g[0], g64, g[1], g[3]};
    k1<<<grid, kThreads, sm, s>>>(a, op, q);
    q = MfVec<T>{ya, v, v64, yb, acc, g[1], g[0], g64, g[2], g[3]};
    k2<<<grid, kThreads, sm, s>>>(a, op, q);
    q = MfVec<T>{yb, v, v64, ya, acc, g[2], g[0], g64, g[1], g[3]};
    k3<<<grid, kThreads, sm, s>>>(a, op, q);
    q = MfVec<T>{ya, v, v64, nullptr, acc, g[1], g[0], g64, nullptr, g[3]};
    k4<<<grid, kThreads, sm, s>>>(a, op, q);
}

template <int BH, int BG, int BL, bool REAL>
struct Inst64 {
    using G = Geo<BH, BG, BL>;
    static size_t smem() { return sizeof(double2) * (size_t)G::total; }
    static void set_attributes() {
        const int b = (int)smem();
        GK_CUDA(cudaFuncSetAttribute(k_mf_stage<1, BH, BG, BL, REAL, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
        GK_CUDA(cudaFuncSetAttribute(k_mf_stage<2, BH, BG, BL, REAL, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
        GK_CUDA(cudaFuncSetAttribute(k_mf_stage<3, BH, BG, BL, REAL, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
        GK_CUDA(cudaFuncSetAttribute(k_mf_stage<4, BH, BG, BL, REAL, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
    }
    static void step(const MfArgs &a, const MfOps<double> &op, unsigned grid, cudaStream_t s, gksl_ctx *c) {
        MfBands &m = c->mf;
        double *g[4] = {m.img64[0].p, m.img64[1].p, m.img64[2].p, m.img64[3].p};
        four_stages<double>(k_mf_stage<1, BH, BG, BL, REAL, double>, k_mf_stage<2, BH, BG, BL, REAL, double>,
                            k_mf_stage<3, BH, BG, BL, REAL, double>, k_mf_stage<4, BH, BG, BL, REAL, double>, a, op,
                            grid, smem(), s, c->v.p, nullptr, c->yA.p, c->yB.p, c->acc.p, g, nullptr);
    }
};

template <int BR, int BL>
struct Inst32 {
    using G = Geo32<BR, BL>;
    static size_t smem() { return sizeof(float2) * (size_t)G::total; }
    static void set_attributes() {
        const int b = (int)smem();
        GK_CUDA(cudaFuncSetAttribute(k_mf_stage32<1, BR, BL>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
        GK_CUDA(cudaFuncSetAttribute(k_mf_stage32<2, BR, BL>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
        GK_CUDA(cudaFuncSetAttribute(k_mf_stage32<3, BR, BL>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
        GK_CUDA(cudaFuncSetAttribute(k_mf_stage32<4, BR, BL>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
    }
    static void step(const MfArgs &a, const MfOps32 &op, unsigned grid, cudaStream_t s, gksl_ctx *c) {
        MfBands &m = c->mf;
        float *g[4] = {m.img32[0].p, m.img32[1].p, m.img32[2].p, m.img32[3].p};
        four_stages<float>(k_mf_stage32<1, BR, BL>, k_mf_stage32<2, BR, BL>, k_mf_stage32<3, BR, BL>,
                           k_mf_stage32<4, BR, BL>, a, op, grid, smem(), s, c->v32.p, c->v.p, c->yA32.p, c->yB32.p,
                           c->acc32.p, g, m.img64[0].p);
    }
};

// the two instantiations: tridiagonal real operators (pentadiagonal Gamma), and any complex
// operators of half-bandwidth <= 4
using Narrow64 = Inst64<1, 2, 1, true>;
using Wide64 = Inst64<4, 8, 4, false>;
using Narrow32 = Inst32<2, 1>;
using Wide32 = Inst32<8, 4>;

int half_bandwidth(const Op &op) {
    int b = 0;
    for (int r = 0; r < (int)op.h_rowptr.size() - 1; ++r)
        for (int e = op.h_rowptr[r]; e < op.h_rowptr[r + 1]; ++e)
            if (op.h_re[e] != 0.0 || op.h_im[e] != 0.0) b = std::max(b, std::abs(op.h_col[e] - r));
    return b;
}

bool op_real(const Op &op) {
    for (double x : op.h_im)
        if (x != 0.0) return false;
    return true;
}

// add w * X into the band array [N][2B+1] (complex interleaved)
void add_band(std::vector<double> &band, int N, int B, const Op &op, std::complex<double> w) {
    const int W = 2 * B + 1;
    for (int r = 0; r < N; ++r)
        for (int e = op.h_rowptr[r]; e < op.h_rowptr[r + 1]; ++e) {
            const int d = op.h_col[e] - r;
            const std::complex<double> x = w * std::complex<double>(op.h_re[e], op.h_im[e]);
            band[2 * ((size_t)r * W + d + B)] += x.real();
            band[2 * ((size_t)r * W + d + B) + 1] += x.imag();
        }
}

template <typename T>
void upload(DBuf<T> &dst, const std::vector<double> &src, cudaStream_t s) {
    dst.alloc(src.size());
    std::vector<T> tmp(src.begin(), src.end());
    GK_CUDA(cudaMemcpyAsync(dst.p, tmp.data(), sizeof(T) * tmp.size(), cudaMemcpyHostToDevice, s));
    GK_CUDA(cudaStreamSynchronize(s));
}

// float pair (hi, lo) with hi + lo = x to ~2^-48 relative
void split(double x, double *out) {
    const float hi = (float)x;
    out[0] = hi;
    out[1] = (float)(x - (double)hi);
}

// FP32 stage data (see the FP32 paragraph at the top): from the FP64 bands h0, h1 (width BH)
// and L'_p (width BL, channel after channel)
void build_fp32(MfBands &m, int N, int BH, int BL, int BR, int P, const std::vector<double> &h0,
                const std::vector<double> &h1, const std::vector<double> &l, cudaStream_t s) {
    using cd = std::complex<double>;
    const int WH = 2 * BH + 1, WL = 2 * BL + 1, WR = 2 * BR + 1, WM = 4 * BL + 1;
    auto H0 = [&](int j, int d) { return cd(h0[2 * ((size_t)j * WH + d + BH)], h0[2 * ((size_t)j * WH + d + BH) + 1]); };
    auto H1 = [&](int j, int d) { return cd(h1[2 * ((size_t)j * WH + d + BH)], h1[2 * ((size_t)j * WH + d + BH) + 1]); };
    auto Lp = [&](int p, int j, int d) {
        const size_t o = 2 * (((size_t)p * N + j) * WL + d + BL);
        return cd(l[o], l[o + 1]);
    };
    std::vector<double> r((size_t)2 * N * WR, 0.0), h1o((size_t)2 * N * WR, 0.0), dg((size_t)8 * N, 0.0);
    std::vector<double> lo((size_t)2 * N * WL * std::max(P, 1), 0.0), ld((size_t)4 * N * std::max(P, 1), 0.0);
    for (int j = 0; j < N; ++j)
        for (int d = -BH; d <= BH; ++d) {
            if (d == 0) continue;
            const cd x = cd(0, -1) * H0(j, d);
            r[2 * ((size_t)j * WR + d + BR)] += x.real();
            r[2 * ((size_t)j * WR + d + BR) + 1] += x.imag();
            h1o[2 * ((size_t)j * WR + d + BR)] = H1(j, d).real();
            h1o[2 * ((size_t)j * WR + d + BR) + 1] = H1(j, d).imag();
        }
    std::vector<double> off((size_t)N, 0.0);
    for (int p = 0; p < P; ++p) {
        // M = L'^+ L' on the band |b - a| <= 2 BL: M_(a,b) = sum_i conj(L'_ia) L'_ib
        std::vector<cd> M((size_t)N * WM, cd(0, 0));
        for (int i = 0; i < N; ++i)
            for (int da = -BL; da <= BL; ++da) {
                const int a = i + da;
                if (a < 0 || a >= N) continue;
                const cd la = Lp(p, i, da);
                if (la == cd(0, 0)) continue;
                if (da != 0) off[a] += 0.5 * std::norm(la);
                for (int db = -BL; db <= BL; ++db) {
                    const int b = i + db;
                    if (b < 0 || b >= N) continue;
                    M[(size_t)a * WM + (b - a) + 2 * BL] += std::conj(la) * Lp(p, i, db);
                }
            }
        for (int j = 0; j < N; ++j) {
            const cd ljj = Lp(p, j, 0);
            for (int d = -2 * BL; d <= 2 * BL; ++d) {
                if (d == 0 || j + d < 0 || j + d >= N) continue;
                cd x = -0.5 * M[(size_t)j * WM + d + 2 * BL];
                if (d >= -BL && d <= BL) x += Lp(p, j, d) * std::conj(ljj);
                r[2 * ((size_t)j * WR + d + BR)] += x.real();
                r[2 * ((size_t)j * WR + d + BR) + 1] += x.imag();
            }
            for (int d = -BL; d <= BL; ++d) {
                if (d == 0) continue;
                const size_t o = 2 * (((size_t)p * N + j) * WL + d + BL);
                lo[o] = Lp(p, j, d).real();
                lo[o + 1] = Lp(p, j, d).imag();
            }
            split(ljj.real(), &ld[4 * ((size_t)p * N + j)]);
            split(ljj.imag(), &ld[4 * ((size_t)p * N + j) + 2]);
        }
    }
    for (int j = 0; j < N; ++j) {
        split(H0(j, 0).real(), &dg[8 * (size_t)j]);
        split(H1(j, 0).real(), &dg[8 * (size_t)j + 2]);
        dg[8 * (size_t)j + 4] = off[j];
    }
    m.h1_offdiag = std::any_of(h1o.begin(), h1o.end(), [](double x) { return x != 0.0; });
    upload(m.r32, r, s);
    upload(m.h1o32, h1o, s);
    upload(m.dg32, dg, s);
    upload(m.lo32, lo, s);
    upload(m.ld32, ld, s);
}


}  // namespace

void mf_build(gksl_ctx *c, bool fp32) {
    MfBands &m = c->mf;
    m = MfBands();
    const int N = c->N;
    cudaStream_t s = c->stream;
    int bh = 0, bl = 0;
    bool real = true;
    for (int k = 0; k < GKSL_MAX_H0; ++k)
        if (c->h0[k].set) { bh = std::max(bh, half_bandwidth(c->h0[k])); real = real && op_real(c->h0[k]); }
    if (c->h1.set) { bh = std::max(bh, half_bandwidth(c->h1)); real = real && op_real(c->h1); }
    std::vector<int> chans;
    for (int p = 0; p < GKSL_MAX_P; ++p)
        if (c->diss[p].set) {
            GK_REQUIRE(!c->diss[p].km, GKSL_ERR_ARG,
                       "the matrix-free form needs jump operators, not a full-rank Kossakowski matrix");
            chans.push_back(p);
            bl = std::max(bl, half_bandwidth(c->diss[p]));
            real = real && op_real(c->diss[p]);
        }
    GK_REQUIRE(N <= 32768, GKSL_ERR_ARG, "the matrix-free form is limited to N <= 32768");
    GK_REQUIRE(bh <= 4 && bl <= 4, GKSL_ERR_ARG,
               "the matrix-free form needs H0_k, H1 and L_p of half-bandwidth <= 4");
    const bool narrow = real && bh <= 1 && bl <= 1;
    const int BH = narrow ? 1 : 4, BG = narrow ? 2 : 8, BL = narrow ? 1 : 4;
    const int WH = 2 * BH + 1, WG = 2 * BG + 1, WL = 2 * BL + 1;
    std::vector<double> h0((size_t)2 * N * WH, 0.0), h1((size_t)2 * N * WH, 0.0), g((size_t)2 * N * WG, 0.0);
    std::vector<double> l((size_t)2 * N * WL * std::max<size_t>(chans.size(), 1), 0.0);
    for (int k = 0; k < GKSL_MAX_H0; ++k)
        if (c->h0[k].set) add_band(h0, N, BH, c->h0[k], c->h0[k].weight);
    if (c->h1.set) {
        add_band(h0, N, BH, c->h1, c->E);
        add_band(h1, N, BH, c->h1, 1.0);
    }
    // Gamma = 1/2 sum_p gamma_p L_p^+ L_p: (L^+ L)_(a,b) = sum_i conj(L_ia) L_ib, row by row of L
    for (size_t q = 0; q < chans.size(); ++q) {
        const Op &L = c->diss[chans[q]];
        const double gam = L.weight;
        for (int i = 0; i < N; ++i)
            for (int e1 = L.h_rowptr[i]; e1 < L.h_rowptr[i + 1]; ++e1) {
                const int a = L.h_col[e1];
                const std::complex<double> la(L.h_re[e1], L.h_im[e1]);
                for (int e2 = L.h_rowptr[i]; e2 < L.h_rowptr[i + 1]; ++e2) {
                    const int b = L.h_col[e2];
                    const std::complex<double> x = 0.5 * gam * std::conj(la) * std::complex<double>(L.h_re[e2], L.h_im[e2]);
                    const size_t o = 2 * ((size_t)a * WG + (b - a) + BG);
                    g[o] += x.real();
                    g[o + 1] += x.imag();
                }
            }
        std::vector<double> lb((size_t)2 * N * WL, 0.0);
        add_band(lb, N, BL, L, std::sqrt(gam));
        std::copy(lb.begin(), lb.end(), l.begin() + (ptrdiff_t)(q * lb.size()));
    }
    upload(m.h0, h0, s);
    upload(m.h1, h1, s);
    upload(m.g, g, s);
    upload(m.l, l, s);
    if (fp32) build_fp32(m, N, BH, BL, narrow ? 2 : 8, (int)chans.size(), h0, h1, l, s);
    // every tile (rows [a TJ, (a+1) TJ), columns [b TK, (b+1) TK)) holding some j <= k
    const int nt = (N + kTJ - 1) / kTJ, ntk = (N + kTK - 1) / kTK;
    std::vector<int> tiles;
    for (int a = 0; a < nt; ++a)
        for (int b = (a * kTJ) / kTK; b < ntk; ++b) { tiles.push_back(a); tiles.push_back(b); }
    m.tiles.alloc(tiles.size());
    GK_CUDA(cudaMemcpyAsync(m.tiles.p, tiles.data(), sizeof(int) * tiles.size(), cudaMemcpyHostToDevice, s));
    m.n_tiles = (int)(tiles.size() / 2);
    m.n_diag = nt;
    for (int i = 0; i < 4; ++i) {
        m.img64[i].alloc((size_t)N);
        GK_CUDA(cudaMemsetAsync(m.img64[i].p, 0, sizeof(double) * N, s));
        if (fp32) {
            m.img32[i].alloc((size_t)N);
            GK_CUDA(cudaMemsetAsync(m.img32[i].p, 0, sizeof(float) * N, s));
        }
    }
    if (narrow) { Narrow64::set_attributes(); Narrow32::set_attributes(); }
    else { Wide64::set_attributes(); Wide32::set_attributes(); }
    GK_CUDA(cudaStreamSynchronize(s));
    m.bh = BH;
    m.bg = BG;
    m.bl = BL;
    m.P = (int)chans.size();
    m.real = real;
    m.ready = true;
}

void mf_prep(gksl_ctx *c, int precision) {
    MfBands &m = c->mf;
    k_mf_prep<<<1, kThreads, 0, c->stream>>>(c->N, c->P2, c->v.p, m.img64[0].p,
                                             precision == 32 ? m.img32[0].p : nullptr);
    GK_LAUNCH_CHECK();
}

void mf_post(gksl_ctx *c, int precision) {
    MfBands &m = c->mf;
    k_mf_post<<<1, kThreads, 0, c->stream>>>(c->N, c->P2, m.img64[0].p, c->v.p, precision == 32 ? c->v32.p : nullptr);
    GK_LAUNCH_CHECK();
}

void mf_step(gksl_ctx *c, int precision, double h, const double *tab, long long local) {
    MfBands &m = c->mf;
    MfArgs a;
    a.N = c->N;
    a.P2 = c->P2;
    a.P = m.P;
    a.tiles = m.tiles.p;
    a.eps_tab = tab;
    a.base = c->step_base.p;
    a.local = local;
    a.hc.h = h;
    a.hc.h2 = 0.5 * h;
    a.hc.h6 = h / 6.0;
    a.hc.hf = (float)h;
    a.hc.h2f = 0.5f * (float)h;
    a.hc.h6f = (float)(h / 6.0);
    a.diag0 = M_SQRT2 / (double)c->N;
    a.diag0f = (float)a.diag0;
    const unsigned grid = (unsigned)m.n_tiles;
    const bool narrow = m.bh == 1;
    if (precision == 64) {
        MfOps<double> op{m.h0.p, m.h1.p, m.g.p, m.l.p};
        if (narrow) Narrow64::step(a, op, grid, c->stream, c);
        else Wide64::step(a, op, grid, c->stream, c);
    } else {
        MfOps32 op{m.r32.p, m.h1_offdiag ? m.h1o32.p : nullptr, m.dg32.p, m.lo32.p, m.ld32.p};
        if (narrow) Narrow32::step(a, op, grid, c->stream, c);
        else Wide32::step(a, op, grid, c->stream, c);
    }
    GK_LAUNCH_CHECK();
}

}  // namespace gk
