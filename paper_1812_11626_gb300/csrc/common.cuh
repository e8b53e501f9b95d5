// Internal declarations of libgksl: context, device buffers, errors, and the
// closed-form index arithmetic of the SU(N) generator basis (Sec. II list).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gksl.h"

namespace gk {

// ------------------------------------------------------------------ errors

struct Error {
    gksl_status st;
    std::string msg;
};

[[noreturn]] void throw_cuda(cudaError_t e, const char *what, const char *file, int line);

#define GK_CUDA(call)                                                     \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) ::gk::throw_cuda(e_, #call, __FILE__, __LINE__); \
    } while (0)

#define GK_REQUIRE(cond, status, message)                                  \
    do {                                                                   \
        if (!(cond)) throw ::gk::Error{(status), std::string(message)};   \
    } while (0)

#define GK_LAUNCH_CHECK() GK_CUDA(cudaGetLastError())

// NVTX range over a library call (header-only NVTX3: inert unless a profiler or tracer is
// attached), so timelines and ncu --nvtx filters see assembly, propagation and gradients
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// ------------------------------------------------------------------ device buffers

// Owning device allocation.  Freed on destruction; move-only.
template <typename T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    DBuf() = default;
    explicit DBuf(size_t count) { alloc(count); }
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    DBuf(DBuf &&o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
    DBuf &operator=(DBuf &&o) noexcept {
        if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
        return *this;
    }
    ~DBuf() { release(); }
    void alloc(size_t count) {
        release();
        if (count == 0) count = 1;
        cudaError_t e = cudaMalloc(&p, count * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            cudaGetLastError();
            throw Error{GKSL_ERR_OOM, "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed: " +
                                          cudaGetErrorString(e)};
        }
        n = count;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    size_t bytes() const { return n * sizeof(T); }
    T *get() const { return p; }
};

// ------------------------------------------------------------------ CSR on the device

// D x D (or rectangular) CSR with int32 column indices; values real or complex.
struct CsrR {
    long long rows = 0, cols = 0, nnz = 0;
    DBuf<int> rowptr;   // rows + 1 (int32: nnz < 2^31 is checked at build)
    DBuf<int> col;
    DBuf<double> val;
    size_t bytes() const { return rowptr.bytes() + col.bytes() + val.bytes(); }
};

struct CsrC {
    long long rows = 0, cols = 0, nnz = 0;
    DBuf<int> rowptr;
    DBuf<int> col;
    DBuf<double2> val;
};

// Hybrid propagation format: an ELL block of `width` slots for every row, stored slot-major
// (entry j of row r at j * ld + r) so that consecutive rows are consecutive addresses, plus
// warp-per-row CSR tails for the rows marked long (ELL column -1 in slot 0).
template <typename VT>
struct Hyb {
    long long rows = 0;   // rows covered
    long long ld = 0;     // leading dimension of the ELL block (rows rounded up to 32)
    int width = 0;
    DBuf<int> ell_col;
    DBuf<VT> ell_val;
    long long n_long = 0;
    DBuf<int> long_rows;  // row ids handled warp-per-row
    DBuf<int> tail_ptr;   // n_long + 1
    DBuf<int> tail_col;
    DBuf<VT> tail_val;
    long long tail_nnz = 0;
    // Compact copy of ell_col (empty when not built): slot entry e = (delta << 1) | s holds the
    // column delta + (s ? partner(r) : r), partner(r) being the S/J partner of basis row r
    // (r +- pairs for the S and J rows, r itself for the D rows), |delta| <= kC16Max.  Rows that
    // do not fit (listed in c16_esc, read through ell_col by threads of their own) and long rows
    // hold kC16Esc in slot 0.
    DBuf<short> ell_c16;
    long long c16_pairs = 0;   // N(N-1)/2
    long long n_esc = 0;       // short rows read through ell_col
    DBuf<int> c16_esc;
    size_t bytes() const {
        return ell_col.bytes() + ell_val.bytes() + long_rows.bytes() + tail_ptr.bytes() + tail_col.bytes() +
               tail_val.bytes() + ell_c16.bytes() + c16_esc.bytes();
    }
};

constexpr int kC16Max = 16383;
constexpr int kC16Esc = -32767;   // (-16384 << 1) | 1: a delta out of range, never a column

__device__ __host__ inline long long c16_partner(long long r, long long pairs) {
    return r < pairs ? r + pairs : (r < 2 * pairs ? r - pairs : r);
}

// Plain-pointer view of a Hyb matrix for kernels.
template <typename VT>
struct HybView {
    const int *ell_col;
    const VT *ell_val;
    long long ld;
    int width;
    const int *tail_ptr;
    const int *tail_col;
    const VT *tail_val;
    const short *ell_c16;
    long long c16_pairs;
};

template <typename VT>
inline HybView<VT> view(const Hyb<VT> &h) {
    return HybView<VT>{h.ell_col.p,  h.ell_val.p,  h.ld,        h.width,     h.tail_ptr.p,
                       h.tail_col.p, h.tail_val.p, h.ell_c16.p, h.c16_pairs};
}

// Band data of the matrix-free form: the operators of L(rho) as complex diagonals, row-major
// [N][2B+1] with entry (j, d + B) = X_(j, j+d), interleaved (re, im).
struct MfBands {
    bool ready = false;
    int bh = 0, bg = 0, bl = 0;   // half-bandwidths of the instantiation (H, Gamma, L)
    int P = 0;                    // channels
    bool real = false;            // every band real
    bool h1_offdiag = false;      // H1 has entries off its diagonal (the FP32 stages load them)
    int n_tiles = 0, n_diag = 0;  // upper-triangle tiles, of which on the diagonal
    // FP64 stages: H0 + E H1 (+ sum theta_k H0_k), H1, Gamma = 1/2 sum gamma L^+L, L' = sqrt(gamma) L
    DBuf<double> h0, h1, g, l;
    // FP32 stages (diagonals split off, off-diagonal couplings combined in FP64 first):
    // r: R_(j,a) for a != j; h1o: H1 off the diagonal; dg: H0_jj, H1_jj (hi/lo), 1/2 sum_p off_pj;
    // lo: L'_p off the diagonal; ld: L'_p,jj (hi/lo of re, im)
    DBuf<float> r32, h1o32, dg32, lo32, ld32;
    DBuf<int> tiles;              // (tile row, tile column) per block
    // diagonal images sqrt(2) sum_l y_l (D^l)_jj of v, yA, yB, acc during a run of steps
    // (FP64 stages and the FP64 master of the FP32 form; FP32 stages)
    DBuf<double> img64[4];
    DBuf<float> img32[4];
};

// An N x N input operator copied to the device (CSR, complex).
struct Op {
    bool set = false;
    int nnz = 0;
    DBuf<int> rowptr, col;
    DBuf<double> re, im;
    std::vector<int> h_rowptr, h_col;      // host copies (validation, stability bound)
    std::vector<double> h_re, h_im;
    double weight = 0.0;   // theta_k or gamma_p
    bool km = false;       // dissipator channel holding a whole Kossakowski matrix (gksl_ctx::km_A)
    double km_trace = 0.0; // Tr A of that matrix (the stability bound's dissipator norm)
};

}  // namespace gk

// ------------------------------------------------------------------ the context

struct gksl_ctx {
    int N = 0;
    long long P2 = 0, D = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;

    gk::Op h0[GKSL_MAX_H0];
    gk::Op h1;
    gk::Op diss[GKSL_MAX_P];
    double E = 0.0, A = 0.0, omega = 1.0;
    int drive_shape = 0;   // GKSL_DRIVE_SIN or GKSL_DRIVE_SQUARE
    bool drive_set = false;

    // components (unfolded, unit weight), rebuilt when an operator changes
    bool comp_dirty = true;
    gk::CsrR QH0[GKSL_MAX_H0];
    gk::CsrR Q1;
    gk::CsrR R[GKSL_MAX_P];
    gk::DBuf<double> Kp[GKSL_MAX_P];
    bool has_h0[GKSL_MAX_H0] = {};
    bool has_r[GKSL_MAX_P] = {};
    gk::DBuf<double2> km_A;    // Kossakowski matrix of the dense route (D x D), see Op::km
    bool comp_dense = false;   // components built with GKSL_ASM_DENSE_DISSIPATORS

    // combined, rebuilt when a weight or E changes
    bool assembled = false;
    unsigned asm_flags = 0;
    gk::CsrR Q0;        // sum theta Q(H0_k) + sum gamma R_p
    gk::DBuf<double> K; // sum gamma K_p
    double max_abs_q0 = 0.0;
    long long nnz_q0e = 0;
    gk::Hyb<double> hyb0, hyb1;   // propagation format of [Q0 + E Q1 | K] and Q1
    gk::Hyb<float> hyb0f, hyb1f;  // FP32 copies
    // Q1 folded into slot 0 of hyb0 (every short row has at most one Q1 entry, at a column of
    // its [Q0 + E Q1] row, moved to slot 0): the stage takes slot 0 as q0 + (eps - E) q1 and
    // reads no Q1 ELL; q1v[r] is that Q1 value (0 without one), long rows keep the Q1 tails
    bool q1_folded = false;
    gk::DBuf<double> q1v;
    gk::DBuf<float> q1vf;
    gk::MfBands mf;               // matrix-free form (GKSL_ASM_MATRIX_FREE)
    // adjoint: one channel per parameter matrix, transposed (Q(H)^T = -Q(H) is stored negated),
    // all channels sharing one long-row set: H0 components, then Q1, then the dissipators
    static constexpr int kMaxCh = GKSL_MAX_H0 + 1 + GKSL_MAX_P;
    gk::Hyb<double> adj[kMaxCh];
    gk::Hyb<float> adjf[kMaxCh];
    int adj_n = 0;
    int adj_kind[kMaxCh] = {};    // 0: H0 component, 1: Q1, 2: dissipator
    int adj_index[kMaxCh] = {};   // component or channel index
    bool has_adj = false;
    double assemble_seconds = 0.0;

    // state (length D + 1; entry D holds the constant 1 that carries K)
    gk::DBuf<double> v;
    double t = 0.0;
    bool state_set = false;
    // RK4 work vectors
    gk::DBuf<double> yA, yB, acc;
    gk::DBuf<float> v32, yA32, yB32, acc32;
    gk::DBuf<long long> step_base;   // device-side step counter base for graph replays
    gk::DBuf<double> eps_tab;        // eps(t) - E at the three stage times of every step of a run
    gk::DBuf<int> flag;              // device-side status flags (non-finite state)
    // stage-kernel variant per precision (index 0: FP64, 1: FP32), chosen by timing
    int rk4_var[2] = {0, 0};
    bool rk4_tuned[2] = {false, false};
    double rk4_var_us[2][4] = {};
    bool rk4_c16[2] = {false, false};   // stage columns from Hyb::ell_c16 (chosen with the variant)
    double rk4_var_us_c16[2][4] = {};
    // cached CUDA graphs for chunks of steps
    struct Graph {
        long long steps = 0;
        int precision = 0;
        double h = 0.0;
        cudaGraphExec_t exec = nullptr;
        int variant = 0;
    };
    std::vector<Graph> graphs;
};

struct gksl_batch;

// ------------------------------------------------------------------ basis index math

namespace gk {

struct El {
    int kind;  // 0: S^(a,b), 1: J^(a,b), 2: D^a
    int a, b;
};

struct Basis {
    int N;
    long long P2, D;
    __host__ __device__ Basis(int n) : N(n), P2((long long)n * (n - 1) / 2), D((long long)n * n - 1) {}
    // lexicographic pair index of j < k
    __host__ __device__ long long pair(int j, int k) const {
        return (long long)j * N - ((long long)j * (j + 1)) / 2 + (k - j - 1);
    }
    __host__ __device__ long long pair_start(int j) const { return (long long)j * N - ((long long)j * (j + 1)) / 2; }
    __host__ __device__ void unpair(long long p, int &j, int &k) const {
        double b = 2.0 * N - 1.0;
        double disc = b * b - 8.0 * (double)p;
        int jj = (int)((b - sqrt(disc > 0 ? disc : 0.0)) * 0.5);
        if (jj < 0) jj = 0;
        if (jj > N - 2) jj = N - 2;
        while (jj > 0 && pair_start(jj) > p) --jj;
        while (jj + 1 <= N - 2 && pair_start(jj + 1) <= p) ++jj;
        j = jj;
        k = (int)(p - pair_start(jj)) + jj + 1;
    }
    __host__ __device__ El decode(long long s) const {
        El e;
        if (s < P2) { e.kind = 0; unpair(s, e.a, e.b); }
        else if (s < 2 * P2) { e.kind = 1; unpair(s - P2, e.a, e.b); }
        else { e.kind = 2; e.a = (int)(s - 2 * P2) + 1; e.b = -1; }
        return e;
    }
    __host__ __device__ long long encode(const El &e) const {
        if (e.kind == 2) return 2 * P2 + e.a - 1;
        return (e.kind == 1 ? P2 : 0) + pair(e.a, e.b);
    }
};

// c_l = 1/sqrt(l(l+1))
__host__ __device__ inline double cl(int l) { return 1.0 / sqrt((double)l * ((double)l + 1.0)); }

// (D^l)_{jj}: c_l for j < l, -l c_l for j = l, 0 for j > l
__host__ __device__ inline double dl_diag(int l, int j) {
    if (j < l) return cl(l);
    if (j == l) return -(double)l * cl(l);
    return 0.0;
}

#define GK_RSQRT2 0.70710678118654752440

// Closed forms of f and d for three pair generators on the triangle p < q < r with the pairs
// in canonical order (pq, qr, pr) and kinds t0, t1, t2 (0 = S, 1 = J).  They follow from
// multiplying the matrix units of the Sec. II list: e.g. [S_pq, S_qr] = (i/sqrt2) J_pr.
__host__ __device__ inline double f_triangle(int t0, int t1, int t2) {
    int code = t0 * 4 + t1 * 2 + t2;
    switch (code) {
        case 1: return GK_RSQRT2;   // S S J
        case 2: return -GK_RSQRT2;  // S J S
        case 4: return -GK_RSQRT2;  // J S S
        case 7: return -GK_RSQRT2;  // J J J
        default: return 0.0;
    }
}
__host__ __device__ inline double d_triangle(int t0, int t1, int t2) {
    int code = t0 * 4 + t1 * 2 + t2;
    switch (code) {
        case 0: return GK_RSQRT2;   // S S S
        case 3: return GK_RSQRT2;   // S J J
        case 5: return GK_RSQRT2;   // J S J
        case 6: return -GK_RSQRT2;  // J J S
        default: return 0.0;
    }
}

// f_{xyz} (which = 0) or d_{xyz} (which = 1) of Eq. 5 from the closed forms, for any
// three generators.  Zero outside the nonzero set.
__host__ __device__ inline double structure_value(int which, const El &x, const El &y, const El &z) {
    const El e[3] = {x, y, z};
    int nd = (x.kind == 2) + (y.kind == 2) + (z.kind == 2);
    if (nd == 0) {
        // three pairs: must be the three edges of one triangle p < q < r
        int v[6] = {x.a, x.b, y.a, y.b, z.a, z.b};
        int p = v[0], q = -1, r = -1;
        // collect distinct vertices
        int dv[6], nv = 0;
        for (int i = 0; i < 6; ++i) {
            bool seen = false;
            for (int k = 0; k < nv; ++k) seen = seen || (dv[k] == v[i]);
            if (!seen) dv[nv++] = v[i];
        }
        if (nv != 3) return 0.0;
        // sort the three vertices
        for (int i = 0; i < 3; ++i)
            for (int k = i + 1; k < 3; ++k)
                if (dv[k] < dv[i]) { int t = dv[i]; dv[i] = dv[k]; dv[k] = t; }
        p = dv[0]; q = dv[1]; r = dv[2];
        // position of each argument among (pq, qr, pr)
        int pos[3];
        for (int i = 0; i < 3; ++i) {
            if (e[i].a == p && e[i].b == q) pos[i] = 0;
            else if (e[i].a == q && e[i].b == r) pos[i] = 1;
            else if (e[i].a == p && e[i].b == r) pos[i] = 2;
            else return 0.0;
        }
        if (pos[0] == pos[1] || pos[1] == pos[2] || pos[0] == pos[2]) return 0.0;
        int t[3];
        for (int i = 0; i < 3; ++i) t[pos[i]] = e[i].kind;
        // sign of the permutation i -> pos[i]
        int inv = (pos[0] > pos[1]) + (pos[0] > pos[2]) + (pos[1] > pos[2]);
        if (which == 0) return (inv & 1 ? -1.0 : 1.0) * f_triangle(t[0], t[1], t[2]);
        return d_triangle(t[0], t[1], t[2]);
    }
    if (nd == 1) {
        // two generators of the same pair (a, b) and one D^l
        int id = x.kind == 2 ? 0 : (y.kind == 2 ? 1 : 2);
        const El &P = e[(id + 1) % 3], &R = e[(id + 2) % 3];
        if (P.a != R.a || P.b != R.b) return 0.0;
        int l = e[id].a;
        if (which == 0) {
            if (P.kind == R.kind) return 0.0;
            // f(S, J, D) = delta_l(a) - delta_l(b); cyclic order (P, R) after D keeps the sign
            double v = dl_diag(l, P.a) - dl_diag(l, P.b);
            return P.kind == 0 ? v : -v;
        }
        if (P.kind != R.kind) return 0.0;
        return dl_diag(l, P.a) + dl_diag(l, P.b);
    }
    if (nd == 2) return 0.0;
    // three diagonal generators: only d, only with two equal indices
    if (which == 0) return 0.0;
    int l0 = x.a, l1 = y.a, l2 = z.a;
    if (l0 == l1 && l1 == l2) return 2.0 * cl(l0) * (1.0 - (double)l0);
    int lo, hi;
    if (l0 == l1) { lo = l0; hi = l2; }
    else if (l0 == l2) { lo = l0; hi = l1; }
    else if (l1 == l2) { lo = l1; hi = l0; }
    else return 0.0;
    return hi > lo ? 2.0 * cl(hi) : 0.0;
}

// ------------------------------------------------------------------ launch helpers

// theta of the drive eps = E + A theta at the three stage times of the step [tn, tn + h]
// (square shape: theta at the step midpoint for every stage)
__host__ __device__ inline void drive_theta(int shape, double omega, double tn, double h, double th[3]) {
    if (shape == 1) {
        const double T = 2.0 * 3.14159265358979323846 / omega;
        double m = fmod(tn + 0.5 * h, T);
        if (m < 0) m += T;
        const double s = m < 0.5 * T ? 1.0 : -1.0;
        th[0] = th[1] = th[2] = s;
        return;
    }
    th[0] = sin(omega * tn);
    th[1] = sin(omega * (tn + 0.5 * h));
    th[2] = sin(omega * (tn + h));
}

inline unsigned grid_for(long long n, int threads) {
    long long g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    return (unsigned)g;
}

bool is_device_ptr(const void *p);
// copy `bytes` from a host-or-device pointer to device memory on stream s
void copy_in(void *dst_dev, const void *src, size_t bytes, cudaStream_t s);
// copy `bytes` from device memory to a host-or-device pointer (synchronises for host targets)
void copy_out(void *dst, const void *src_dev, size_t bytes, cudaStream_t s);

}  // namespace gk
