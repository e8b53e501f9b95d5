// Dense dissipators: the dissipator matrix R and vector K of Eq. 8 when the jump operator is
// dense or the Kossakowski matrix has full rank (Table II, dense column; Sec. VI, random
// Lindbladians).
//
// The sparse route (assemble.cu) contracts the structure constants with the coefficients of L;
// for a dense L its product F''^T Z'' has O(N^5) terms (5.5e9 at N = 100).  Here the dissipator
// is taken through its matrix-unit form instead.  For the Eq. 8 term
//     D(rho) = sum_jk A_jk (F_j rho F_k - 1/2 {F_k F_j, rho})
// define the N^2 x N^2 kernel and the N x N matrix
//     M[a,c; d,b] = sum_jk (F_j)_ac A_jk (F_k)_db,      G = sum_jk A_jk F_k F_j,
// so that D(E_cd)_ab = M[a,c; d,b] - 1/2 G_ac [b = d] - 1/2 [a = c] G_db for the matrix unit
// E_cd, and G_xy = sum_z M[z,y; x,z].  For one jump operator L at unit rate (trace part
// included, no H_eff needed) M[a,c; d,b] = L_ac conj(L_bd) and G = L^+ L.  Then
//     R_sm = Re Tr(F_s D(F_m)) = Re sum (F_s)_ba (F_m)_cd D(E_cd)_ab,
//     K_s  = Re Tr(F_s D(1/N)) = (1/N) Re sum (F_s)_ba (sum_c M[a,c; c,b] - G_ab),
// each sum running over the (at most 2, or l + 1 for D^l) nonzero entries of the generators
// (Sec. II list).  Every entry of R is formed by one thread; the work is
// (sum_s nnz(F_s))^2 ~ 6 N^4 complex multiply-adds, the memory D^2 doubles for R plus, for a
// Kossakowski matrix, N^4 complex for M (built from A through the sparse basis matrix in
// O(D^2 + N^5) operations).  R is then compressed to CSR without its exact zeros.
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"
#include "prim.cuh"

namespace gk {
namespace {

constexpr int kT = 256;

__device__ inline double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ inline double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ inline double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ inline double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

// Entry t of generator s as (row, col, value); count() entries in all.  S^(x,y): (x,y), (y,x)
// with 1/sqrt2; J^(x,y): (x,y) with -i/sqrt2, (y,x) with +i/sqrt2; D^l: (c,c) with
// (D^l)_cc for c = 0..l.
struct Gen {
    int kind, x, y;   // kind 0: S, 1: J, 2: D^x
    double cl;        // c_x = 1/sqrt(x(x+1)) of a D generator, computed once
    __device__ Gen(const Basis &B, long long s) {
        El e = B.decode(s);
        kind = e.kind;
        x = e.a;
        y = e.b;
        cl = kind == 2 ? gk::cl(x) : 0.0;
    }
    __device__ int count() const { return kind == 2 ? x + 1 : 2; }
    __device__ void entry(int t, int &r, int &c, double2 &v) const {
        if (kind == 2) {   // (D^x)_tt = c_x for t < x, -x c_x for t = x
            r = c = t;
            v = make_double2(t < x ? cl : -(double)x * cl, 0.0);
        } else if (t == 0) {
            r = x; c = y;
            v = kind == 0 ? make_double2(GK_RSQRT2, 0.0) : make_double2(0.0, -GK_RSQRT2);
        } else {
            r = y; c = x;
            v = kind == 0 ? make_double2(GK_RSQRT2, 0.0) : make_double2(0.0, GK_RSQRT2);
        }
    }
};

// The kernel M[a,c; d,b] of the jump term: one channel L (MODE 0) or a materialised N^4 array
// (MODE 1, index ((a N + c) N + d) N + b).
template <int MODE>
struct Kern {
    const double2 *L;   // MODE 0: N x N row-major
    const double2 *M;   // MODE 1
    int N;
    __device__ double2 operator()(int a, int c, int d, int b) const {
        if (MODE == 0) return cmul(L[(long long)a * N + c], cconj(L[(long long)b * N + d]));
        return M[(((long long)a * N + c) * N + d) * N + b];
    }
};

// R_sm for every (s, m) of a block of rows [s0, s0 + rows), dense row-major into out.
template <int MODE>
__global__ void __launch_bounds__(kT) k_dense_R(Basis B, Kern<MODE> kern, const double2 *__restrict__ G,
                                                 long long s0, long long rows, double *__restrict__ out) {
    const long long D = B.D;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * D) return;
    const long long s = s0 + i / D, m = i % D;
    const int N = B.N;
    Gen fs(B, s), fm(B, m);
    double acc = 0.0;
    const int ns = fs.count(), nm = fm.count();
    for (int u = 0; u < ns; ++u) {
        int b, a;
        double2 ws;
        fs.entry(u, b, a, ws);   // (F_s)_ba
        for (int t = 0; t < nm; ++t) {
            int c, d;
            double2 wm;
            fm.entry(t, c, d, wm);   // (F_m)_cd
            double2 w = kern(a, c, d, b);
            if (b == d) w = cadd(w, cscale(G[(long long)a * N + c], -0.5));
            if (a == c) w = cadd(w, cscale(G[(long long)d * N + b], -0.5));
            acc += cmul(cmul(ws, wm), w).x;
        }
    }
    out[i] = acc;
}

// K_s = (1/N) Re sum (F_s)_ba (sum_c M[a,c; c,b] - G_ab)
template <int MODE>
__global__ void __launch_bounds__(kT) k_dense_K(Basis B, Kern<MODE> kern, const double2 *__restrict__ G,
                                                 double *__restrict__ K) {
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B.D) return;
    const int N = B.N;
    Gen fs(B, s);
    double acc = 0.0;
    for (int u = 0; u < fs.count(); ++u) {
        int b, a;
        double2 ws;
        fs.entry(u, b, a, ws);
        double2 p = cscale(G[(long long)a * N + b], -1.0);
        for (int c = 0; c < N; ++c) p = cadd(p, kern(a, c, c, b));
        acc += cmul(ws, p).x;
    }
    K[s] = acc / N;
}

// dense N x N copy of a CSR operator
__global__ void k_densify(const int *__restrict__ rp, const int *__restrict__ col, const double *__restrict__ re,
                          const double *__restrict__ im, int N, double2 *__restrict__ out) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    for (int e = rp[r]; e < rp[r + 1]; ++e) {
        double2 &o = out[(long long)r * N + col[e]];
        o.x += re[e];
        o.y += im ? im[e] : 0.0;
    }
}

// G_xy = sum_z M[z,y; x,z]
template <int MODE>
__global__ void k_dense_G(Kern<MODE> kern, int N, double2 *__restrict__ G) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)N * N) return;
    int x = (int)(i / N), y = (int)(i % N);
    double2 g = make_double2(0.0, 0.0);
    for (int z = 0; z < N; ++z) g = cadd(g, kern(z, y, x, z));
    G[i] = g;
}

// Bm[j; d,b] = sum_k A_jk (F_k)_db  (D x N^2).  Off the diagonal (d != b) only the S and J
// generators of the pair {d, b} have a (d, b) entry; on it, the D^l with l >= max(d, 1).
__global__ void k_km_B(Basis B, const double2 *__restrict__ A, double2 *__restrict__ Bm) {
    const long long N2 = (long long)B.N * B.N;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B.D * N2) return;
    const long long j = i / N2;
    const int d = (int)((i % N2) / B.N), b = (int)(i % B.N);
    const double2 *Aj = A + j * B.D;
    double2 v = make_double2(0.0, 0.0);
    if (d != b) {
        int lo = d < b ? d : b, hi = d < b ? b : d;
        long long p = B.pair(lo, hi);
        double2 aS = Aj[p], aJ = Aj[B.P2 + p];
        // (F_S)_db = 1/sqrt2; (F_J)_db = -i/sqrt2 above the diagonal (d < b), +i/sqrt2 below
        double sg = d < b ? -GK_RSQRT2 : GK_RSQRT2;
        v = make_double2(GK_RSQRT2 * aS.x - sg * aJ.y, GK_RSQRT2 * aS.y + sg * aJ.x);
    } else {
        for (int l = d > 1 ? d : 1; l < B.N; ++l) v = cadd(v, cscale(Aj[2 * B.P2 + l - 1], dl_diag(l, d)));
    }
    Bm[i] = v;
}

// M[a,c; d,b] = sum_j (F_j)_ac Bm[j; d,b]  (N^4, index ((a N + c) N + d) N + b)
__global__ void k_km_M(Basis B, const double2 *__restrict__ Bm, double2 *__restrict__ M) {
    const int N = B.N;
    const long long N2 = (long long)N * N;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N2 * N2) return;
    const long long ac = i / N2, db = i % N2;
    const int a = (int)(ac / N), c = (int)(ac % N);
    double2 v = make_double2(0.0, 0.0);
    if (a != c) {
        int lo = a < c ? a : c, hi = a < c ? c : a;
        long long p = B.pair(lo, hi);
        double2 bS = Bm[p * N2 + db], bJ = Bm[(B.P2 + p) * N2 + db];
        double sg = a < c ? -GK_RSQRT2 : GK_RSQRT2;   // (F_J)_ac = sg * i
        v = make_double2(GK_RSQRT2 * bS.x - sg * bJ.y, GK_RSQRT2 * bS.y + sg * bJ.x);
    } else {
        for (int l = a > 1 ? a : 1; l < N; ++l) v = cadd(v, cscale(Bm[(2 * B.P2 + l - 1) * N2 + db], dl_diag(l, a)));
    }
    M[i] = v;
}

// nonzeros of each row of a dense rows x ncols block (one warp per row)
__global__ void k_row_nnz(const double *__restrict__ X, long long rows, long long ncols, long long *__restrict__ cnt) {
    long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (w >= rows) return;
    const double *x = X + w * ncols;
    long long n = 0;
    for (long long j = lane; j < ncols; j += 32) n += x[j] != 0.0;
    for (int o = 16; o > 0; o >>= 1) n += __shfl_down_sync(0xffffffffu, n, o);
    if (lane == 0) cnt[w] = n;
}

// compress the nonzeros of each row in column order (one warp per row, ballot + prefix count)
__global__ void k_row_fill(const double *__restrict__ X, long long rows, long long ncols, long long row0,
                           const long long *__restrict__ off, int *__restrict__ col, double *__restrict__ val) {
    long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (w >= rows) return;
    const double *x = X + w * ncols;
    long long pos = off[row0 + w];
    for (long long j0 = 0; j0 < ncols; j0 += 32) {
        long long j = j0 + lane;
        double v = j < ncols ? x[j] : 0.0;
        unsigned m = __ballot_sync(0xffffffffu, v != 0.0);
        if (v != 0.0) {
            long long p = pos + __popc(m & ((1u << lane) - 1u));
            col[p] = (int)j;
            val[p] = v;
        }
        pos += __popc(m);
    }
}

__global__ void k_ll_to_int(const long long *__restrict__ in, long long n, int *__restrict__ out) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (int)in[i];
}

// R (CSR at unit weight, exact zeros left out) and K of a dissipator given by its kernel.  The
// dense rows are formed in blocks of about 2^27 entries, twice: once to count each row's
// nonzeros, once to write them, so the transient stays at 1 GB whatever D is.
template <int MODE>
void dense_R_K(gksl_ctx *c, const Kern<MODE> &kern, CsrR &R, DBuf<double> &K) {
    Basis B(c->N);
    cudaStream_t s = c->stream;
    const long long D = B.D;
    const long long NN = (long long)c->N * c->N;
    DBuf<double2> G((size_t)NN);
    k_dense_G<MODE><<<grid_for(NN, kT), kT, 0, s>>>(kern, c->N, G.p);
    GK_LAUNCH_CHECK();
    K.alloc((size_t)D);
    k_dense_K<MODE><<<grid_for(D, kT), kT, 0, s>>>(B, kern, G.p, K.p);
    GK_LAUNCH_CHECK();
    const long long per = std::max(1LL, (1LL << 27) / D);
    DBuf<double> blk((size_t)(std::min(per, D) * D));
    DBuf<long long> cnt((size_t)D), off((size_t)D + 1);
    for (long long r0 = 0; r0 < D; r0 += per) {
        const long long nr = std::min(per, D - r0);
        k_dense_R<MODE><<<grid_for(nr * D, kT), kT, 0, s>>>(B, kern, G.p, r0, nr, blk.p);
        GK_LAUNCH_CHECK();
        k_row_nnz<<<grid_for(nr * 32, kT), kT, 0, s>>>(blk.p, nr, D, cnt.p + r0);
        GK_LAUNCH_CHECK();
    }
    const long long nnz = scan_ll(cnt.p, off.p, D, true, true, s);
    GK_REQUIRE(nnz < (1LL << 31), GKSL_ERR_ARG, "dense dissipator has more than 2^31 - 1 nonzeros");
    R = CsrR();
    R.rows = R.cols = D;
    R.nnz = nnz;
    R.rowptr.alloc((size_t)D + 1);
    R.col.alloc((size_t)std::max(1LL, nnz));
    R.val.alloc((size_t)std::max(1LL, nnz));
    k_ll_to_int<<<grid_for(D + 1, kT), kT, 0, s>>>(off.p, D + 1, R.rowptr.p);
    GK_LAUNCH_CHECK();
    for (long long r0 = 0; r0 < D; r0 += per) {
        const long long nr = std::min(per, D - r0);
        k_dense_R<MODE><<<grid_for(nr * D, kT), kT, 0, s>>>(B, kern, G.p, r0, nr, blk.p);
        GK_LAUNCH_CHECK();
        k_row_fill<<<grid_for(nr * 32, kT), kT, 0, s>>>(blk.p, nr, D, r0, off.p, R.col.p, R.val.p);
        GK_LAUNCH_CHECK();
    }
    GK_CUDA(cudaStreamSynchronize(s));
}

// Kossakowski matrix upload (gksl_set_kossakowski at N > 64): interleave the planar entries into A
// and flag a non-finite entry (bit 1); the largest |a_jk| goes to *maxbits as the bit pattern of a
// non-negative double (whose unsigned order is the order of the values), one atomic per warp.
__global__ void k_km_pack(const double *__restrict__ re, const double *__restrict__ im, long long n,
                          double2 *__restrict__ A, unsigned long long *__restrict__ maxbits, int *__restrict__ flag) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double m = 0.0;
    if (i < n) {
        const double x = re[i], y = im ? im[i] : 0.0;
        A[i] = make_double2(x, y);
        if (!isfinite(x) || !isfinite(y)) atomicOr(flag, 1);
        else m = hypot(x, y);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(maxbits, (unsigned long long)__double_as_longlong(m));
}

// Necessary conditions of positive semidefiniteness and Hermiticity for entry (j, k), k >= j
// (thread x walks k, so the reads of row j are coalesced): |a_jk - conj(a_kj)| within tol_h
// (bit 2), a_jj >= -eps (bit 4), |a_jk|^2 <= max(a_jj, 0) max(a_kk, 0) + minor_eps (bit 8).
__global__ void k_km_check(const double2 *__restrict__ A, long long D, double tol_h, double eps, double minor_eps,
                           int *__restrict__ flag) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long j = blockIdx.y;
    if (k >= D || k < j) return;
    const double2 a = A[j * D + k], b = A[k * D + j];
    int f = 0;
    if (fabs(a.x - b.x) > tol_h || fabs(a.y + b.y) > tol_h) f |= 2;
    const double ajj = A[j * D + j].x;
    if (k == j) {
        if (ajj < -eps) f |= 4;
    } else {
        const double akk = A[k * D + k].x;
        if (a.x * a.x + a.y * a.y > fmax(ajj, 0.0) * fmax(akk, 0.0) + minor_eps) f |= 8;
    }
    if (f) atomicOr(flag, f);
}

__global__ void k_km_diag(const double2 *__restrict__ A, long long D, double *__restrict__ d) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < D) d[j] = A[j * D + j].x;
}

}  // namespace

double kossakowski_upload_checked(gksl_ctx *c, const double *a_re, const double *a_im, DBuf<double2> &A) {
    NvtxRange nv("Kossakowski matrix: upload and checks");
    cudaStream_t s = c->stream;
    const long long D = c->D;
    const size_t DD = (size_t)D * (size_t)D;
    // planar copies of host input and of another GPU's memory (this device's is read in place)
    DBuf<double> dre, dim;
    const double *re = a_re, *im = a_im;
    if (!device_local_ptr(a_re, c->device)) {
        dre.alloc(DD);
        GK_CUDA(cudaMemcpyAsync(dre.p, a_re, sizeof(double) * DD, cudaMemcpyDefault, s));
        re = dre.p;
    }
    if (a_im && !device_local_ptr(a_im, c->device)) {
        dim.alloc(DD);
        GK_CUDA(cudaMemcpyAsync(dim.p, a_im, sizeof(double) * DD, cudaMemcpyDefault, s));
        im = dim.p;
    }
    A.alloc(DD);
    DBuf<int> flag(1);
    DBuf<unsigned long long> maxbits(1);
    GK_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), s));
    GK_CUDA(cudaMemsetAsync(maxbits.p, 0, sizeof(unsigned long long), s));
    k_km_pack<<<grid_for((long long)DD, kT), kT, 0, s>>>(re, im, (long long)DD, A.p, maxbits.p, flag.p);
    GK_LAUNCH_CHECK();
    int hf = 0;
    unsigned long long hb = 0;
    GK_CUDA(cudaMemcpyAsync(&hf, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaMemcpyAsync(&hb, maxbits.p, sizeof(hb), cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaStreamSynchronize(s));
    dre.release();
    dim.release();
    GK_REQUIRE(!(hf & 1), GKSL_ERR_ARG, "non-finite Kossakowski entry");
    double mx;
    std::memcpy(&mx, &hb, sizeof mx);
    const double eps = 1e-12 * mx;
    k_km_check<<<dim3((unsigned)((D + kT - 1) / kT), (unsigned)D), kT, 0, s>>>(A.p, D, 1e-12 * mx, eps, eps * mx * 4.0,
                                                                           flag.p);
    GK_LAUNCH_CHECK();
    DBuf<double> dg((size_t)D);
    k_km_diag<<<grid_for(D, kT), kT, 0, s>>>(A.p, D, dg.p);
    GK_LAUNCH_CHECK();
    std::vector<double> hd((size_t)D);
    GK_CUDA(cudaMemcpyAsync(hd.data(), dg.p, sizeof(double) * D, cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaMemcpyAsync(&hf, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaStreamSynchronize(s));
    GK_REQUIRE(!(hf & 2), GKSL_ERR_ARG, "Kossakowski matrix is not Hermitian");
    GK_REQUIRE(!(hf & 4), GKSL_ERR_ARG, "Kossakowski matrix is not positive semidefinite");
    GK_REQUIRE(!(hf & 8), GKSL_ERR_ARG,
               "Kossakowski matrix is not positive semidefinite (a 2 x 2 principal minor is negative)");
    double tr = 0.0;
    for (long long j = 0; j < D; ++j) tr += hd[(size_t)j];
    return tr;
}

void dense_dissipator_channel(gksl_ctx *c, const Op &op, CsrR &R, DBuf<double> &K) {
    NvtxRange nv("dense dissipator (channel)");
    GK_REQUIRE(c->N <= kDenseDissMaxN, GKSL_ERR_ARG, "the dense dissipator route is limited to N <= 200");
    cudaStream_t s = c->stream;
    const int N = c->N;
    DBuf<double2> L((size_t)N * N);
    GK_CUDA(cudaMemsetAsync(L.p, 0, sizeof(double2) * N * N, s));
    k_densify<<<grid_for(N, 128), 128, 0, s>>>(op.rowptr.p, op.col.p, op.re.p, op.im.p, N, L.p);
    GK_LAUNCH_CHECK();
    Kern<0> k{L.p, nullptr, N};
    dense_R_K<0>(c, k, R, K);
}

void dense_dissipator_kossakowski(gksl_ctx *c, const double2 *A, CsrR &R, DBuf<double> &K) {
    NvtxRange nv("dense dissipator (Kossakowski)");
    GK_REQUIRE(c->N <= kDenseKmMaxN, GKSL_ERR_ARG, "the dense Kossakowski route is limited to N <= 128");
    Basis B(c->N);
    cudaStream_t s = c->stream;
    const long long N2 = (long long)c->N * c->N;
    DBuf<double2> M((size_t)(N2 * N2));
    {
        DBuf<double2> Bm((size_t)(B.D * N2));
        k_km_B<<<grid_for(B.D * N2, kT), kT, 0, s>>>(B, A, Bm.p);
        GK_LAUNCH_CHECK();
        k_km_M<<<grid_for(N2 * N2, kT), kT, 0, s>>>(B, Bm.p, M.p);
        GK_LAUNCH_CHECK();
        GK_CUDA(cudaStreamSynchronize(s));
    }
    Kern<1> k{nullptr, M.p, c->N};
    dense_R_K<1>(c, k, R, K);
}

}  // namespace gk
