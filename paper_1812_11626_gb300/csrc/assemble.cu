// Assembly of the unfolded system (Sec. IV steps 2.2-2.5) on the device.
//
// For a coefficient vector x over the generators (x_m = Tr(F_m X)) two contractions with the
// structure constants of Eq. 5 are formed:
//     Q(x)_{s n} = sum_m x_m f_{m n s}                         (Eq. 7)
//     Z(x)_{n s} = sum_m x_m z_{m n s},  z = f + i d           (the F'' / Z'' sums of step 2.5)
// The nonzero (m, n, s) of f and d come from closed forms (common.cuh); for each nonzero
// coefficient x_m of pair type the two-dimensional section {(n, s)} is enumerated (O(N) entries),
// and the diagonal coefficients x_{D^l} are contracted in closed form, since
// sum_l x_l f(D^l, S_jk, J_jk) = Xd_j - Xd_k and sum_l x_l d(D^l, S_jk, S_jk) = Xd_j + Xd_k with
// Xd = sum_l x_l D^l (a suffix sum over l).  The entries are emitted as (row, column, value)
// triplets, sorted and summed into CSR (the paper's coordinate format, sort and two-pass CRS).
//
// With F''^T = Q(conj l) and Z'' = Z(l), Eq. 10 (prefactor -1/4, see below) and Eq. 11 become
//     R = -(1/2) Re(Q(conj l) Z(l)),        K = -(i/N) Q(conj l) l      (per unit rate),
// the first a sparse-sparse product formed row by row (the paper accumulates the same products
// in one red-black tree per row).  Readings of the paper used here: the two-term form of Eq. 10
// needs -1/4 (not -1/2) to equal Tr(F_s L(F_m)); Eq. 11 carries the rate gamma_p; a dissipator
// with trace part l0 = Tr(L)/N adds the Hamiltonian H_eff = (i/2)(conj(l0) L' - l0 L'^+),
// coefficients -Im(conj(l0) l_j) per unit rate.
#include <chrono>

#include "internal.cuh"
#include "prim.cuh"

namespace gk {

namespace {

__device__ inline uint64_t mkkey(long long row, long long col, long long ncols) {
    return (uint64_t)row * (uint64_t)ncols + (uint64_t)col;
}

__device__ inline double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// ---- compaction of the nonzero pair coefficients

__global__ void k_nz_flags(const double2 *__restrict__ coef, long long n, long long *__restrict__ flag) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = (coef[i].x != 0.0 || coef[i].y != 0.0) ? 1 : 0;
}

__global__ void k_nz_gather(const double2 *__restrict__ coef, long long n, const long long *__restrict__ flag,
                            const long long *__restrict__ pos, bool conj, long long *__restrict__ nzi,
                            double2 *__restrict__ nzv) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flag[i]) {
        nzi[pos[i]] = i;
        double2 x = coef[i];
        nzv[pos[i]] = conj ? make_double2(x.x, -x.y) : x;
    }
}

// Xd_j = sum_l x_l (D^l)_jj = sum_{l>j} c_l x_l - j c_j x_j;  suf_j = sum_{l>j} c_l x_l
__global__ void k_dpart_prep(int N, long long P2, const double2 *__restrict__ coef, bool conj,
                             double2 *__restrict__ Xd, double2 *__restrict__ suf) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double2 s = make_double2(0.0, 0.0);
    for (int j = N - 1; j >= 0; --j) {
        suf[j] = s;
        double2 own = make_double2(0.0, 0.0);
        if (j >= 1) {
            double2 x = coef[2 * P2 + j - 1];
            if (conj) x.y = -x.y;
            double c = cl(j);
            own = make_double2(-(double)j * c * x.x, -(double)j * c * x.y);
            s.x += c * x.x;
            s.y += c * x.y;
        }
        Xd[j] = make_double2(suf[j].x + own.x, suf[j].y + own.y);
    }
}

// ---- sections of f and d for the nonzero pair coefficients
// MODE 0: Q(x)_{s n} += x_m f(m, n, s);  MODE 1: Z(x)_{n s} += x_m (f + i d)(m, n, s).
// One item per (coefficient t, third index c); c is the third vertex of a triangle and also
// the index l of a D^l partner.
template <int MODE, bool FILL>
__global__ void k_emit_pairs(Basis B, const long long *__restrict__ nzi, const double2 *__restrict__ nzv,
                             long long nnz, long long *__restrict__ cnt, const long long *__restrict__ off,
                             uint64_t *__restrict__ keys, double2 *__restrict__ vals) {
    long long item = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= nnz * B.N) return;
    long long t = item / B.N;
    int c = (int)(item % B.N);
    El m = B.decode(nzi[t]);
    double2 x = nzv[t];
    long long o = FILL ? off[item] : 0;
    int k = 0;
    auto put = [&](const El &n, const El &s) {
        double fv = structure_value(0, m, n, s);
        double dv = MODE == 1 ? structure_value(1, m, n, s) : 0.0;
        if (fv == 0.0 && dv == 0.0) return;
        if (FILL) {
            if (MODE == 0) {
                keys[o + k] = mkkey(B.encode(s), B.encode(n), B.D);
                vals[o + k] = make_double2(x.x * fv, x.y * fv);
            } else {
                keys[o + k] = mkkey(B.encode(n), B.encode(s), B.D);
                vals[o + k] = make_double2(x.x * fv - x.y * dv, x.y * fv + x.x * dv);
            }
        }
        ++k;
    };
    if (c != m.a && c != m.b) {
        int u1 = min(m.a, c), v1 = max(m.a, c), u2 = min(m.b, c), v2 = max(m.b, c);
        for (int tn = 0; tn < 2; ++tn)
            for (int ts = 0; ts < 2; ++ts) {
                put(El{tn, u1, v1}, El{ts, u2, v2});
                put(El{tn, u2, v2}, El{ts, u1, v1});
            }
    }
    if (c >= 1) {
        El Dl{2, c, -1};
        for (int tn = 0; tn < 2; ++tn) {
            El P{tn, m.a, m.b};
            put(P, Dl);
            put(Dl, P);
        }
    }
    if (!FILL) cnt[item] = k;
}

// ---- the diagonal coefficients, contracted in closed form
// items [0, P2): pair (j, k);  MODE 1 also [P2, P2 + (N-1)^2): the D^a, D^b block of
// sum_l x_l d(D^l, D^a, D^b) = [a == b] (2 c_a (1 - a) x_a + 2 sum_{l>a} c_l x_l)
//                            + [a < b] 2 c_b x_a + [a > b] 2 c_a x_b.
template <int MODE, bool FILL>
__global__ void k_emit_dpart(Basis B, const double2 *__restrict__ coef, bool conj, const double2 *__restrict__ Xd,
                             const double2 *__restrict__ suf, long long *__restrict__ cnt,
                             const long long *__restrict__ off, uint64_t *__restrict__ keys,
                             double2 *__restrict__ vals) {
    long long item = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long nd = (long long)(B.N - 1) * (B.N - 1);
    long long total = B.P2 + (MODE == 1 ? nd : 0);
    if (item >= total) return;
    long long o = FILL ? off[item] : 0;
    int k = 0;
    auto put = [&](long long row, long long col, double2 v) {
        if (v.x == 0.0 && v.y == 0.0) return;
        if (FILL) {
            keys[o + k] = mkkey(row, col, B.D);
            vals[o + k] = v;
        }
        ++k;
    };
    if (item < B.P2) {
        int j, kk;
        B.unpair(item, j, kk);
        double2 df = make_double2(Xd[j].x - Xd[kk].x, Xd[j].y - Xd[kk].y);
        long long sI = item, jI = B.P2 + item;
        if (MODE == 0) {
            put(jI, sI, df);                               // f(D, S, J): row J, column S
            put(sI, jI, make_double2(-df.x, -df.y));
        } else {
            double2 ds = make_double2(Xd[j].x + Xd[kk].x, Xd[j].y + Xd[kk].y);
            put(sI, jI, df);                               // Z_{S J} = sum x f(D, S, J)
            put(jI, sI, make_double2(-df.x, -df.y));
            put(sI, sI, make_double2(-ds.y, ds.x));        // i (Xd_j + Xd_k)
            put(jI, jI, make_double2(-ds.y, ds.x));
        }
    } else {
        long long q = item - B.P2;
        int a = (int)(q / (B.N - 1)) + 1, b = (int)(q % (B.N - 1)) + 1;
        auto xd = [&](int l) {
            double2 x = coef[2 * B.P2 + l - 1];
            if (conj) x.y = -x.y;
            return x;
        };
        double2 v;
        if (a == b) {
            double2 xa = xd(a);
            double ca = cl(a);
            v = make_double2(2.0 * ca * (1.0 - (double)a) * xa.x + 2.0 * suf[a].x,
                             2.0 * ca * (1.0 - (double)a) * xa.y + 2.0 * suf[a].y);
        } else if (a < b) {
            double2 xa = xd(a);
            v = make_double2(2.0 * cl(b) * xa.x, 2.0 * cl(b) * xa.y);
        } else {
            double2 xb = xd(b);
            v = make_double2(2.0 * cl(a) * xb.x, 2.0 * cl(a) * xb.y);
        }
        put(2 * B.P2 + a - 1, 2 * B.P2 + b - 1, make_double2(-v.y, v.x));   // times i
    }
    if (!FILL) cnt[item] = k;
}

// ---- sparse-sparse product, one thread per run of 8 products

__global__ void k_rowids(const int *__restrict__ rowptr, long long nrows, int *__restrict__ rowid) {
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    for (int e = rowptr[r]; e < rowptr[r + 1]; ++e) rowid[e] = (int)r;
}

__global__ void k_spgemm_count(const int *__restrict__ acol, long long nnza, const int *__restrict__ bptr,
                               long long *__restrict__ cnt) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nnza) cnt[e] = bptr[acol[e] + 1] - bptr[acol[e]];
}

// R-type product: value = scale * Re(a_e * b_f)
__global__ void k_spgemm_fill(const int *__restrict__ arow, const int *__restrict__ acol,
                              const double2 *__restrict__ aval, long long nnza, const int *__restrict__ bptr,
                              const int *__restrict__ bcol, const double2 *__restrict__ bval,
                              const long long *__restrict__ off, long long P, long long ncols, double scale,
                              uint64_t *__restrict__ keys, double *__restrict__ vals) {
    long long p0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 8;
    if (p0 >= P) return;
    long long lo = 0, hi = nnza;   // largest e with off[e] <= p0
    while (lo < hi) {
        long long mid = (lo + hi + 1) >> 1;
        if (off[mid] <= p0) lo = mid;
        else hi = mid - 1;
    }
    long long e = lo;
    long long pend = p0 + 8 < P ? p0 + 8 : P;
    for (long long p = p0; p < pend; ++p) {
        while (off[e + 1] <= p) ++e;
        long long f = bptr[acol[e]] + (p - off[e]);
        keys[p] = mkkey(arow[e], bcol[f], ncols);
        double2 a = aval[e], b = bval[f];
        vals[p] = scale * (a.x * b.x - a.y * b.y);
    }
}

// K per unit rate: K_s = -(i/N) sum_l Q(conj l)_{s l} l_l, the real part Im(sum)/N
__global__ void k_kvec(const int *__restrict__ aptr, const int *__restrict__ acol, const double2 *__restrict__ aval,
                       long long rows, const double2 *__restrict__ l, int N, double *__restrict__ K) {
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= rows) return;
    double2 sum = make_double2(0.0, 0.0);
    for (int e = aptr[s]; e < aptr[s + 1]; ++e) {
        double2 p = cmul(aval[e], l[acol[e]]);
        sum.x += p.x;
        sum.y += p.y;
    }
    K[s] = sum.y / (double)N;
}

// coefficients of the trace-part Hamiltonian per unit rate: -Im(conj(l0) l_j)
__global__ void k_heff_coef(const double2 *__restrict__ l, long long D, double2 l0, double2 *__restrict__ out) {
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= D) return;
    double2 x = l[j];
    // conj(l0) * x = (l0r - i l0i)(xr + i xi); imaginary part l0r xi - l0i xr
    out[j] = make_double2(-(l0.x * x.y - l0.y * x.x), 0.0);
}

__global__ void k_real_of(const double2 *__restrict__ in, double *__restrict__ out, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i].x;
}

__global__ void k_emit_csr(const int *__restrict__ rowptr, const int *__restrict__ col, const double *__restrict__ val,
                           long long nrows, long long ncols, double w, uint64_t *__restrict__ keys,
                           double *__restrict__ vals) {
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    for (int e = rowptr[r]; e < rowptr[r + 1]; ++e) {
        keys[e] = mkkey(r, col[e], ncols);
        vals[e] = w * val[e];
    }
}

__global__ void k_emit_transposed(const int *__restrict__ rowptr, const int *__restrict__ col,
                                  const double *__restrict__ val, long long nrows, long long ncols_t,
                                  uint64_t *__restrict__ keys, double *__restrict__ vals) {
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    for (int e = rowptr[r]; e < rowptr[r + 1]; ++e) {
        keys[e] = mkkey(col[e], r, ncols_t);
        vals[e] = val[e];
    }
}

__global__ void k_emit_kcol(const double *__restrict__ K, long long D, uint64_t *__restrict__ keys,
                            double *__restrict__ vals) {
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= D) return;
    keys[r] = mkkey(r, D, D + 1);
    vals[r] = K[r];
}

__global__ void k_axpy(double *__restrict__ y, const double *__restrict__ x, double a, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] += a * x[i];
}

// ---- helpers

struct Coo {
    DBuf<uint64_t> keys;
    DBuf<double2> vals;
    long long n = 0;
};

// Emit Q(x) (MODE 0) or Z(x) (MODE 1) for a dense coefficient vector into a complex COO.
template <int MODE>
void emit_contraction(gksl_ctx *c, const double2 *coef, bool conj, Coo &out) {
    Basis B(c->N);
    cudaStream_t s = c->stream;
    long long npair = 2 * B.P2;
    // nonzero pair coefficients
    DBuf<long long> flag((size_t)npair), pos((size_t)npair + 1);
    k_nz_flags<<<grid_for(npair, 256), 256, 0, s>>>(coef, npair, flag.p);
    GK_LAUNCH_CHECK();
    long long nnz = scan_ll(flag.p, pos.p, npair, true, true, s);
    DBuf<long long> nzi((size_t)nnz);
    DBuf<double2> nzv((size_t)nnz);
    k_nz_gather<<<grid_for(npair, 256), 256, 0, s>>>(coef, npair, flag.p, pos.p, conj, nzi.p, nzv.p);
    GK_LAUNCH_CHECK();
    flag.release();
    pos.release();
    // diagonal part
    DBuf<double2> Xd((size_t)c->N), suf((size_t)c->N);
    k_dpart_prep<<<1, 1, 0, s>>>(c->N, B.P2, coef, conj, Xd.p, suf.p);
    GK_LAUNCH_CHECK();
    long long items_p = nnz * (long long)c->N;
    long long items_d = B.P2 + (MODE == 1 ? (long long)(c->N - 1) * (c->N - 1) : 0);
    GK_REQUIRE(items_p < (1LL << 40), GKSL_ERR_ARG, "operator too dense for the sparse contraction");
    long long items = items_p + items_d;
    DBuf<long long> cnt((size_t)items), off((size_t)items + 1);
    if (items_p > 0) {
        k_emit_pairs<MODE, false><<<grid_for(items_p, 256), 256, 0, s>>>(B, nzi.p, nzv.p, nnz, cnt.p, nullptr,
                                                                          nullptr, nullptr);
        GK_LAUNCH_CHECK();
    }
    k_emit_dpart<MODE, false><<<grid_for(items_d, 256), 256, 0, s>>>(B, coef, conj, Xd.p, suf.p, cnt.p + items_p,
                                                                      nullptr, nullptr, nullptr);
    GK_LAUNCH_CHECK();
    long long total = scan_ll(cnt.p, off.p, items, true, true, s);
    out.keys.alloc((size_t)total);
    out.vals.alloc((size_t)total);
    out.n = total;
    if (items_p > 0) {
        k_emit_pairs<MODE, true><<<grid_for(items_p, 256), 256, 0, s>>>(B, nzi.p, nzv.p, nnz, nullptr, off.p,
                                                                         out.keys.p, out.vals.p);
        GK_LAUNCH_CHECK();
    }
    k_emit_dpart<MODE, true><<<grid_for(items_d, 256), 256, 0, s>>>(B, coef, conj, Xd.p, suf.p, nullptr,
                                                                     off.p + items_p, out.keys.p, out.vals.p);
    GK_LAUNCH_CHECK();
    GK_CUDA(cudaStreamSynchronize(s));
}

void to_real(const CsrC &a, CsrR &r, cudaStream_t s) {
    r.rows = a.rows;
    r.cols = a.cols;
    r.nnz = a.nnz;
    r.rowptr.alloc((size_t)a.rows + 1);
    r.col.alloc((size_t)(a.nnz > 0 ? a.nnz : 1));
    r.val.alloc((size_t)(a.nnz > 0 ? a.nnz : 1));
    GK_CUDA(cudaMemcpyAsync(r.rowptr.p, a.rowptr.p, sizeof(int) * (a.rows + 1), cudaMemcpyDeviceToDevice, s));
    if (a.nnz > 0) {
        GK_CUDA(cudaMemcpyAsync(r.col.p, a.col.p, sizeof(int) * a.nnz, cudaMemcpyDeviceToDevice, s));
        k_real_of<<<grid_for(a.nnz, 256), 256, 0, s>>>(a.val.p, r.val.p, a.nnz);
        GK_LAUNCH_CHECK();
    }
    GK_CUDA(cudaStreamSynchronize(s));
}

// Q(x) of a Hermitian operator's coefficients, real CSR
void hamiltonian_matrix(gksl_ctx *c, const Op &op, CsrR &out) {
    DBuf<double2> coef;
    expand_op(c, op, coef);
    Coo coo;
    emit_contraction<0>(c, coef.p, false, coo);
    CsrC q;
    coo_to_csr_cplx(coo.keys, coo.vals, coo.n, c->D, c->D, 0.0, q, c->stream);
    to_real(q, out, c->stream);
}

// R_p and K_p at unit rate for one dissipator
void dissipator_matrix(gksl_ctx *c, const Op &op, CsrR &R, DBuf<double> &K) {
    cudaStream_t s = c->stream;
    long long D = c->D;
    DBuf<double2> l;
    expand_op(c, op, l);
    // F''^T = Q(conj l), Z'' = Z(l)
    CsrC A, Z;
    {
        Coo coo;
        emit_contraction<0>(c, l.p, true, coo);
        coo_to_csr_cplx(coo.keys, coo.vals, coo.n, D, D, 0.0, A, s);
    }
    {
        Coo coo;
        emit_contraction<1>(c, l.p, false, coo);
        coo_to_csr_cplx(coo.keys, coo.vals, coo.n, D, D, 0.0, Z, s);
    }
    // K = -(i/N) Q(conj l) l
    K.alloc((size_t)D);
    k_kvec<<<grid_for(D, 256), 256, 0, s>>>(A.rowptr.p, A.col.p, A.val.p, D, l.p, c->N, K.p);
    GK_LAUNCH_CHECK();
    // trace part of L: l0 = Tr(L)/N, from the host copy of the diagonal
    double2 l0 = make_double2(0.0, 0.0);
    {
        std::vector<int> rp(c->N + 1), cc(op.nnz > 0 ? op.nnz : 1);
        std::vector<double> re(op.nnz > 0 ? op.nnz : 1), im(op.nnz > 0 ? op.nnz : 1);
        GK_CUDA(cudaMemcpyAsync(rp.data(), op.rowptr.p, sizeof(int) * (c->N + 1), cudaMemcpyDeviceToHost, s));
        if (op.nnz > 0) {
            GK_CUDA(cudaMemcpyAsync(cc.data(), op.col.p, sizeof(int) * op.nnz, cudaMemcpyDeviceToHost, s));
            GK_CUDA(cudaMemcpyAsync(re.data(), op.re.p, sizeof(double) * op.nnz, cudaMemcpyDeviceToHost, s));
            GK_CUDA(cudaMemcpyAsync(im.data(), op.im.p, sizeof(double) * op.nnz, cudaMemcpyDeviceToHost, s));
        }
        GK_CUDA(cudaStreamSynchronize(s));
        for (int r = 0; r < c->N; ++r)
            for (int e = rp[r]; e < rp[r + 1]; ++e)
                if (cc[e] == r) { l0.x += re[e]; l0.y += im[e]; }
        l0.x /= c->N;
        l0.y /= c->N;
    }
    // products of the row-wise sparse-sparse product
    long long nnza = A.nnz;
    DBuf<int> arow((size_t)(nnza > 0 ? nnza : 1));
    k_rowids<<<grid_for(D, 256), 256, 0, s>>>(A.rowptr.p, D, arow.p);
    GK_LAUNCH_CHECK();
    DBuf<long long> cnt((size_t)(nnza > 0 ? nnza : 1)), off((size_t)nnza + 1);
    if (nnza > 0) {
        k_spgemm_count<<<grid_for(nnza, 256), 256, 0, s>>>(A.col.p, nnza, Z.rowptr.p, cnt.p);
        GK_LAUNCH_CHECK();
    }
    long long P = scan_ll(cnt.p, off.p, nnza, true, true, s);
    if (P > 2 * D * D && c->N <= kDenseDissMaxN) {
        // a dense operator: the product has more terms than R has entries, so form R entry by
        // entry from the matrix-unit form instead (dense_diss.cu)
        cnt.release();
        off.release();
        arow.release();
        dense_dissipator_channel(c, op, R, K);
        return;
    }
    // trace-part Hamiltonian entries (complex COO, real parts used)
    Coo heff;
    if (l0.x != 0.0 || l0.y != 0.0) {
        DBuf<double2> hc((size_t)D);
        k_heff_coef<<<grid_for(D, 256), 256, 0, s>>>(l.p, D, l0, hc.p);
        GK_LAUNCH_CHECK();
        emit_contraction<0>(c, hc.p, false, heff);
    }
    long long n = P + heff.n;
    DBuf<uint64_t> keys((size_t)n);
    DBuf<double> vals((size_t)n);
    if (P > 0) {
        k_spgemm_fill<<<grid_for((P + 7) / 8, 256), 256, 0, s>>>(arow.p, A.col.p, A.val.p, nnza, Z.rowptr.p, Z.col.p,
                                                                   Z.val.p, off.p, P, D, -0.5, keys.p, vals.p);
        GK_LAUNCH_CHECK();
    }
    if (heff.n > 0) {
        GK_CUDA(cudaMemcpyAsync(keys.p + P, heff.keys.p, sizeof(uint64_t) * heff.n, cudaMemcpyDeviceToDevice, s));
        k_real_of<<<grid_for(heff.n, 256), 256, 0, s>>>(heff.vals.p, vals.p + P, heff.n);
        GK_LAUNCH_CHECK();
    }
    GK_CUDA(cudaStreamSynchronize(s));
    cnt.release();
    off.release();
    arow.release();
    coo_to_csr_real(keys, vals, n, D, D, 0.0, R, s);
}

// sum_i w_i M_i (+ optional K column at index D) -> CSR, dropping |q| <= drop_rel * max|q|
void merge(gksl_ctx *c, const std::vector<std::pair<const CsrR *, double>> &terms, const double *Kcol,
           double drop_rel, CsrR &out, double *max_abs_out) {
    cudaStream_t s = c->stream;
    long long D = c->D;
    long long ncols = Kcol ? D + 1 : D;
    long long n = Kcol ? D : 0;
    for (auto &t : terms) n += t.first->nnz;
    DBuf<uint64_t> keys((size_t)n);
    DBuf<double> vals((size_t)n);
    long long o = 0;
    for (auto &t : terms) {
        if (t.first->nnz > 0) {
            k_emit_csr<<<grid_for(D, 256), 256, 0, s>>>(t.first->rowptr.p, t.first->col.p, t.first->val.p, D, ncols,
                                                         t.second, keys.p + o, vals.p + o);
            GK_LAUNCH_CHECK();
        }
        o += t.first->nnz;
    }
    if (Kcol) {
        k_emit_kcol<<<grid_for(D, 256), 256, 0, s>>>(Kcol, D, keys.p + o, vals.p + o);
        GK_LAUNCH_CHECK();
    }
    GK_CUDA(cudaStreamSynchronize(s));
    CsrR tmp;
    coo_to_csr_real(keys, vals, n, D, ncols, 0.0, tmp, s);
    double mx = max_abs(tmp.val.p, tmp.nnz, s);
    if (max_abs_out) *max_abs_out = mx;
    if (drop_rel > 0.0 && tmp.nnz > 0) {
        // rebuild from the reduced entries with the drop applied
        DBuf<uint64_t> k2((size_t)tmp.nnz);
        DBuf<double> v2((size_t)tmp.nnz);
        k_emit_csr<<<grid_for(D, 256), 256, 0, s>>>(tmp.rowptr.p, tmp.col.p, tmp.val.p, D, ncols, 1.0, k2.p, v2.p);
        GK_LAUNCH_CHECK();
        GK_CUDA(cudaStreamSynchronize(s));
        coo_to_csr_real(k2, v2, tmp.nnz, D, ncols, drop_rel * mx, out, s);
    } else {
        out = std::move(tmp);
    }
}

}  // namespace

void merge_terms(gksl_ctx *c, const std::vector<std::pair<const CsrR *, double>> &terms, const double *Kcol,
                 CsrR &out) {
    merge(c, terms, Kcol, 0.0, out, nullptr);
}

void csr_transpose(const CsrR &a, CsrR &t, cudaStream_t s) {
    DBuf<uint64_t> keys((size_t)(a.nnz > 0 ? a.nnz : 1));
    DBuf<double> vals((size_t)(a.nnz > 0 ? a.nnz : 1));
    if (a.nnz > 0) {
        k_emit_transposed<<<grid_for(a.rows, 256), 256, 0, s>>>(a.rowptr.p, a.col.p, a.val.p, a.rows, a.rows, keys.p,
                                                                vals.p);
        GK_LAUNCH_CHECK();
    }
    GK_CUDA(cudaStreamSynchronize(s));
    coo_to_csr_real(keys, vals, a.nnz, a.cols, a.rows, -1.0, t, s);
}

void assemble(gksl_ctx *c, unsigned flags) {
    auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = c->stream;
    long long D = c->D;
    GK_REQUIRE(c->drive_set, GKSL_ERR_STATE, "gksl_set_drive must be called before gksl_assemble");
    bool any = c->h1.set;
    for (int k = 0; k < GKSL_MAX_H0; ++k) any = any || c->h0[k].set;
    for (int p = 0; p < GKSL_MAX_P; ++p) any = any || c->diss[p].set;
    GK_REQUIRE(any, GKSL_ERR_STATE, "no operator set before gksl_assemble");
    if (flags & GKSL_ASM_MATRIX_FREE) {
        GK_REQUIRE(!(flags & GKSL_ASM_TRANSPOSE), GKSL_ERR_ARG,
                   "GKSL_ASM_MATRIX_FREE excludes GKSL_ASM_TRANSPOSE (the adjoint needs CSR matrices)");
        c->Q0 = CsrR();
        c->K.release();
        c->hyb0 = Hyb<double>();
        c->hyb1 = Hyb<double>();
        c->hyb0f = Hyb<float>();
        c->hyb1f = Hyb<float>();
        c->q1_folded = false;
        c->q1v.release();
        c->q1vf.release();
        for (int i = 0; i < gksl_ctx::kMaxCh; ++i) {
            c->adj[i] = Hyb<double>();
            c->adjf[i] = Hyb<float>();
        }
        c->has_adj = false;
        c->adj_n = 0;
        c->nnz_q0e = 0;
        c->max_abs_q0 = 0.0;
        mf_build(c, (flags & GKSL_ASM_FP32) != 0);
        c->asm_flags = flags;
        c->assembled = true;
        c->rk4_tuned[0] = c->rk4_tuned[1] = false;
        clear_graphs(c);
        c->assemble_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        return;
    }
    c->mf = MfBands();
    const bool dense_diss = (flags & GKSL_ASM_DENSE_DISSIPATORS) != 0;
    if (dense_diss != c->comp_dense) c->comp_dirty = true;
    if (c->comp_dirty) {
        for (int k = 0; k < GKSL_MAX_H0; ++k) {
            c->has_h0[k] = c->h0[k].set;
            if (c->h0[k].set) hamiltonian_matrix(c, c->h0[k], c->QH0[k]);
            else c->QH0[k] = CsrR();
        }
        if (c->h1.set) hamiltonian_matrix(c, c->h1, c->Q1);
        else {
            Op zero;
            zero.set = true;
            zero.nnz = 0;
            zero.rowptr.alloc((size_t)c->N + 1);
            GK_CUDA(cudaMemsetAsync(zero.rowptr.p, 0, sizeof(int) * (c->N + 1), s));
            hamiltonian_matrix(c, zero, c->Q1);
        }
        for (int p = 0; p < GKSL_MAX_P; ++p) {
            c->has_r[p] = c->diss[p].set;
            if (!c->diss[p].set) { c->R[p] = CsrR(); c->Kp[p].release(); }
            else if (c->diss[p].km) dense_dissipator_kossakowski(c, c->km_A.p, c->R[p], c->Kp[p]);
            else if (dense_diss) dense_dissipator_channel(c, c->diss[p], c->R[p], c->Kp[p]);
            else dissipator_matrix(c, c->diss[p], c->R[p], c->Kp[p]);
        }
        c->comp_dense = dense_diss;
        c->comp_dirty = false;
    }
    // K = sum_p gamma_p K_p
    c->K.alloc((size_t)D + 1);
    GK_CUDA(cudaMemsetAsync(c->K.p, 0, sizeof(double) * (D + 1), s));
    for (int p = 0; p < GKSL_MAX_P; ++p)
        if (c->has_r[p]) {
            k_axpy<<<grid_for(D, 256), 256, 0, s>>>(c->K.p, c->Kp[p].p, c->diss[p].weight, D);
            GK_LAUNCH_CHECK();
        }
    double drop = (flags & GKSL_ASM_NO_DROP) ? 0.0 : 64.0 * 2.220446049250313e-16;
    std::vector<std::pair<const CsrR *, double>> terms;
    for (int k = 0; k < GKSL_MAX_H0; ++k)
        if (c->has_h0[k]) terms.push_back({&c->QH0[k], c->h0[k].weight});
    for (int p = 0; p < GKSL_MAX_P; ++p)
        if (c->has_r[p]) terms.push_back({&c->R[p], c->diss[p].weight});
    merge(c, terms, nullptr, drop, c->Q0, nullptr);
    // propagation matrix [Q0 + E Q1 | K]
    auto terms_e = terms;
    terms_e.push_back({&c->Q1, c->E});
    CsrR q0e;
    merge(c, terms_e, c->K.p, drop, q0e, &c->max_abs_q0);
    c->nnz_q0e = q0e.nnz;
    bool fp32 = (flags & GKSL_ASM_FP32) != 0;
    build_hyb_pair(q0e, c->Q1, D, c->hyb0, c->hyb1, fp32 ? &c->hyb0f : nullptr, fp32 ? &c->hyb1f : nullptr, s);
    c->q1_folded = !(flags & GKSL_ASM_NO_FOLD) &&
                   fold_q1(q0e, c->Q1, D, c->hyb0, fp32 ? &c->hyb0f : nullptr, c->q1v, c->q1vf, s);
    // 16-bit relative columns for the folded stage stream (built from the final slot order)
    drop_c16(c->hyb0);
    drop_c16(c->hyb0f);
    if (c->q1_folded && !(flags & GKSL_ASM_WIDE_COLUMNS)) {
        build_c16(c->hyb0, c->P2, s);
        if (fp32) build_c16(c->hyb0f, c->P2, s);
    }
    c->has_adj = false;
    c->adj_n = 0;
    if (flags & GKSL_ASM_TRANSPOSE) {
        std::vector<const CsrR *> ms;
        std::vector<double> sc;
        std::vector<CsrR> rts((size_t)GKSL_MAX_P);
        int n = 0;
        for (int k = 0; k < GKSL_MAX_H0; ++k)
            if (c->has_h0[k]) {
                ms.push_back(&c->QH0[k]);
                sc.push_back(-1.0);   // Q(H)^T = -Q(H)
                c->adj_kind[n] = 0;
                c->adj_index[n++] = k;
            }
        ms.push_back(&c->Q1);
        sc.push_back(-1.0);
        c->adj_kind[n] = 1;
        c->adj_index[n++] = 0;
        for (int p = 0; p < GKSL_MAX_P; ++p)
            if (c->has_r[p]) {
                csr_transpose(c->R[p], rts[p], s);
                ms.push_back(&rts[p]);
                sc.push_back(1.0);
                c->adj_kind[n] = 2;
                c->adj_index[n++] = p;
            }
        std::vector<Hyb<double> *> out;
        std::vector<Hyb<float> *> outf;
        for (int i = 0; i < n; ++i) {
            c->adj[i] = Hyb<double>();
            c->adjf[i] = Hyb<float>();
            out.push_back(&c->adj[i]);
            outf.push_back(fp32 ? &c->adjf[i] : nullptr);
        }
        build_hyb_multi(ms, sc, D, out, outf, s);
        c->adj_n = n;
        c->has_adj = true;
    }
    c->asm_flags = flags;
    c->assembled = true;
    c->rk4_tuned[0] = c->rk4_tuned[1] = false;   // a new matrix: time the stage-kernel variants again
    clear_graphs(c);
    GK_CUDA(cudaStreamSynchronize(s));
    c->assemble_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

void csr_copy_out(gksl_ctx *c, const CsrR &m, long long *nnz, int *rowptr, int *col, double *val) {
    *nnz = m.nnz;
    if (!rowptr) return;
    copy_out(rowptr, m.rowptr.p, sizeof(int) * (m.rows + 1), c->stream);
    if (m.nnz > 0) {
        if (col) copy_out(col, m.col.p, sizeof(int) * m.nnz, c->stream);
        if (val) copy_out(val, m.val.p, sizeof(double) * m.nnz, c->stream);
    }
    GK_CUDA(cudaStreamSynchronize(c->stream));
}

}  // namespace gk
