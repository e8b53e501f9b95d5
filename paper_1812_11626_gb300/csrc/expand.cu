// Expansion over the generator basis (Sec. IV step 2.1: h_j, l_j; step 2.6: v(0)),
// observables and the density matrix from the Bloch vector (Eq. 6).
#include "internal.cuh"
#include "prim.cuh"

namespace gk {

namespace {

// Off-diagonal entries of an N x N CSR operator X: entry (r, c), r != c, belongs to the pair
// (a, b) = (min, max) and adds X_rc/sqrt2 to Tr(S_ab X) and +-i X_rc/sqrt2 to Tr(J_ab X)
// (+ for r < c).  Each coefficient receives at most two contributions, so the atomic sum is
// order independent.  Diagonal entries are collected for the D^l coefficients.
__global__ void k_expand_offdiag(Basis B, const int *__restrict__ rowptr, const int *__restrict__ col,
                                 const double *__restrict__ re, const double *__restrict__ im,
                                 double2 *__restrict__ coef, double2 *__restrict__ diag) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= B.N) return;
    for (int e = rowptr[r]; e < rowptr[r + 1]; ++e) {
        int c = col[e];
        double xr = re[e], xi = im ? im[e] : 0.0;
        if (c == r) {
            diag[r] = make_double2(xr, xi);
            continue;
        }
        int a = r < c ? r : c, b = r < c ? c : r;
        long long p = B.pair(a, b);
        atomicAdd(&coef[p].x, xr * GK_RSQRT2);
        atomicAdd(&coef[p].y, xi * GK_RSQRT2);
        // i * (xr + i xi) = -xi + i xr
        double sg = r < c ? 1.0 : -1.0;
        atomicAdd(&coef[B.P2 + p].x, -sg * xi * GK_RSQRT2);
        atomicAdd(&coef[B.P2 + p].y, sg * xr * GK_RSQRT2);
    }
}

// Tr(D^l X) = c_l (sum_{k<l} X_kk - l X_ll), l = 1..N-1, from the diagonal by a block scan.
__global__ void k_expand_diag(int N, long long P2, const double2 *__restrict__ diag, double2 *__restrict__ coef) {
    __shared__ double2 carry;
    __shared__ double2 wsum[32];
    if (threadIdx.x == 0) carry = make_double2(0.0, 0.0);
    __syncthreads();
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int base = 0; base < N; base += blockDim.x) {
        int k = base + threadIdx.x;
        double2 x = k < N ? diag[k] : make_double2(0.0, 0.0);
        // inclusive scan of x over the block
        double2 inc = x;
        for (int o = 1; o < 32; o <<= 1) {
            double yx = __shfl_up_sync(0xffffffffu, inc.x, o), yy = __shfl_up_sync(0xffffffffu, inc.y, o);
            if (lane >= o) { inc.x += yx; inc.y += yy; }
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            double2 w = lane < nw ? wsum[lane] : make_double2(0.0, 0.0);
            double2 wi = w;
            for (int o = 1; o < 32; o <<= 1) {
                double yx = __shfl_up_sync(0xffffffffu, wi.x, o), yy = __shfl_up_sync(0xffffffffu, wi.y, o);
                if (lane >= o) { wi.x += yx; wi.y += yy; }
            }
            if (lane < nw) wsum[lane] = make_double2(wi.x - w.x, wi.y - w.y);
        }
        __syncthreads();
        double2 excl = make_double2(carry.x + wsum[warp].x + inc.x - x.x, carry.y + wsum[warp].y + inc.y - x.y);
        if (k >= 1 && k < N) {
            double c = cl(k);
            coef[2 * P2 + k - 1] = make_double2(c * (excl.x - (double)k * x.x), c * (excl.y - (double)k * x.y));
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = make_double2(excl.x + x.x, excl.y + x.y);
        __syncthreads();
    }
}

// dense matrix (row-major, N x N) -> real coefficients; off-diagonal part
__global__ void k_expand_dense_pairs(Basis B, const double *__restrict__ re, const double *__restrict__ im,
                                     double *__restrict__ v) {
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= B.P2) return;
    int a, b;
    B.unpair(p, a, b);
    double xab_r = re[(long long)a * B.N + b], xba_r = re[(long long)b * B.N + a];
    double xab_i = im ? im[(long long)a * B.N + b] : 0.0, xba_i = im ? im[(long long)b * B.N + a] : 0.0;
    // Re Tr(S X) = Re(X_ab + X_ba)/sqrt2; Re Tr(J X) = Re(i (X_ab - X_ba))/sqrt2 = -(Im X_ab - Im X_ba)/sqrt2
    v[p] = (xab_r + xba_r) * GK_RSQRT2;
    v[B.P2 + p] = -(xab_i - xba_i) * GK_RSQRT2;
}

__global__ void k_gather_diag(int N, const double *__restrict__ re, const double *__restrict__ im,
                              double2 *__restrict__ diag) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < N) diag[k] = make_double2(re[(long long)k * N + k], im ? im[(long long)k * N + k] : 0.0);
}

__global__ void k_real_part(const double2 *__restrict__ c, double *__restrict__ v, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = c[i].x;
}

// <O> = c0 + sum_l w_l v_{D^l}; one block per vector, fixed-order reduction
__global__ void k_observable(const double *__restrict__ w, const double *__restrict__ c0, long long P2, int N,
                             const double *__restrict__ v, long long ldv, double *__restrict__ out) {
    const double *vv = v + (long long)blockIdx.x * ldv + 2 * P2;
    double s = 0.0;
    for (int l = threadIdx.x; l < N - 1; l += blockDim.x) s += w[2 * P2 + l] * vv[l];
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = *c0 + red[0];
}

// w_l = Tr(O D^l) = c_l (sum_{k<l} o_k - l o_l), c0 = Tr(O)/N  (small N-length sequential scan)
__global__ void k_obs_weights(int N, long long P2, long long D, const double *__restrict__ o,
                              double *__restrict__ w, double *__restrict__ c0) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double pre = 0.0;
    for (int l = 0; l < N; ++l) {
        if (l >= 1) w[2 * P2 + l - 1] = cl(l) * (pre - (double)l * o[l]);
        pre += o[l];
    }
    *c0 = pre / N;
}

__global__ void k_zero(double *w, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) w[i] = 0.0;
}

// rho = 1/N + sum_j v_j F_j: off-diagonal entries from the S/J pair coefficients
__global__ void k_rho_pairs(Basis B, const double *__restrict__ v, double *__restrict__ re, double *__restrict__ im) {
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= B.P2) return;
    int a, b;
    B.unpair(p, a, b);
    double s = v[p] * GK_RSQRT2, j = v[B.P2 + p] * GK_RSQRT2;
    // S_ab: 1/sqrt2 at (a,b),(b,a); J_ab: -i/sqrt2 at (a,b), +i/sqrt2 at (b,a)
    re[(long long)a * B.N + b] = s;
    im[(long long)a * B.N + b] = -j;
    re[(long long)b * B.N + a] = s;
    im[(long long)b * B.N + a] = j;
}

// diagonal: rho_kk = 1/N + sum_{l>k} c_l v_{D^l} - k c_k v_{D^k}
__global__ void k_rho_diag(int N, long long P2, const double *__restrict__ v, double *__restrict__ re,
                           double *__restrict__ im) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double suf = 0.0;
    for (int k = N - 1; k >= 0; --k) {
        double own = k >= 1 ? -(double)k * cl(k) * v[2 * P2 + k - 1] : 0.0;
        re[(long long)k * N + k] = 1.0 / N + suf + own;
        im[(long long)k * N + k] = 0.0;
        if (k >= 1) suf += cl(k) * v[2 * P2 + k - 1];
    }
}

}  // namespace

void expand_op(gksl_ctx *c, const Op &op, DBuf<double2> &coef) {
    Basis B(c->N);
    coef.alloc((size_t)B.D);
    DBuf<double2> diag((size_t)c->N);
    GK_CUDA(cudaMemsetAsync(coef.p, 0, sizeof(double2) * B.D, c->stream));
    GK_CUDA(cudaMemsetAsync(diag.p, 0, sizeof(double2) * c->N, c->stream));
    if (op.nnz > 0) {
        k_expand_offdiag<<<grid_for(c->N, 128), 128, 0, c->stream>>>(B, op.rowptr.p, op.col.p, op.re.p, op.im.p,
                                                                      coef.p, diag.p);
        GK_LAUNCH_CHECK();
    }
    k_expand_diag<<<1, 1024, 0, c->stream>>>(c->N, B.P2, diag.p, coef.p);
    GK_LAUNCH_CHECK();
    GK_CUDA(cudaStreamSynchronize(c->stream));
}

void expand_dense(gksl_ctx *c, const double *re, const double *im, double *v) {
    Basis B(c->N);
    k_expand_dense_pairs<<<grid_for(B.P2, 256), 256, 0, c->stream>>>(B, re, im, v);
    GK_LAUNCH_CHECK();
    DBuf<double2> diag((size_t)c->N), coef((size_t)B.D);
    k_gather_diag<<<grid_for(c->N, 256), 256, 0, c->stream>>>(c->N, re, im, diag.p);
    GK_LAUNCH_CHECK();
    k_expand_diag<<<1, 1024, 0, c->stream>>>(c->N, B.P2, diag.p, coef.p);
    GK_LAUNCH_CHECK();
    k_real_part<<<grid_for(c->N, 256), 256, 0, c->stream>>>(coef.p + 2 * B.P2, v + 2 * B.P2, c->N - 1);
    GK_LAUNCH_CHECK();
    GK_CUDA(cudaStreamSynchronize(c->stream));
}

void observable_weights(gksl_ctx *c, const double *o, double *w, double *c0) {
    Basis B(c->N);
    k_zero<<<grid_for(B.D, 256), 256, 0, c->stream>>>(w, B.D);
    GK_LAUNCH_CHECK();
    k_obs_weights<<<1, 1, 0, c->stream>>>(c->N, B.P2, B.D, o, w, c0);
    GK_LAUNCH_CHECK();
}

void observable_apply(gksl_ctx *c, const double *w, const double *c0, const double *v, long long count, long long ldv,
                      double *out) {
    Basis B(c->N);
    if (count > 0) {
        k_observable<<<(unsigned)count, 256, 0, c->stream>>>(w, c0, B.P2, c->N, v, ldv, out);
        GK_LAUNCH_CHECK();
    }
}

void observable_diag(gksl_ctx *c, const double *o, const double *v, long long count, long long ldv, double *out) {
    Basis B(c->N);
    DBuf<double> w((size_t)B.D), c0(1);
    observable_weights(c, o, w.p, c0.p);
    observable_apply(c, w.p, c0.p, v, count, ldv, out);
    GK_CUDA(cudaStreamSynchronize(c->stream));
}

void rho_dense(gksl_ctx *c, const double *v, double *re, double *im) {
    Basis B(c->N);
    k_rho_pairs<<<grid_for(B.P2, 256), 256, 0, c->stream>>>(B, v, re, im);
    GK_LAUNCH_CHECK();
    k_rho_diag<<<1, 1, 0, c->stream>>>(c->N, B.P2, v, re, im);
    GK_LAUNCH_CHECK();
    GK_CUDA(cudaStreamSynchronize(c->stream));
}

}  // namespace gk
