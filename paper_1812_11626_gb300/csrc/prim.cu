// Scan, stable LSD radix sort and COO -> CSR reduction (assembly building blocks).
#include "prim.cuh"

#include <cstring>

namespace gk {

namespace {

constexpr int kT = 256;          // threads per block for scans and the sort
constexpr int kI = 8;            // items per thread
constexpr int kTile = kT * kI;   // 2048
constexpr unsigned kFull = 0xffffffffu;

template <typename T>
__device__ T warp_inclusive(T x) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// exclusive scan across a 256-thread block; `total` receives the block sum
template <typename T>
__device__ T block_exclusive(T x, T &total) {
    __shared__ T wsum[kT / 32 + 1];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = warp_inclusive(x);
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < kT / 32 ? wsum[lane] : T(0);
        T wi = warp_inclusive(w);
        if (lane < kT / 32) wsum[lane] = wi - w;
        if (lane == kT / 32 - 1) wsum[kT / 32] = wi;  // block total (slot 8 of a 9-slot array below)
    }
    __syncthreads();
    T r = wsum[warp] + inc - x;
    total = wsum[kT / 32];
    __syncthreads();
    return r;
}

template <typename TIn>
__global__ void k_tile_sums(const TIn *__restrict__ in, long long n, long long *__restrict__ sums) {
    long long base = (long long)blockIdx.x * kTile;
    long long s = 0;
    for (int i = threadIdx.x; i < kTile; i += kT) {
        long long j = base + i;
        if (j < n) s += (long long)in[j];
    }
    // block reduction
    __shared__ long long red[kT];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = kT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = red[0];
}

template <typename TIn>
__global__ void k_tile_apply(const TIn *__restrict__ in, long long *__restrict__ out, long long n,
                             const long long *__restrict__ offs) {
    long long base = (long long)blockIdx.x * kTile + (long long)threadIdx.x * kI;
    long long loc[kI];
    long long run = 0;
#pragma unroll
    for (int i = 0; i < kI; ++i) {
        long long j = base + i;
        long long x = j < n ? (long long)in[j] : 0;
        loc[i] = run;
        run += x;
    }
    long long tot;
    long long pre = block_exclusive<long long>(run, tot);
    long long off = offs[blockIdx.x] + pre;
#pragma unroll
    for (int i = 0; i < kI; ++i) {
        long long j = base + i;
        if (j < n) out[j] = off + loc[i];
    }
}

__global__ void k_set_ll(long long *p, long long v) { *p = v; }

template <typename TIn>
long long scan_impl(const TIn *in, long long *out, long long n, bool with_total, bool want_total, cudaStream_t s) {
    if (n <= 0) {
        if (with_total) { k_set_ll<<<1, 1, 0, s>>>(out, 0); GK_LAUNCH_CHECK(); }
        return 0;
    }
    long long nt = (n + kTile - 1) / kTile;
    DBuf<long long> sums((size_t)nt), offs((size_t)nt + 1);
    k_tile_sums<TIn><<<(unsigned)nt, kT, 0, s>>>(in, n, sums.p);
    GK_LAUNCH_CHECK();
    if (nt == 1) {
        // one tile: its offset is 0 and the total is its sum (no further recursion)
        k_set_ll<<<1, 1, 0, s>>>(offs.p, 0);
        GK_LAUNCH_CHECK();
        GK_CUDA(cudaMemcpyAsync(offs.p + 1, sums.p, sizeof(long long), cudaMemcpyDeviceToDevice, s));
    } else {
        scan_impl<long long>(sums.p, offs.p, nt, true, false, s);
    }
    k_tile_apply<TIn><<<(unsigned)nt, kT, 0, s>>>(in, out, n, offs.p);
    GK_LAUNCH_CHECK();
    if (with_total) GK_CUDA(cudaMemcpyAsync(out + n, offs.p + nt, sizeof(long long), cudaMemcpyDeviceToDevice, s));
    long long total = 0;
    if (want_total) {
        GK_CUDA(cudaMemcpyAsync(&total, offs.p + nt, sizeof(long long), cudaMemcpyDeviceToHost, s));
        GK_CUDA(cudaStreamSynchronize(s));
    } else {
        // keep the temporaries alive until the kernels using them have run
        GK_CUDA(cudaStreamSynchronize(s));
    }
    return total;
}

// ------------------------------------------------------------------ radix sort

constexpr int kBins = 256;

__global__ void k_iota(uint32_t *p, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = (uint32_t)i;
}

__global__ void k_rs_hist(const uint64_t *__restrict__ keys, long long n, int shift, long long *__restrict__ hist,
                          long long ntiles) {
    __shared__ unsigned h[kBins];
    for (int i = threadIdx.x; i < kBins; i += kT) h[i] = 0;
    __syncthreads();
    long long base = (long long)blockIdx.x * kTile;
    for (int i = threadIdx.x; i < kTile; i += kT) {
        long long j = base + i;
        if (j < n) atomicAdd(&h[(unsigned)(keys[j] >> shift) & (kBins - 1)], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kBins; b += kT) hist[(long long)b * ntiles + blockIdx.x] = h[b];
}

// Stable scatter: each warp owns 256 consecutive items (8 rounds of 32); ranks within a round
// come from __match_any_sync, within a warp from per-warp digit counters, across warps from
// a prefix over the 8 warps, across tiles from the scanned histogram.
__global__ void k_rs_scatter(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                             uint64_t *__restrict__ kout, uint32_t *__restrict__ vout, long long n, int shift,
                             const long long *__restrict__ offs, long long ntiles) {
    __shared__ unsigned wcnt[kT / 32][kBins];
    __shared__ long long boff[kBins];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < (kT / 32) * kBins; i += kT) (&wcnt[0][0])[i] = 0;
    for (int b = threadIdx.x; b < kBins; b += kT) boff[b] = offs[(long long)b * ntiles + blockIdx.x];
    __syncthreads();
    long long base = (long long)blockIdx.x * kTile + (long long)warp * (32 * kI);
    uint64_t k[kI];
    uint32_t v[kI];
    unsigned rank[kI];
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < kI; ++r) {
        long long j = base + (long long)r * 32 + lane;
        bool valid = j < n;
        unsigned active = __ballot_sync(kFull, valid);
        unsigned d = 0;
        if (valid) {
            k[r] = kin[j];
            v[r] = vin[j];
            d = (unsigned)(k[r] >> shift) & (kBins - 1);
            unsigned peers = __match_any_sync(active, d);
            rank[r] = wcnt[warp][d] + __popc(peers & lt);
            __syncwarp(active);
            if ((peers & lt) == 0) wcnt[warp][d] += __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kBins; b += kT) {
        unsigned run = 0;
        for (int w = 0; w < kT / 32; ++w) {
            unsigned t = wcnt[w][b];
            wcnt[w][b] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kI; ++r) {
        long long j = base + (long long)r * 32 + lane;
        if (j < n) {
            unsigned d = (unsigned)(k[r] >> shift) & (kBins - 1);
            long long pos = boff[d] + wcnt[warp][d] + rank[r];
            kout[pos] = k[r];
            vout[pos] = v[r];
        }
    }
}

// ------------------------------------------------------------------ reduce by key

__global__ void k_heads(const uint64_t *__restrict__ keys, long long n, long long *__restrict__ flag) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

template <typename VT>
__device__ inline VT vzero();
template <>
__device__ inline double vzero<double>() { return 0.0; }
template <>
__device__ inline double2 vzero<double2>() { return make_double2(0.0, 0.0); }
__device__ inline double vadd(double a, double b) { return a + b; }
__device__ inline double2 vadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ inline bool vkeep(double a, double drop) { return drop < 0 || fabs(a) > drop; }
__device__ inline bool vkeep(double2 a, double drop) { return drop < 0 || fabs(a.x) > drop || fabs(a.y) > drop; }

template <typename VT>
__global__ void k_reduce(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ idx,
                         const VT *__restrict__ vals, long long n, const long long *__restrict__ pos,
                         uint64_t *__restrict__ uk, VT *__restrict__ uv) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t key = keys[i];
    if (i > 0 && keys[i - 1] == key) return;
    VT s = vzero<VT>();
    for (long long j = i; j < n && keys[j] == key; ++j) s = vadd(s, vals[idx[j]]);
    uk[pos[i]] = key;
    uv[pos[i]] = s;
}

template <typename VT>
__global__ void k_keep_flags(const VT *__restrict__ v, long long n, double drop, long long *__restrict__ flag) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = vkeep(v[i], drop) ? 1 : 0;
}

template <typename VT>
__global__ void k_compact(const uint64_t *__restrict__ uk, const VT *__restrict__ uv, long long n,
                          const long long *__restrict__ flag, const long long *__restrict__ pos,
                          uint64_t *__restrict__ ok, VT *__restrict__ ov) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flag[i]) {
        ok[pos[i]] = uk[i];
        ov[pos[i]] = uv[i];
    }
}

__global__ void k_rowptr(const uint64_t *__restrict__ keys, long long n, long long nrows, long long ncols,
                         int *__restrict__ rowptr) {
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r > nrows) return;
    uint64_t target = (uint64_t)r * (uint64_t)ncols;
    long long lo = 0, hi = n;
    while (lo < hi) {
        long long mid = (lo + hi) >> 1;
        if (keys[mid] < target) lo = mid + 1;
        else hi = mid;
    }
    rowptr[r] = (int)lo;
}

__global__ void k_cols(const uint64_t *__restrict__ keys, long long n, long long ncols, int *__restrict__ col) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) col[i] = (int)(keys[i] % (uint64_t)ncols);
}

template <typename VT, typename CSR>
void coo_to_csr_impl(DBuf<uint64_t> &keys, DBuf<VT> &vals, long long n, long long nrows, long long ncols,
                     double drop, CSR &out, cudaStream_t s) {
    out.rows = nrows;
    out.cols = ncols;
    GK_REQUIRE(n < (1LL << 31), GKSL_ERR_ARG, "sparse product too large for int32 indexing");
    if (n == 0) {
        out.nnz = 0;
        out.rowptr.alloc((size_t)nrows + 1);
        GK_CUDA(cudaMemsetAsync(out.rowptr.p, 0, sizeof(int) * (nrows + 1), s));
        out.col.alloc(1);
        out.val.alloc(1);
        GK_CUDA(cudaStreamSynchronize(s));
        return;
    }
    int kb = bits_for((unsigned long long)nrows * (unsigned long long)ncols);
    DBuf<uint32_t> idx((size_t)n);
    k_iota<<<grid_for(n, 256), 256, 0, s>>>(idx.p, n);
    GK_LAUNCH_CHECK();
    radix_sort(keys, idx, n, kb, s);
    DBuf<long long> flag((size_t)n), pos((size_t)n + 1);
    k_heads<<<grid_for(n, 256), 256, 0, s>>>(keys.p, n, flag.p);
    GK_LAUNCH_CHECK();
    long long nu = scan_ll(flag.p, pos.p, n, true, true, s);
    DBuf<uint64_t> uk((size_t)nu);
    DBuf<VT> uv((size_t)nu);
    k_reduce<VT><<<grid_for(n, 256), 256, 0, s>>>(keys.p, idx.p, vals.p, n, pos.p, uk.p, uv.p);
    GK_LAUNCH_CHECK();
    GK_CUDA(cudaStreamSynchronize(s));
    idx.release();
    flag.release();
    pos.release();
    long long nk = nu;
    DBuf<uint64_t> fk;
    DBuf<VT> fv;
    if (drop >= 0) {
        DBuf<long long> kf((size_t)nu), kp((size_t)nu + 1);
        k_keep_flags<VT><<<grid_for(nu, 256), 256, 0, s>>>(uv.p, nu, drop, kf.p);
        GK_LAUNCH_CHECK();
        nk = scan_ll(kf.p, kp.p, nu, true, true, s);
        fk.alloc((size_t)nk);
        fv.alloc((size_t)nk);
        k_compact<VT><<<grid_for(nu, 256), 256, 0, s>>>(uk.p, uv.p, nu, kf.p, kp.p, fk.p, fv.p);
        GK_LAUNCH_CHECK();
        GK_CUDA(cudaStreamSynchronize(s));
    } else {
        fk = std::move(uk);
        fv = std::move(uv);
    }
    out.nnz = nk;
    out.rowptr.alloc((size_t)nrows + 1);
    out.col.alloc((size_t)nk);
    k_rowptr<<<grid_for(nrows + 1, 256), 256, 0, s>>>(fk.p, nk, nrows, ncols, out.rowptr.p);
    GK_LAUNCH_CHECK();
    k_cols<<<grid_for(nk, 256), 256, 0, s>>>(fk.p, nk, ncols, out.col.p);
    GK_LAUNCH_CHECK();
    out.val = std::move(fv);
    GK_CUDA(cudaStreamSynchronize(s));
}

__global__ void k_max_abs(const double *__restrict__ v, long long n, unsigned long long *__restrict__ out) {
    double m = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m = fmax(m, fabs(v[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(kFull, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

}  // namespace

int bits_for(unsigned long long x) {
    int b = 0;
    while (b < 64 && (x >> b) != 0) ++b;
    return b < 1 ? 1 : b;
}

long long scan_ll(const long long *in, long long *out, long long n, bool with_total, bool want_total,
                  cudaStream_t s) {
    return scan_impl<long long>(in, out, n, with_total, want_total, s);
}

long long scan_u32_to_ll(const unsigned *in, long long *out, long long n, bool want_total, cudaStream_t s) {
    return scan_impl<unsigned>(in, out, n, true, want_total, s);
}

void radix_sort(DBuf<uint64_t> &keys, DBuf<uint32_t> &idx, long long n, int key_bits, cudaStream_t s) {
    if (n <= 1) return;
    long long ntiles = (n + kTile - 1) / kTile;
    DBuf<uint64_t> k2((size_t)n);
    DBuf<uint32_t> v2((size_t)n);
    DBuf<long long> hist((size_t)(kBins * ntiles)), offs((size_t)(kBins * ntiles) + 1);
    for (int shift = 0; shift < key_bits; shift += 8) {
        k_rs_hist<<<(unsigned)ntiles, kT, 0, s>>>(keys.p, n, shift, hist.p, ntiles);
        GK_LAUNCH_CHECK();
        scan_ll(hist.p, offs.p, kBins * ntiles, false, false, s);
        k_rs_scatter<<<(unsigned)ntiles, kT, 0, s>>>(keys.p, idx.p, k2.p, v2.p, n, shift, offs.p, ntiles);
        GK_LAUNCH_CHECK();
        std::swap(keys.p, k2.p);
        std::swap(keys.n, k2.n);
        std::swap(idx.p, v2.p);
        std::swap(idx.n, v2.n);
    }
    GK_CUDA(cudaStreamSynchronize(s));
}

void coo_to_csr_real(DBuf<uint64_t> &keys, DBuf<double> &vals, long long n, long long nrows, long long ncols,
                     double drop, CsrR &out, cudaStream_t s) {
    coo_to_csr_impl<double, CsrR>(keys, vals, n, nrows, ncols, drop, out, s);
}

void coo_to_csr_cplx(DBuf<uint64_t> &keys, DBuf<double2> &vals, long long n, long long nrows, long long ncols,
                     double drop, CsrC &out, cudaStream_t s) {
    coo_to_csr_impl<double2, CsrC>(keys, vals, n, nrows, ncols, drop, out, s);
}

double max_abs(const double *val, long long n, cudaStream_t s) {
    DBuf<unsigned long long> m(1);
    GK_CUDA(cudaMemsetAsync(m.p, 0, sizeof(unsigned long long), s));
    if (n > 0) {
        long long g = (n + 255) / 256;
        if (g > 4096) g = 4096;
        k_max_abs<<<(unsigned)g, 256, 0, s>>>(val, n, m.p);
        GK_LAUNCH_CHECK();
    }
    unsigned long long h = 0;
    GK_CUDA(cudaMemcpyAsync(&h, m.p, sizeof h, cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaStreamSynchronize(s));
    double r;
    memcpy(&r, &h, sizeof r);
    return r;
}

}  // namespace gk
