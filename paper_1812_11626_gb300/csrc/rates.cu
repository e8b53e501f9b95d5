// Measured rates of the current GPU that bound the library's kernels where no driver-measured
// peak exists: the FP64 fused multiply-add rate (the co-limit of the FP64 stage kernels) and
// the read rate of data resident in L2 (the bound of the batched stage, whose state matrices
// live in L2).  Both kernels check their own results, so a rate is reported only for work
// that was actually done.
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace gk {
namespace {

constexpr int kChains = 8;

// Every thread runs kChains independent recurrences x <- fma(x, a, b) for `iters` steps from
// seeds that depend on the chain only, so every thread ends with the same kChains values; the
// first thread of each block stores them and every thread counts a disagreement with them.
__global__ void __launch_bounds__(256) k_fma_chains(long long iters, double a, double b, double *__restrict__ out,
                                                     unsigned long long *__restrict__ bad) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 0.125 * c;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    __shared__ double ref[kChains];
    if (threadIdx.x == 0)
        for (int c = 0; c < kChains; ++c) ref[c] = x[c];
    __syncthreads();
    int mism = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) mism += x[c] != ref[c];
    if (mism) atomicAdd(bad, (unsigned long long)mism);
    if (blockIdx.x == 0 && threadIdx.x == 0)
        for (int c = 0; c < kChains; ++c) out[c] = x[c];
}

// Sum of `reps` passes over an L2-resident buffer of n float4 (every component 1.0), read with
// ld.global.cg (cached in L2, not in L1).  Each thread keeps four independent loads in flight
// (elements i, i + S, i + 2S, i + 3S of a pass with grid stride S) and four float partial sums,
// which stay exact (small integers); the double total is exact as well.
__global__ void __launch_bounds__(256) k_l2_read(const float4 *__restrict__ buf, long long n, int reps,
                                                  double *__restrict__ total) {
    const long long S = (long long)gridDim.x * blockDim.x;
    const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double acc = 0.0;
    for (int r = 0; r < reps; ++r) {
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
        long long i = i0;
        for (; i + 3 * S < n; i += 4 * S) {
            const float4 a = __ldcg(buf + i), b = __ldcg(buf + i + S), c = __ldcg(buf + i + 2 * S),
                         d = __ldcg(buf + i + 3 * S);
            s0 += (a.x + a.y) + (a.z + a.w);
            s1 += (b.x + b.y) + (b.z + b.w);
            s2 += (c.x + c.y) + (c.z + c.w);
            s3 += (d.x + d.y) + (d.z + d.w);
        }
        for (; i < n; i += S) {
            const float4 a = __ldcg(buf + i);
            s0 += (a.x + a.y) + (a.z + a.w);
        }
        acc += (double)s0 + (double)s1 + (double)s2 + (double)s3;
    }
    atomicAdd(total, acc);
}

__global__ void k_fill_ones(float4 *buf, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) buf[i] = make_float4(1.0f, 1.0f, 1.0f, 1.0f);
}

}  // namespace
}  // namespace gk

using namespace gk;

extern "C" gksl_status gksl_measure_rates(int device, double *fp64_fma_per_s, double *l2_read_bytes_per_s) {
    if (!fp64_fma_per_s && !l2_read_bytes_per_s) return GKSL_ERR_ARG;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) {
        cudaGetLastError();
        return GKSL_ERR_CUDA;
    }
    struct Restore {
        int dev;
        ~Restore() { cudaSetDevice(dev); }
    } restore{prev};
    try {
        GK_CUDA(cudaSetDevice(device));
        int sms = 0;
        GK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
        cudaEvent_t e0, e1;
        GK_CUDA(cudaEventCreate(&e0));
        GK_CUDA(cudaEventCreate(&e1));
        if (fp64_fma_per_s) {
            const double a = 1.0 - std::ldexp(1.0, -20), b = std::ldexp(1.0, -21);
            const long long iters = 1LL << 16;
            const unsigned grid = (unsigned)sms * 4;
            DBuf<double> out(kChains);
            DBuf<unsigned long long> bad(1);
            GK_CUDA(cudaMemset(bad.p, 0, sizeof(unsigned long long)));
            k_fma_chains<<<grid, 256>>>(1024, a, b, out.p, bad.p);   // warm-up
            GK_LAUNCH_CHECK();
            GK_CUDA(cudaEventRecord(e0));
            k_fma_chains<<<grid, 256>>>(iters, a, b, out.p, bad.p);
            GK_LAUNCH_CHECK();
            GK_CUDA(cudaEventRecord(e1));
            GK_CUDA(cudaEventSynchronize(e1));
            float ms = 0.0f;
            GK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            double got[kChains];
            unsigned long long nbad = 0;
            GK_CUDA(cudaMemcpy(got, out.p, sizeof(got), cudaMemcpyDeviceToHost));
            GK_CUDA(cudaMemcpy(&nbad, bad.p, sizeof(nbad), cudaMemcpyDeviceToHost));
            // the same recurrence on the host: fma is correctly rounded on both sides
            bool ok = nbad == 0;
            for (int c = 0; c < kChains; ++c) {
                double x = 1.0 + 0.125 * c;
                for (long long i = 0; i < iters; ++i) x = std::fma(x, a, b);
                ok = ok && x == got[c];
            }
            if (!ok) throw Error{GKSL_ERR_STATE, "FP64 rate probe: results differ from the host recurrence"};
            *fp64_fma_per_s = (double)grid * 256.0 * (double)iters * kChains / (ms * 1e-3);
        }
        if (l2_read_bytes_per_s) {
            const long long n = (32LL << 20) / 16;   // 32 MiB, well inside the L2
            const int reps = 64;
            DBuf<float4> buf((size_t)n);
            DBuf<double> total(1);
            k_fill_ones<<<grid_for(n, 256), 256>>>(buf.p, n);
            GK_LAUNCH_CHECK();
            const unsigned grid = (unsigned)sms * 4;
            for (int pass = 0; pass < 2; ++pass) {   // the first pass warms the L2
                GK_CUDA(cudaMemset(total.p, 0, sizeof(double)));
                GK_CUDA(cudaEventRecord(e0));
                k_l2_read<<<grid, 256>>>(buf.p, n, reps, total.p);
                GK_LAUNCH_CHECK();
                GK_CUDA(cudaEventRecord(e1));
                GK_CUDA(cudaEventSynchronize(e1));
            }
            float ms = 0.0f;
            GK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            double got = 0.0;
            GK_CUDA(cudaMemcpy(&got, total.p, sizeof(double), cudaMemcpyDeviceToHost));
            if (got != 4.0 * (double)n * reps)
                throw Error{GKSL_ERR_STATE, "L2 rate probe: the sum of the buffer is wrong"};
            *l2_read_bytes_per_s = 16.0 * (double)n * reps / (ms * 1e-3);
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        GK_CUDA(cudaDeviceSynchronize());
        return GKSL_OK;
    } catch (const Error &e) {
        return e.st;
    }
}
