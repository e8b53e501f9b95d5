// Allocation-free RK4 propagation entry point.
//
// gksl_propagate keeps its RK4 work vectors in device memory it allocates per context.  Some
// callers cannot let a library allocate: services that hand all device memory to their own
// pool up front (so a cudaMalloc would fail or fragment the pool), and loops that must not
// stall the whole device (cudaMalloc and cudaFree can synchronise the GPU).  This entry point
// takes the matrices, K and the state from the caller and keeps its three work vectors in one
// fixed array compiled into the library, so it calls no allocator at all.
//
// The array is a file-scope __device__ variable: every GPU that loads the library holds it
// (3 x GKSL_NOALLOC_MAX_D doubles, 6 MiB) until the process exits, and every call on that GPU
// shares it.  Host code cannot use the array's name as a device address, so the first call on
// each device looks the address up with cudaGetSymbolAddress (with that device current) and
// keeps it for the life of the process; that first call should therefore happen before any
// stream capture.  After cudaDeviceReset the kept address no longer names the array, so this
// entry point must not be called again on a device that has been reset.  Calls whose kernels
// overlap on the GPU (two streams, or two host threads) race on the array.  Nothing in the array
// needs to start at zero: every element a stage reads was written earlier in the same step.
//
// Errors: a CUDA error already pending when the call starts (left by other work) is reported as
// GKSL_ERR_CUDA without launching anything and is left for its owner to read; a failed launch of
// this call is cleared and reported as GKSL_ERR_CUDA.
#include <cmath>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/gksl.h"

namespace {

constexpr long long kMaxD = GKSL_NOALLOC_MAX_D;
constexpr int kMaxDevices = 64;
constexpr int kThreads = 256;

// y_a, y_b and acc of the RK4 stages, back to back
static __device__ __align__(256) double g_rk4_work[3 * kMaxD];

std::mutex g_mu;
double *g_work_addr[kMaxDevices] = {};

struct Csr {
    const int *rowptr;
    const int *col;
    const double *val;
};

// One RK4 stage of v' = (A0 + eps A1) v + K, one thread per row (the CSR counterpart of the
// hybrid-format stage kernel): k = A0 y + eps A1 y + K, then the stage's update of
// y_next / acc / v.
template <int STAGE>
__global__ void __launch_bounds__(kThreads) k_stage_csr(long long D, Csr a0, Csr a1, const double *__restrict__ K,
                                                        double eps, const double *__restrict__ y, double *v,
                                                        double *__restrict__ yn, double *__restrict__ acc, double h,
                                                        double h2, double h6) {
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= D) return;
    double s0 = 0.0, s1 = 0.0;
    for (int e = a0.rowptr[r]; e < a0.rowptr[r + 1]; ++e) s0 += a0.val[e] * y[a0.col[e]];
    if (a1.rowptr)
        for (int e = a1.rowptr[r]; e < a1.rowptr[r + 1]; ++e) s1 += a1.val[e] * y[a1.col[e]];
    double k = s0 + eps * s1 + (K ? K[r] : 0.0);
    if (STAGE == 1) { yn[r] = v[r] + h2 * k; acc[r] = k; }
    if (STAGE == 2) { yn[r] = v[r] + h2 * k; acc[r] = acc[r] + 2.0 * k; }
    if (STAGE == 3) { yn[r] = v[r] + h * k; acc[r] = acc[r] + 2.0 * k; }
    if (STAGE == 4) { v[r] = v[r] + h6 * (acc[r] + k); }
}

// Device address of the work array on the current device, looked up once per device.  Called
// with no error pending, so an error raised here is this call's own and is cleared.
gksl_status work_address(double **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return GKSL_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return GKSL_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_work_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_rk4_work) != cudaSuccess || !p) {
            cudaGetLastError();
            return GKSL_ERR_CUDA;
        }
        g_work_addr[dev] = static_cast<double *>(p);
    }
    *out = g_work_addr[dev];
    return GKSL_OK;
}

}  // namespace

extern "C" gksl_status gksl_propagate_csr_noalloc(long long D, const int *a0_rowptr, const int *a0_col,
                                                  const double *a0_val, const int *a1_rowptr, const int *a1_col,
                                                  const double *a1_val, const double *K, double *v, double t0,
                                                  double h, long long n_steps, double E, double A, double omega,
                                                  void *cuda_stream) {
    if (D < 1 || D > kMaxD) return GKSL_ERR_ARG;   // larger systems do not fit the fixed work array
    if (!a0_rowptr || !a0_col || !a0_val || !v || n_steps < 0 || !(h > 0.0)) return GKSL_ERR_ARG;
    if (a1_rowptr && (!a1_col || !a1_val)) return GKSL_ERR_ARG;
    if (cudaPeekAtLastError() != cudaSuccess) return GKSL_ERR_CUDA;   // not ours: leave it pending
    double *work = nullptr;
    gksl_status st = work_address(&work);
    if (st != GKSL_OK) return st;
    double *ya = work, *yb = work + kMaxD, *acc = work + 2 * kMaxD;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    Csr m0{a0_rowptr, a0_col, a0_val}, m1{a1_rowptr, a1_col, a1_val};
    const double h2 = 0.5 * h, h6 = h / 6.0;
    const unsigned grid = (unsigned)((D + kThreads - 1) / kThreads);
    for (long long n = 0; n < n_steps; ++n) {
        const double tn = t0 + (double)n * h;
        const double e1 = E + A * std::sin(omega * tn);
        const double e2 = E + A * std::sin(omega * (tn + 0.5 * h));
        const double e4 = E + A * std::sin(omega * (tn + h));
        k_stage_csr<1><<<grid, kThreads, 0, s>>>(D, m0, m1, K, e1, v, v, ya, acc, h, h2, h6);
        if (cudaGetLastError() != cudaSuccess) return GKSL_ERR_CUDA;
        k_stage_csr<2><<<grid, kThreads, 0, s>>>(D, m0, m1, K, e2, ya, v, yb, acc, h, h2, h6);
        if (cudaGetLastError() != cudaSuccess) return GKSL_ERR_CUDA;
        k_stage_csr<3><<<grid, kThreads, 0, s>>>(D, m0, m1, K, e2, yb, v, ya, acc, h, h2, h6);
        if (cudaGetLastError() != cudaSuccess) return GKSL_ERR_CUDA;
        k_stage_csr<4><<<grid, kThreads, 0, s>>>(D, m0, m1, K, e4, ya, v, nullptr, acc, h, h2, h6);
        if (cudaGetLastError() != cudaSuccess) return GKSL_ERR_CUDA;
    }
    return GKSL_OK;
}
