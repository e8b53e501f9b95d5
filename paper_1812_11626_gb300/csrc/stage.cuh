// RK4 stage epilogues shared by the CSR stage kernels (rk4.cu) and the matrix-free stage
// kernels (mfree.cu).  With k the stage derivative at row r:
//   stage 1: y2 = v + h/2 k1, acc = k1          stage 2: y3 = v + h/2 k2, acc += 2 k2
//   stage 3: y4 = v + h k3,   acc += 2 k3       stage 4: v += h/6 (acc + k4)
// The FP32 form adds the FP32 increment of stage 4 to an FP64 master state v64 and refreshes
// the FP32 mirror from it.
#pragma once

#include "common.cuh"

namespace gk {

template <int STAGE>
__device__ inline int eps_slot() { return STAGE == 1 ? 0 : (STAGE == 4 ? 2 : 1); }

// step-size constants, computed once on the host (no per-thread FP64 division)
struct HConst {
    double h, h2, h6;   // h, h/2, h/6
    float hf, h2f, h6f;
};

// ---- FP64 epilogue
template <int STAGE>
__device__ inline void epi64(long long r, double k, double *v, double *__restrict__ yn, double *__restrict__ acc,
                             const HConst &c) {
    if (STAGE == 1) { yn[r] = v[r] + c.h2 * k; acc[r] = k; }
    if (STAGE == 2) { yn[r] = v[r] + c.h2 * k; acc[r] = acc[r] + 2.0 * k; }
    if (STAGE == 3) { yn[r] = v[r] + c.h * k; acc[r] = acc[r] + 2.0 * k; }
    if (STAGE == 4) { v[r] = v[r] + c.h6 * (acc[r] + k); }
}

// ---- FP32 epilogue (v32: FP32 mirror, v64: master)
template <int STAGE>
__device__ inline void epi32(long long r, float k, float *v32, double *v64, float *__restrict__ yn,
                             float *__restrict__ acc, const HConst &c) {
    if (STAGE == 1) { yn[r] = v32[r] + c.h2f * k; acc[r] = k; }
    if (STAGE == 2) { yn[r] = v32[r] + c.h2f * k; acc[r] = acc[r] + 2.0f * k; }
    if (STAGE == 3) { yn[r] = v32[r] + c.hf * k; acc[r] = acc[r] + 2.0f * k; }
    if (STAGE == 4) {
        float inc = c.h6f * (acc[r] + k);
        double nv = v64[r] + (double)inc;
        v64[r] = nv;
        v32[r] = (float)nv;
    }
}

template <typename VT>
struct Vec2;
template <>
struct Vec2<double> { using T = double2; };
template <>
struct Vec2<float> { using T = float2; };

template <int STAGE, typename VT>
__device__ inline void epi(long long r, VT k, VT *v, double *v64, VT *__restrict__ yn, VT *__restrict__ acc,
                           const HConst &hc);
template <>
__device__ inline void epi<1, double>(long long r, double k, double *v, double *, double *yn, double *acc,
                                      const HConst &hc) { epi64<1>(r, k, v, yn, acc, hc); }
template <>
__device__ inline void epi<2, double>(long long r, double k, double *v, double *, double *yn, double *acc,
                                      const HConst &hc) { epi64<2>(r, k, v, yn, acc, hc); }
template <>
__device__ inline void epi<3, double>(long long r, double k, double *v, double *, double *yn, double *acc,
                                      const HConst &hc) { epi64<3>(r, k, v, yn, acc, hc); }
template <>
__device__ inline void epi<4, double>(long long r, double k, double *v, double *, double *yn, double *acc,
                                      const HConst &hc) { epi64<4>(r, k, v, yn, acc, hc); }
template <>
__device__ inline void epi<1, float>(long long r, float k, float *v, double *v64, float *yn, float *acc,
                                     const HConst &hc) { epi32<1>(r, k, v, v64, yn, acc, hc); }
template <>
__device__ inline void epi<2, float>(long long r, float k, float *v, double *v64, float *yn, float *acc,
                                     const HConst &hc) { epi32<2>(r, k, v, v64, yn, acc, hc); }
template <>
__device__ inline void epi<3, float>(long long r, float k, float *v, double *v64, float *yn, float *acc,
                                     const HConst &hc) { epi32<3>(r, k, v, v64, yn, acc, hc); }
template <>
__device__ inline void epi<4, float>(long long r, float k, float *v, double *v64, float *yn, float *acc,
                                     const HConst &hc) { epi32<4>(r, k, v, v64, yn, acc, hc); }

// Split form of the same updates for kernels that load every operand of a thread's rows first:
// epi_load gathers what the stage reads (v, acc; the FP64 master in stage 4 of the FP32 form),
// epi_store applies the update with the same arithmetic as epi64 / epi32.
template <typename VT>
struct EpIn {
    VT v = VT(0), acc = VT(0);
    double v64 = 0.0;
};

template <int STAGE, typename VT>
__device__ inline void epi_load(long long r, const VT *v, const double *v64, const VT *acc, EpIn<VT> &e) {
    constexpr bool F64 = sizeof(VT) == 8;
    if (STAGE != 4 || F64) e.v = v[r];
    if (STAGE >= 2) e.acc = acc[r];
    if (STAGE == 4 && !F64) e.v64 = v64[r];
}

template <int STAGE, typename VT>
__device__ inline void epi_store(long long r, VT k, const EpIn<VT> &e, VT *v, double *v64, VT *__restrict__ yn,
                                 VT *__restrict__ acc, const HConst &c) {
    if constexpr (sizeof(VT) == 8) {
        if (STAGE == 1) { yn[r] = e.v + c.h2 * k; acc[r] = k; }
        if (STAGE == 2) { yn[r] = e.v + c.h2 * k; acc[r] = e.acc + 2.0 * k; }
        if (STAGE == 3) { yn[r] = e.v + c.h * k; acc[r] = e.acc + 2.0 * k; }
        if (STAGE == 4) { v[r] = e.v + c.h6 * (e.acc + k); }
    } else {
        if (STAGE == 1) { yn[r] = e.v + c.h2f * k; acc[r] = k; }
        if (STAGE == 2) { yn[r] = e.v + c.h2f * k; acc[r] = e.acc + 2.0f * k; }
        if (STAGE == 3) { yn[r] = e.v + c.hf * k; acc[r] = e.acc + 2.0f * k; }
        if (STAGE == 4) {
            const float inc = c.h6f * (e.acc + k);
            const double nv = e.v64 + (double)inc;
            v64[r] = nv;
            v[r] = (float)nv;
        }
    }
}

}  // namespace gk
