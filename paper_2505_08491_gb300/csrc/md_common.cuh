// Device-side helpers shared by the md kernels.
#pragma once
#include "md_internal.h"

// Precision-dependent views of an instance descriptor.
template <typename T> struct Pr;
template <> struct Pr<float> {
    __device__ static float st(const InstDesc& d, int c) { return d.st32[c]; }
    __device__ static const float* pi(const InstDesc& d) { return d.pi_v32; }
    __device__ static const float* psa(const InstDesc& d) { return d.psa32; }
    __device__ static const float* psb(const InstDesc& d) { return d.psb32; }
    __device__ static const float* tn(const InstDesc& d) { return d.tn_v32; }
    __device__ static const float* k1(const InstDesc& d) { return d.k1_v32; }
    __device__ static const float* pw(const InstDesc& d) { return d.pw_v32; }
    __device__ static float* t(const InstDesc& d) { return d.t32; }
    __device__ static const float* dinv(const InstDesc& d) { return d.dinv32; }
};
template <> struct Pr<double> {
    __device__ static double st(const InstDesc& d, int c) { return d.st64[c]; }
    __device__ static const double* pi(const InstDesc& d) { return d.pi_v64; }
    __device__ static const double* psa(const InstDesc& d) { return d.psa64; }
    __device__ static const double* psb(const InstDesc& d) { return d.psb64; }
    __device__ static const double* tn(const InstDesc& d) { return d.tn_v64; }
    __device__ static const double* k1(const InstDesc& d) { return d.k1_v64; }
    __device__ static const double* pw(const InstDesc& d) { return d.pw_v64; }
    __device__ static double* t(const InstDesc& d) { return d.t64; }
    __device__ static const double* dinv(const InstDesc& d) { return d.dinv64; }
};

// Block-wide sum of R values per thread (FP64), result valid in thread 0.
// `sh` must hold R * 32 doubles.
template <int R>
__device__ inline void block_sum(double (&v)[R], double* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        double x = v[r];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) sh[r * 32 + warp] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += sh[r * 32 + w];
            v[r] = s;
        }
    }
    __syncthreads();
}

// Runtime-count variant: v has `count` entries in shared memory per warp
// slot layout sh[r * 32 + warp]; sums `count` per-thread values given by f(r).
__device__ inline double warp_sum(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Last-block-done: every block of an instance writes its partials, then the
// last one to arrive (counted on `counter`) returns true and sees all
// partials.  The counter is reset by that block, so no clearing is needed
// between launches.
__device__ inline bool last_block_arrive(unsigned int* counter, int count) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int prev = atomicAdd(counter, 1u);
        last = (prev == (unsigned int)(count - 1));
        if (last) *counter = 0u;
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// GELU(x) = x Phi(x), Phi the standard normal CDF, branch-free.
// Phi(x) = 1/2 erfc(-x / sqrt 2) with erfc(z) = P(t) exp(-z^2), t = 1/(1 + p z)
// for z >= 0: the rational approximation 7.1.26 of Abramowitz & Stegun
// (|erf error| <= 1.5e-7).  For x < 0, Phi = 1/2 P(t) e^{-z^2} directly (no
// cancellation); for x >= 0, Phi = 1 - 1/2 P(t) e^{-z^2}.  So
// |GELU_here(x) - GELU(x)| <= 7.5e-8 |x| + FP32 rounding, far below the BF16
// resolution (2^-9 relative) the activations are stored in.
__device__ __forceinline__ float gelu_fast(float x) {
    const float z = fabsf(x) * 0.70710678118654752f;
    const float t = __frcp_rn(fmaf(0.3275911f, z, 1.0f));
    float poly = fmaf(1.061405429f, t, -1.453152027f);
    poly = fmaf(poly, t, 1.421413741f);
    poly = fmaf(poly, t, -0.284496736f);
    poly = fmaf(poly, t, 0.254829592f);
    poly *= t;
    const float h = 0.5f * poly * __expf(-z * z);
    const float phi = x < 0.0f ? h : 1.0f - h;
    return x * phi;
}

// GELU'(x) = Phi(x) + x phi(x), phi(x) = exp(-x^2/2) / sqrt(2 pi); Phi from
// the same rational approximation as gelu_fast (e^{-z^2} with z^2 = x^2/2 is
// also the Gaussian factor of phi).
__device__ __forceinline__ float gelu_grad_fast(float x) {
    const float z = fabsf(x) * 0.70710678118654752f;
    const float t = __frcp_rn(fmaf(0.3275911f, z, 1.0f));
    float poly = fmaf(1.061405429f, t, -1.453152027f);
    poly = fmaf(poly, t, 1.421413741f);
    poly = fmaf(poly, t, -0.284496736f);
    poly = fmaf(poly, t, 0.254829592f);
    poly *= t;
    const float e = __expf(-z * z);
    const float h = 0.5f * poly * e;
    const float cdf = x < 0.0f ? h : 1.0f - h;
    return cdf + x * (0.3989422804014327f * e);
}

__device__ inline unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
