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
// (|erf error| <= 1.5e-7).  With h = 1/2 P(t) e^{-z^2} (the 1/2 folded into
// the coefficients), Phi = h for x < 0 (no cancellation) and 1 - h for
// x >= 0, so GELU = x h or x - x h.  The reciprocal and 2^w are the PTX
// approximate instructions (rcp.approx, ex2.approx: a few ulp), so
// |GELU_here(x) - GELU(x)| <= ~1e-7 |x| + FP32 rounding, far below the BF16
// resolution (2^-9 relative) the activations are stored in.
namespace gelu_as {
constexpr float P = 0.3275911f;
constexpr float H1 = 0.5f * 0.254829592f, H2 = 0.5f * -0.284496736f, H3 = 0.5f * 1.421413741f,
                H4 = 0.5f * -1.453152027f, H5 = 0.5f * 1.061405429f;
constexpr float RSQRT2 = 0.70710678118654752f;
constexpr float NEG_LOG2E = -1.4426950408889634f;
}  // namespace gelu_as

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float ex2_approx(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float gelu_fast(float x) {
    using namespace gelu_as;
    const float z = fabsf(x) * RSQRT2;
    const float t = rcp_approx(fmaf(P, z, 1.0f));
    float poly = fmaf(H5, t, H4);
    poly = fmaf(poly, t, H3);
    poly = fmaf(poly, t, H2);
    poly = fmaf(poly, t, H1);
    poly = poly * t;
    const float e = ex2_approx(z * (z * NEG_LOG2E));
    const float xh = x * (poly * e);
    return x < 0.0f ? xh : x - xh;
}

// Two GELUs with the packed FP32 pair instructions of sm_100+ (fma/mul
// .rn.f32x2) for the arithmetic that is not per-lane: the same operations
// in the same order as gelu_fast, so the results are identical.
struct f32x2_t {
    unsigned long long v;
};
__device__ __forceinline__ f32x2_t pk2(float a, float b) {
    f32x2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(f32x2_t p, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(p.v));
}
__device__ __forceinline__ f32x2_t fma2(f32x2_t a, f32x2_t b, f32x2_t c) {
    f32x2_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}
__device__ __forceinline__ f32x2_t mul2(f32x2_t a, f32x2_t b) {
    f32x2_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}

__device__ __forceinline__ void gelu_fast2(float& x0, float& x1) {
    using namespace gelu_as;
    const f32x2_t Z = pk2(fabsf(x0) * RSQRT2, fabsf(x1) * RSQRT2);
    float d0, d1;
    upk2(fma2(pk2(P, P), Z, pk2(1.0f, 1.0f)), d0, d1);
    const f32x2_t T = pk2(rcp_approx(d0), rcp_approx(d1));
    f32x2_t poly = fma2(pk2(H5, H5), T, pk2(H4, H4));
    poly = fma2(poly, T, pk2(H3, H3));
    poly = fma2(poly, T, pk2(H2, H2));
    poly = fma2(poly, T, pk2(H1, H1));
    poly = mul2(poly, T);
    float w0, w1;
    upk2(mul2(Z, mul2(Z, pk2(NEG_LOG2E, NEG_LOG2E))), w0, w1);
    const f32x2_t E = pk2(ex2_approx(w0), ex2_approx(w1));
    float h0, h1;
    upk2(mul2(pk2(x0, x1), mul2(poly, E)), h0, h1);
    x0 = x0 < 0.0f ? h0 : x0 - h0;
    x1 = x1 < 0.0f ? h1 : x1 - h1;
}

// GELU'(x) = Phi(x) + x phi(x), phi(x) = exp(-x^2/2) / sqrt(2 pi); Phi from
// the same rational approximation as gelu_fast (e^{-z^2} with z^2 = x^2/2 is
// also the Gaussian factor of phi).
__device__ __forceinline__ float gelu_grad_fast(float x) {
    using namespace gelu_as;
    const float z = fabsf(x) * RSQRT2;
    const float t = rcp_approx(fmaf(P, z, 1.0f));
    float poly = fmaf(H5, t, H4);
    poly = fmaf(poly, t, H3);
    poly = fmaf(poly, t, H2);
    poly = fmaf(poly, t, H1);
    poly = poly * t;
    const float e = ex2_approx(z * (z * NEG_LOG2E));
    const float h = poly * e;
    const float cdf = x < 0.0f ? h : 1.0f - h;
    return cdf + x * (0.3989422804014327f * e);
}

__device__ inline unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Device timestamp of a point in a stream (or captured graph): the global
// nanosecond timer when the kernel runs, i.e. after everything before it on
// the stream has finished.  One per translation unit (internal linkage).
static __global__ void k_stamp(unsigned long long* at) { *at = globaltimer(); }
