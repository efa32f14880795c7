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

// One row of a CSR product, sum over jj in [j0, j1) of vals[jj] x[cols[jj]],
// added in row order.  The column indices of eight entries are loaded before
// any value they point to, so a row costs about two memory round trips per
// eight entries instead of two per entry (the gathers from x depend on the
// index loads).
template <typename T, typename V>
__device__ __forceinline__ T csr_row(const int* __restrict__ cols, const V* __restrict__ vals, int j0, int j1,
                                     const T* __restrict__ x) {
    T acc = T(0);
    for (int jb = j0; jb < j1; jb += 8) {
        int c[8];
        T v[8], xv[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const bool in = jb + k < j1;
            c[k] = in ? cols[jb + k] : 0;
            v[k] = in ? (T)vals[jb + k] : T(0);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) xv[k] = (jb + k < j1) ? x[c[k]] : T(0);
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (jb + k < j1) acc += v[k] * xv[k];
    }
    return acc;
}

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

// GELU(x) = x Phi(x), Phi the standard normal CDF, in the tanh form of
// Hendrycks & Gimpel (2016):
//     GELU(x) ~ x/2 (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))),
// within 4.8e-4 of x Phi(x) everywhere, with the hyperbolic tangent from the
// one-instruction tanh.approx.f32 (absolute error about 2^-11).  The
// network's activations are stored in BF16 (relative resolution 2^-9): an
// O(1) activation is rounded by up to ~4e-3, several times the error of this
// form, which is the cheapest branch-free one (3 multiply-adds and one
// special-function instruction per value).
namespace gelu_t {
constexpr float C0 = 0.7978845608028654f;              // sqrt(2/pi)
constexpr float C1 = 0.7978845608028654f * 0.044715f;  // sqrt(2/pi) * 0.044715
}  // namespace gelu_t

__device__ __forceinline__ float tanh_approx(float x) {
    float r;
    asm("tanh.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float gelu_fast(float x) {
    using namespace gelu_t;
    const float u = x * fmaf(C1, x * x, C0);
    const float h = 0.5f * x;
    return fmaf(h, tanh_approx(u), h);
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
    using namespace gelu_t;
    const f32x2_t X = pk2(x0, x1);
    const f32x2_t U = mul2(X, fma2(pk2(C1, C1), mul2(X, X), pk2(C0, C0)));
    float u0, u1;
    upk2(U, u0, u1);
    const f32x2_t H = mul2(pk2(0.5f, 0.5f), X);
    upk2(fma2(H, pk2(tanh_approx(u0), tanh_approx(u1)), H), x0, x1);
}

// GELU'(x) of the same form: with t = tanh(u), u = sqrt(2/pi)(x + 0.044715 x^3),
//     d/dx [x/2 (1 + t)] = (1 + t)/2 + x/2 (1 - t^2) sqrt(2/pi)(1 + 3 * 0.044715 x^2).
__device__ __forceinline__ float gelu_grad_fast(float x) {
    using namespace gelu_t;
    const float x2 = x * x;
    const float t = tanh_approx(x * fmaf(C1, x2, C0));
    const float du = fmaf(3.0f * C1, x2, C0);
    return fmaf(0.5f * x * du, fmaf(-t, t, 1.0f), 0.5f * (1.0f + t));
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
