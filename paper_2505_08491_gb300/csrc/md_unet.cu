// The paper's three-level U-net U3 (Section 4.2; the U3 table of Section 5.1)
// on CUDA cores, batched: `batch` grids of n^3 nodes per call.
//
//   e0 = GELU(conv3(X; 2 -> 32))                           n^3    skip 0
//   e1 = GELU(conv3(maxpool2(e0); 32 -> 64))               m1^3   skip 1   (m1 = n / 2)
//   e2 = GELU(conv3(maxpool2(e1); 64 -> 128))              m2^3            (m2 = m1 / 2)
//   b  = GELU(conv3(e2; 128 -> 128))                       m2^3
//   d1 = GELU(conv3([up2(b; 128 -> 64) | e1]; 128 -> 64))  m1^3
//   d0 = GELU(conv3([up2(d1; 64 -> 32) | e0]; 64 -> 32))   n^3
//   Y  = conv3(d0; 32 -> 1)                                n^3
//
// conv3: 3x3x3 with zero 'same' padding and bias; maxpool2: 2x2x2 windows at
// even offsets (an odd size's last plane dropped); up2: transposed 2x2x2
// convolution with stride 2, zero planes appended up to the skip's size; the
// channel stacking [up | skip] is a shared buffer that up2 writes in its
// first channels and the encoder layer in its last.  GELU is x Phi(x) with
// erff.  FP32 storage and arithmetic, layout (sample, channel, z, y, x).
//
// Parameter vector: the seven conv3 layers in the order above, then the two
// up2 layers, each its weights (conv3: c_out, c_in, 3, 3, 3; up2: c_in, c_out,
// 2, 2, 2) then its biases.
#include <cmath>
#include <cstring>
#include <vector>

#include "md_common.cuh"
#include "md_internal.h"

namespace {

constexpr int UN_CONVS = 7, UN_UPS = 2;
constexpr int kConv[UN_CONVS][2] = {{2, 32}, {32, 64}, {64, 128}, {128, 128}, {128, 64}, {64, 32}, {32, 1}};
constexpr int kUp[UN_UPS][2] = {{128, 64}, {64, 32}};
constexpr int UN_TB = 128;   // threads per block
constexpr int UN_CO = 16;    // output channels per conv thread
constexpr int UN_CI = 8;     // input channels per shared-memory weight chunk

long long un_nparams() {
    long long n = 0;
    for (auto& c : kConv) n += 27LL * c[0] * c[1] + c[1];
    for (auto& u : kUp) n += 8LL * u[0] * u[1] + u[1];
    return n;
}

__device__ __forceinline__ float gelu_exact(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }

// A tensor view: channel c of sample b starts at p + (b * ctot + c0 + c) * vol.
struct View {
    float* p;
    int ctot, c0;
};

// conv3: one thread per output node, UN_CO output channels in registers; the
// weights of UN_CI input channels x 27 taps x UN_CO outputs staged in shared
// memory per step.  grid (node blocks, output-channel blocks, samples).
__global__ void __launch_bounds__(UN_TB) k_un_conv3(View in, int cin, View out, int cout, int n,
                                                    const float* __restrict__ W, const float* __restrict__ bias,
                                                    int act, View zsave) {
    __shared__ float sw[UN_CI * 27 * UN_CO];
    const long long vol = (long long)n * n * n;
    const int b = blockIdx.z, co0 = blockIdx.y * UN_CO;
    const long long node = (long long)blockIdx.x * UN_TB + threadIdx.x;
    const bool live = node < vol;
    const int x = live ? (int)(node % n) : 0;
    const int y = live ? (int)((node / n) % n) : 0;
    const int z = live ? (int)(node / ((long long)n * n)) : 0;
    const float* xin = in.p + ((long long)b * in.ctot + in.c0) * vol;
    float acc[UN_CO];
#pragma unroll
    for (int k = 0; k < UN_CO; ++k) acc[k] = 0.0f;
    for (int ci0 = 0; ci0 < cin; ci0 += UN_CI) {
        __syncthreads();
        for (int e = threadIdx.x; e < UN_CI * 27 * UN_CO; e += UN_TB) {
            const int k = e % UN_CO, t = (e / UN_CO) % 27, cl = e / (UN_CO * 27);
            const int co = co0 + k, ci = ci0 + cl;
            sw[e] = (co < cout && ci < cin) ? W[((long long)co * cin + ci) * 27 + t] : 0.0f;
        }
        __syncthreads();
        if (!live) continue;
        for (int cl = 0; cl < UN_CI && ci0 + cl < cin; ++cl) {
            const float* xc = xin + (long long)(ci0 + cl) * vol;
#pragma unroll
            for (int t = 0; t < 27; ++t) {
                const int zz = z + t / 9 - 1, yy = y + (t / 3) % 3 - 1, xx = x + t % 3 - 1;
                const bool ok = zz >= 0 && zz < n && yy >= 0 && yy < n && xx >= 0 && xx < n;
                const float v = ok ? xc[((long long)zz * n + yy) * n + xx] : 0.0f;
                const float* wr = sw + (cl * 27 + t) * UN_CO;
#pragma unroll
                for (int k = 0; k < UN_CO; ++k) acc[k] = fmaf(wr[k], v, acc[k]);
            }
        }
    }
    if (!live) return;
    float* yo = out.p + ((long long)b * out.ctot + out.c0) * vol + node;
#pragma unroll
    for (int k = 0; k < UN_CO; ++k) {
        const int co = co0 + k;
        if (co < cout) {
            const float v = acc[k] + (bias ? bias[co] : 0.0f);
            yo[(long long)co * vol] = act ? gelu_exact(v) : v;
            if (zsave.p) zsave.p[((long long)b * zsave.ctot + zsave.c0 + co) * vol + node] = v;
        }
    }
}

// maxpool2: one thread per output element (sample, channel, node of m^3).
__global__ void k_un_pool(View in, int c, int n, View out, int m, int batch) {
    const long long mv = (long long)m * m * m, nv = (long long)n * n * n;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= mv * c * batch) return;
    const long long node = e % mv;
    const int ch = (int)((e / mv) % c), b = (int)(e / (mv * c));
    const int x = (int)(node % m), y = (int)((node / m) % m), z = (int)(node / ((long long)m * m));
    const float* src = in.p + ((long long)b * in.ctot + in.c0 + ch) * nv;
    float best = -INFINITY;
    for (int t = 0; t < 8; ++t) {
        const long long q = ((long long)(2 * z + (t >> 2)) * n + (2 * y + ((t >> 1) & 1))) * n + (2 * x + (t & 1));
        best = fmaxf(best, src[q]);
    }
    out.p[((long long)b * out.ctot + out.c0 + ch) * mv + node] = best;
}

// up2: one thread per output node of n^3 (n in {2m, 2m + 1}), UN_CO output
// channels; nodes beyond 2m are the appended zero planes.
__global__ void __launch_bounds__(UN_TB) k_un_up2(View in, int cin, int m, View out, int cout, int n,
                                                  const float* __restrict__ W, const float* __restrict__ bias) {
    const long long nv = (long long)n * n * n, mv = (long long)m * m * m;
    const int b = blockIdx.z, co0 = blockIdx.y * UN_CO;
    const long long node = (long long)blockIdx.x * UN_TB + threadIdx.x;
    if (node >= nv) return;
    const int x = (int)(node % n), y = (int)((node / n) % n), z = (int)(node / ((long long)n * n));
    float* yo = out.p + ((long long)b * out.ctot + out.c0) * nv + node;
    if (x >= 2 * m || y >= 2 * m || z >= 2 * m) {
#pragma unroll
        for (int k = 0; k < UN_CO; ++k)
            if (co0 + k < cout) yo[(long long)(co0 + k) * nv] = 0.0f;
        return;
    }
    const int t = ((z & 1) << 2) | ((y & 1) << 1) | (x & 1);
    const long long p = ((long long)(z >> 1) * m + (y >> 1)) * m + (x >> 1);
    const float* xin = in.p + ((long long)b * in.ctot + in.c0) * mv + p;
    float acc[UN_CO];
#pragma unroll
    for (int k = 0; k < UN_CO; ++k) acc[k] = 0.0f;
    for (int ci = 0; ci < cin; ++ci) {
        const float v = xin[(long long)ci * mv];
        const float* wr = W + ((long long)ci * cout + co0) * 8 + t;
#pragma unroll
        for (int k = 0; k < UN_CO; ++k)
            if (co0 + k < cout) acc[k] = fmaf(wr[k * 8], v, acc[k]);
    }
#pragma unroll
    for (int k = 0; k < UN_CO; ++k)
        if (co0 + k < cout) yo[(long long)(co0 + k) * nv] = acc[k] + bias[co0 + k];
}

// ---- backward ----

// Input-gradient weights of a conv3 layer: the adjoint of conv3 is conv3 with
// the kernel transposed in (c_out, c_in) and flipped in space,
// Wt[ci][co][26 - t] = W[co][ci][t].
__global__ void k_un_flip(const float* __restrict__ W, int cout, int cin, float* __restrict__ Wt) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 27LL * cout * cin) return;
    const int t = (int)(e % 27), ci = (int)((e / 27) % cin), co = (int)(e / (27LL * cin));
    Wt[((long long)ci * cout + co) * 27 + (26 - t)] = W[e];
}

// g *= GELU'(z) = Phi(z) + z phi(z) over `c` channels of every sample.
__global__ void k_un_gelu_back(View g, View z, int c, long long vol, int batch) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= vol * c * batch) return;
    const long long node = e % vol;
    const int ch = (int)((e / vol) % c), b = (int)(e / (vol * c));
    const float zz = z.p[((long long)b * z.ctot + z.c0 + ch) * vol + node];
    const float d = 0.5f * (1.0f + erff(zz * 0.70710678118654752f)) + zz * 0.39894228040143268f * expf(-0.5f * zz * zz);
    g.p[((long long)b * g.ctot + g.c0 + ch) * vol + node] *= d;
}

// Weight gradient of conv3: dW[co][ci][t] += sum_{b, p} dZ[b][co][p] X[b][ci][p + q_t]
// and, from the blocks of ci = 0, db[co] += sum dZ[b][co][p].  A block takes 4
// output channels of one input channel over its share of the (sample, node)
// pairs; its sums are added to dW with atomics (dW, db zeroed before).
constexpr int UN_WCO = 4;
__global__ void __launch_bounds__(UN_TB) k_un_wgrad(View dz, int cout, View x, int cin, int n, int batch,
                                                    float* __restrict__ dW, float* __restrict__ db) {
    const long long vol = (long long)n * n * n, total = vol * batch;
    const int co0 = blockIdx.x * UN_WCO, ci = blockIdx.y;
    const long long per = (total + gridDim.z - 1) / gridDim.z;
    const long long e0 = (long long)blockIdx.z * per, e1 = e0 + per < total ? e0 + per : total;
    float acc[UN_WCO][27], bsum[UN_WCO];
#pragma unroll
    for (int k = 0; k < UN_WCO; ++k) {
        bsum[k] = 0.0f;
#pragma unroll
        for (int t = 0; t < 27; ++t) acc[k][t] = 0.0f;
    }
    for (long long e = e0 + threadIdx.x; e < e1; e += UN_TB) {
        const long long node = e % vol;
        const int b = (int)(e / vol);
        const int xx = (int)(node % n), yy = (int)((node / n) % n), zz = (int)(node / ((long long)n * n));
        float g[UN_WCO];
#pragma unroll
        for (int k = 0; k < UN_WCO; ++k)
            g[k] = co0 + k < cout ? dz.p[((long long)b * dz.ctot + dz.c0 + co0 + k) * vol + node] : 0.0f;
        const float* xc = x.p + ((long long)b * x.ctot + x.c0 + ci) * vol;
#pragma unroll
        for (int t = 0; t < 27; ++t) {
            const int z2 = zz + t / 9 - 1, y2 = yy + (t / 3) % 3 - 1, x2 = xx + t % 3 - 1;
            const bool ok = z2 >= 0 && z2 < n && y2 >= 0 && y2 < n && x2 >= 0 && x2 < n;
            const float v = ok ? xc[((long long)z2 * n + y2) * n + x2] : 0.0f;
#pragma unroll
            for (int k = 0; k < UN_WCO; ++k) acc[k][t] = fmaf(g[k], v, acc[k][t]);
        }
#pragma unroll
        for (int k = 0; k < UN_WCO; ++k) bsum[k] += g[k];
    }
    __shared__ float red[UN_TB / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < UN_WCO; ++k) {
#pragma unroll
        for (int t = 0; t <= 27; ++t) {
            float v = t < 27 ? acc[k][t] : bsum[k];
            for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp] = v;
            __syncthreads();
            if (threadIdx.x == 0 && co0 + k < cout) {
                float sum = 0.0f;
                for (int w = 0; w < UN_TB / 32; ++w) sum += red[w];
                if (t < 27) atomicAdd(&dW[((long long)(co0 + k) * cin + ci) * 27 + t], sum);
                else if (ci == 0) atomicAdd(&db[co0 + k], sum);
            }
            __syncthreads();
        }
    }
}

// up2 input gradient: dX[b][ci][p] = sum_{co, t} W[ci][co][t] dO[b][co][2p + t]
// (the appended planes carry no gradient).  One thread per input node,
// UN_CO input channels.
__global__ void __launch_bounds__(UN_TB) k_un_up2_dgrad(View dO, int cout, int n, View dX, int cin, int m,
                                                        const float* __restrict__ W) {
    const long long nv = (long long)n * n * n, mv = (long long)m * m * m;
    const int b = blockIdx.z, ci0 = blockIdx.y * UN_CO;
    const long long node = (long long)blockIdx.x * UN_TB + threadIdx.x;
    if (node >= mv) return;
    const int x = (int)(node % m), y = (int)((node / m) % m), z = (int)(node / ((long long)m * m));
    const float* g = dO.p + ((long long)b * dO.ctot + dO.c0) * nv;
    float acc[UN_CO];
#pragma unroll
    for (int k = 0; k < UN_CO; ++k) acc[k] = 0.0f;
    for (int co = 0; co < cout; ++co) {
        const float* gc = g + (long long)co * nv;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const float v = gc[((long long)(2 * z + (t >> 2)) * n + (2 * y + ((t >> 1) & 1))) * n + (2 * x + (t & 1))];
#pragma unroll
            for (int k = 0; k < UN_CO; ++k)
                if (ci0 + k < cin) acc[k] = fmaf(W[((long long)(ci0 + k) * cout + co) * 8 + t], v, acc[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < UN_CO; ++k)
        if (ci0 + k < cin) dX.p[((long long)b * dX.ctot + dX.c0 + ci0 + k) * mv + node] = acc[k];
}

// up2 weight gradient: dW[ci][co][t] += sum_{b, p} X[b][ci][p] dO[b][co][2p + t];
// the blocks of ci = 0 also add db[co] += sum over the non-appended outputs.
// A block takes 4 output channels of one input channel over its share of the
// (sample, input node) pairs; atomics into zeroed dW, db.
__global__ void __launch_bounds__(UN_TB) k_un_up2_wgrad(View dO, int cout, int n, View x, int cin, int m, int batch,
                                                        float* __restrict__ dW, float* __restrict__ db) {
    const long long nv = (long long)n * n * n, mv = (long long)m * m * m, total = mv * batch;
    const int co0 = blockIdx.x * UN_WCO, ci = blockIdx.y;
    const long long per = (total + gridDim.z - 1) / gridDim.z;
    const long long e0 = (long long)blockIdx.z * per, e1 = e0 + per < total ? e0 + per : total;
    float acc[UN_WCO][8], bsum[UN_WCO];
#pragma unroll
    for (int k = 0; k < UN_WCO; ++k) {
        bsum[k] = 0.0f;
#pragma unroll
        for (int t = 0; t < 8; ++t) acc[k][t] = 0.0f;
    }
    for (long long e = e0 + threadIdx.x; e < e1; e += UN_TB) {
        const long long node = e % mv;
        const int b = (int)(e / mv);
        const int xx = (int)(node % m), yy = (int)((node / m) % m), zz = (int)(node / ((long long)m * m));
        const float v = x.p[((long long)b * x.ctot + x.c0 + ci) * mv + node];
#pragma unroll
        for (int k = 0; k < UN_WCO; ++k) {
            if (co0 + k >= cout) continue;
            const float* gc = dO.p + ((long long)b * dO.ctot + dO.c0 + co0 + k) * nv;
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const float g = gc[((long long)(2 * zz + (t >> 2)) * n + (2 * yy + ((t >> 1) & 1))) * n + (2 * xx + (t & 1))];
                acc[k][t] = fmaf(v, g, acc[k][t]);
                bsum[k] += g;
            }
        }
    }
    __shared__ float red[UN_TB / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < UN_WCO; ++k) {
#pragma unroll
        for (int t = 0; t <= 8; ++t) {
            float v = t < 8 ? acc[k][t] : bsum[k];
            for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp] = v;
            __syncthreads();
            if (threadIdx.x == 0 && co0 + k < cout) {
                float sum = 0.0f;
                for (int w = 0; w < UN_TB / 32; ++w) sum += red[w];
                if (t < 8) atomicAdd(&dW[((long long)ci * cout + co0 + k) * 8 + t], sum);
                else if (ci == 0) atomicAdd(&db[co0 + k], sum);
            }
            __syncthreads();
        }
    }
}

// maxpool2 backward: the gradient of each output goes to its window's
// maximum, the first in (z, y, x) order among equal ones; added to dX, whose
// windows do not overlap.
__global__ void k_un_pool_back(View dO, View x, int c, int n, View dX, int m, int batch) {
    const long long mv = (long long)m * m * m, nv = (long long)n * n * n;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= mv * c * batch) return;
    const long long node = e % mv;
    const int ch = (int)((e / mv) % c), b = (int)(e / (mv * c));
    const int xo = (int)(node % m), yo = (int)((node / m) % m), zo = (int)(node / ((long long)m * m));
    const float* src = x.p + ((long long)b * x.ctot + x.c0 + ch) * nv;
    long long arg = 0;
    float best = -INFINITY;
    for (int t = 0; t < 8; ++t) {
        const long long q = ((long long)(2 * zo + (t >> 2)) * n + (2 * yo + ((t >> 1) & 1))) * n + (2 * xo + (t & 1));
        if (src[q] > best || t == 0) { best = src[q]; arg = q; }
    }
    dX.p[((long long)b * dX.ctot + dX.c0 + ch) * nv + arg] += dO.p[((long long)b * dO.ctot + dO.c0 + ch) * mv + node];
}

unsigned int blocks(long long n, int per) { return (unsigned int)((n + per - 1) / per); }

// blocks along the (sample, node) pairs of a weight-gradient launch: enough
// for ~4 waves of 152 SMs, each block at least 2,048 pairs
unsigned int wsplit(long long pairs, long long other_blocks) {
    long long want = (608 + other_blocks - 1) / other_blocks;
    const long long cap = (pairs + 2047) / 2048;
    if (want > cap) want = cap;
    return (unsigned int)(want < 1 ? 1 : want);
}

}  // namespace

struct md_unet {
    float* params = nullptr;  // device copy of the flat parameter vector
    long long nparams = 0;
    const float* Wc[UN_CONVS] = {};
    const float* Bc[UN_CONVS] = {};
    const float* Wu[UN_UPS] = {};
    const float* Bu[UN_UPS] = {};
    float* wt = nullptr;      // input-gradient weights of the conv3 layers (k_un_flip)
    float* Wt[UN_CONVS] = {};
    bool wt_ok = false;       // wt matches params
    float* ws = nullptr;      // workspace for the largest (n, batch, training) shape so far
    size_t ws_floats = 0;
    // AdamW state (md_unet_opt_step), allocated at the first step
    float *m = nullptr, *v = nullptr;
    unsigned char* is_weight = nullptr;
    long long step = 0;
};

extern "C" long long md_unet_num_params(void) { return un_nparams(); }

extern "C" md_status md_unet_create(const float* host_params, long long n_params, md_unet** out) {
    if (!out || !host_params) { md_set_error("md_unet_create: NULL argument"); return MD_ERR_ARG; }
    *out = nullptr;
    if (n_params != un_nparams()) {
        md_set_error("md_unet_create: %lld parameters, expected %lld", n_params, un_nparams());
        return MD_ERR_ARG;
    }
    md_unet* u = new md_unet();
    u->nparams = n_params;
    long long nw = 0;
    for (auto& c : kConv) nw += 27LL * c[0] * c[1];
    if (cudaMalloc(&u->params, sizeof(float) * (size_t)n_params) != cudaSuccess ||
        cudaMalloc(&u->wt, sizeof(float) * (size_t)nw) != cudaSuccess) {
        cudaFree(u->params); cudaFree(u->wt); delete u;
        md_set_error("md_unet_create: cudaMalloc failed"); return MD_ERR_OOM;
    }
    cudaError_t e = cudaMemcpy(u->params, host_params, sizeof(float) * (size_t)n_params, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(u->params); cudaFree(u->wt); delete u;
        return md_cuda_status(e, "md_unet_create", __FILE__, __LINE__);
    }
    long long k = 0, kt = 0;
    for (int l = 0; l < UN_CONVS; ++l) {
        u->Wc[l] = u->params + k; k += 27LL * kConv[l][0] * kConv[l][1];
        u->Bc[l] = u->params + k; k += kConv[l][1];
        u->Wt[l] = u->wt + kt; kt += 27LL * kConv[l][0] * kConv[l][1];
    }
    for (int l = 0; l < UN_UPS; ++l) {
        u->Wu[l] = u->params + k; k += 8LL * kUp[l][0] * kUp[l][1];
        u->Bu[l] = u->params + k; k += kUp[l][1];
    }
    *out = u;
    return MD_OK;
}

extern "C" md_status md_unet_set_params(md_unet* u, const float* params, int on_device, md_stream stream) {
    if (!u || !params) { md_set_error("md_unet_set_params: NULL argument"); return MD_ERR_ARG; }
    MD_CUDA(cudaMemcpyAsync(u->params, params, sizeof(float) * (size_t)u->nparams,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, (cudaStream_t)stream));
    u->wt_ok = false;
    return MD_OK;
}

extern "C" md_status md_unet_get_params(const md_unet* u, float* host_params, long long n_params) {
    if (!u || !host_params || n_params != u->nparams) { md_set_error("md_unet_get_params: bad argument"); return MD_ERR_ARG; }
    MD_CUDA(cudaMemcpy(host_params, u->params, sizeof(float) * (size_t)n_params, cudaMemcpyDeviceToHost));
    return MD_OK;
}

extern "C" void md_unet_destroy(md_unet* u) {
    if (!u) return;
    cudaFree(u->params);
    cudaFree(u->wt);
    cudaFree(u->ws);
    cudaFree(u->m);
    cudaFree(u->v);
    cudaFree(u->is_weight);
    delete u;
}

namespace {
// AdamW with decoupled weight decay on the weights (not the biases)
__global__ void k_un_adamw(float* w, const float* __restrict__ g, float* m, float* v, const unsigned char* is_weight,
                           long long n, float lr, float b1, float b2, float eps, float wd, float bc1, float bc2) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        float wi = w[i];
        if (is_weight[i]) wi -= lr * wd * wi;
        w[i] = wi - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
}
}  // namespace

extern "C" md_status md_unet_opt_step(md_unet* u, const float* grad, double lr, double beta1, double beta2, double eps,
                                      double weight_decay, md_stream stream) {
    if (!u || !grad) { md_set_error("md_unet_opt_step: NULL argument"); return MD_ERR_ARG; }
    if (!(lr >= 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0)) {
        md_set_error("md_unet_opt_step: bad hyper-parameters");
        return MD_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)u->nparams;
    if (!u->m) {
        std::vector<unsigned char> isw(n, 0);
        for (int l = 0; l < UN_CONVS; ++l) memset(isw.data() + (u->Wc[l] - u->params), 1, 27ULL * kConv[l][0] * kConv[l][1]);
        for (int l = 0; l < UN_UPS; ++l) memset(isw.data() + (u->Wu[l] - u->params), 1, 8ULL * kUp[l][0] * kUp[l][1]);
        if (cudaMalloc(&u->m, sizeof(float) * n) != cudaSuccess || cudaMalloc(&u->v, sizeof(float) * n) != cudaSuccess ||
            cudaMalloc(&u->is_weight, n) != cudaSuccess) {
            md_set_error("md_unet_opt_step: cudaMalloc failed");
            return MD_ERR_OOM;
        }
        MD_CUDA(cudaMemsetAsync(u->m, 0, sizeof(float) * n, s));
        MD_CUDA(cudaMemsetAsync(u->v, 0, sizeof(float) * n, s));
        MD_CUDA(cudaMemcpyAsync(u->is_weight, isw.data(), n, cudaMemcpyHostToDevice, s));
        MD_CUDA(cudaStreamSynchronize(s));
    }
    u->step += 1;
    const float bc1 = (float)(1.0 - std::pow(beta1, (double)u->step));
    const float bc2 = (float)(1.0 - std::pow(beta2, (double)u->step));
    k_un_adamw<<<256, 256, 0, s>>>(u->params, grad, u->m, u->v, u->is_weight, u->nparams, (float)lr, (float)beta1,
                                   (float)beta2, (float)eps, (float)weight_decay, bc1, bc2);
    MD_CHECK_LAUNCH();
    u->wt_ok = false;
    return MD_OK;
}

namespace {

const View kNone{nullptr, 0, 0};

md_status conv(const View& in, int cin, const View& out, int cout, int n, int batch, const float* W, const float* B,
               int act, cudaStream_t s, const View& zsave = kNone) {
    const long long vol = (long long)n * n * n;
    dim3 grid(blocks(vol, UN_TB), (unsigned)((cout + UN_CO - 1) / UN_CO), (unsigned)batch);
    k_un_conv3<<<grid, UN_TB, 0, s>>>(in, cin, out, cout, n, W, B, act, zsave);
    MD_CHECK_LAUNCH();
    return MD_OK;
}

md_status pool(const View& in, int c, int n, const View& out, int m, int batch, cudaStream_t s) {
    const long long tot = (long long)m * m * m * c * batch;
    k_un_pool<<<blocks(tot, 256), 256, 0, s>>>(in, c, n, out, m, batch);
    MD_CHECK_LAUNCH();
    return MD_OK;
}

md_status up(const View& in, int cin, int m, const View& out, int cout, int n, int batch, const float* W,
             const float* B, cudaStream_t s) {
    const long long vol = (long long)n * n * n;
    dim3 grid(blocks(vol, UN_TB), (unsigned)((cout + UN_CO - 1) / UN_CO), (unsigned)batch);
    k_un_up2<<<grid, UN_TB, 0, s>>>(in, cin, m, out, cout, n, W, B);
    MD_CHECK_LAUNCH();
    return MD_OK;
}

md_status gelu_back(const View& g, const View& z, int c, int n, int batch, cudaStream_t s) {
    const long long vol = (long long)n * n * n;
    k_un_gelu_back<<<blocks(vol * c * batch, 256), 256, 0, s>>>(g, z, c, vol, batch);
    MD_CHECK_LAUNCH();
    return MD_OK;
}

md_status wgrad(const View& dz, int cout, const View& x, int cin, int n, int batch, float* dW, float* db, cudaStream_t s) {
    const long long pairs = (long long)n * n * n * batch;
    const unsigned gx = (unsigned)((cout + UN_WCO - 1) / UN_WCO);
    dim3 grid(gx, (unsigned)cin, wsplit(pairs, (long long)gx * cin));
    k_un_wgrad<<<grid, UN_TB, 0, s>>>(dz, cout, x, cin, n, batch, dW, db);
    MD_CHECK_LAUNCH();
    return MD_OK;
}

md_status up_back(const View& dO, int cout, int n, const View& x, int cin, int m, int batch, const float* W,
                  const View& dX, float* dW, float* db, cudaStream_t s) {
    const long long mv = (long long)m * m * m;
    dim3 g1(blocks(mv, UN_TB), (unsigned)((cin + UN_CO - 1) / UN_CO), (unsigned)batch);
    k_un_up2_dgrad<<<g1, UN_TB, 0, s>>>(dO, cout, n, dX, cin, m, W);
    MD_CHECK_LAUNCH();
    const unsigned gx = (unsigned)((cout + UN_WCO - 1) / UN_WCO);
    dim3 g2(gx, (unsigned)cin, wsplit(mv * batch, (long long)gx * cin));
    k_un_up2_wgrad<<<g2, UN_TB, 0, s>>>(dO, cout, n, x, cin, m, batch, dW, db);
    MD_CHECK_LAUNCH();
    return MD_OK;
}

md_status pool_back(const View& dO, const View& x, int c, int n, const View& dX, int m, int batch, cudaStream_t s) {
    const long long tot = (long long)m * m * m * c * batch;
    k_un_pool_back<<<blocks(tot, 256), 256, 0, s>>>(dO, x, c, n, dX, m, batch);
    MD_CHECK_LAUNCH();
    return MD_OK;
}

// The activations of one pass (per-sample sizes in floats; every buffer holds
// `batch` samples back to back), and with training the pre-activations.
struct Acts {
    float *s0, *p0, *s1, *p1, *e2, *eb, *d1, *d0;    // forward
    float *z0, *z1, *z2, *zb, *zd1, *zd0;            // pre-activations (training)
    float *dd0, *ds0, *dd1, *ds1, *deb, *de2, *dp1, *dp0;  // gradients (training)
};

md_status layout(md_unet* u, int n, int batch, bool train, Acts* a, cudaStream_t s) {
    const int m1 = n / 2, m2 = m1 / 2;
    const long long v0 = (long long)n * n * n, v1 = (long long)m1 * m1 * m1, v2 = (long long)m2 * m2 * m2;
    const long long fwd[8] = {64 * v0, 32 * v1, 128 * v1, 64 * v2, 128 * v2, 128 * v2, 64 * v1, 32 * v0};
    const long long zs[6] = {32 * v0, 64 * v1, 128 * v2, 128 * v2, 64 * v1, 32 * v0};
    const long long gr[8] = {32 * v0, 64 * v0, 64 * v1, 128 * v1, 128 * v2, 128 * v2, 64 * v2, 32 * v1};
    long long per = 0;
    for (long long f : fwd) per += f;
    if (train) {
        for (long long f : zs) per += f;
        for (long long f : gr) per += f;
    }
    const size_t need = (size_t)per * (size_t)batch;
    if (need > u->ws_floats) {
        MD_CUDA(cudaStreamSynchronize(s));
        cudaFree(u->ws);
        u->ws = nullptr;
        u->ws_floats = 0;
        if (cudaMalloc(&u->ws, sizeof(float) * need) != cudaSuccess) { md_set_error("md_unet: cudaMalloc of the workspace failed"); return MD_ERR_OOM; }
        u->ws_floats = need;
    }
    float* q = u->ws;
    auto take = [&](long long floats) { float* p = q; q += floats * batch; return p; };
    float** f[8] = {&a->s0, &a->p0, &a->s1, &a->p1, &a->e2, &a->eb, &a->d1, &a->d0};
    for (int i = 0; i < 8; ++i) *f[i] = take(fwd[i]);
    float** z[6] = {&a->z0, &a->z1, &a->z2, &a->zb, &a->zd1, &a->zd0};
    float** g[8] = {&a->dd0, &a->ds0, &a->dd1, &a->ds1, &a->deb, &a->de2, &a->dp1, &a->dp0};
    for (int i = 0; i < 6; ++i) *z[i] = train ? take(zs[i]) : nullptr;
    for (int i = 0; i < 8; ++i) *g[i] = train ? take(gr[i]) : nullptr;
    return MD_OK;
}

// One forward pass; with train the pre-activations are kept for backward.
md_status forward_pass(md_unet* u, int n, int batch, const float* X, float* Y, const Acts& a, bool train, cudaStream_t s) {
    const int m1 = n / 2, m2 = m1 / 2;
    auto zv = [&](float* p, int c) { return train ? View{p, c, 0} : kNone; };
    const View x{const_cast<float*>(X), 2, 0};
    MD_TRY(conv(x, 2, View{a.s0, 64, 32}, 32, n, batch, u->Wc[0], u->Bc[0], 1, s, zv(a.z0, 32)));  // e0 -> s0[32:64]
    MD_TRY(pool(View{a.s0, 64, 32}, 32, n, View{a.p0, 32, 0}, m1, batch, s));
    MD_TRY(conv(View{a.p0, 32, 0}, 32, View{a.s1, 128, 64}, 64, m1, batch, u->Wc[1], u->Bc[1], 1, s, zv(a.z1, 64)));  // e1
    MD_TRY(pool(View{a.s1, 128, 64}, 64, m1, View{a.p1, 64, 0}, m2, batch, s));
    MD_TRY(conv(View{a.p1, 64, 0}, 64, View{a.e2, 128, 0}, 128, m2, batch, u->Wc[2], u->Bc[2], 1, s, zv(a.z2, 128)));
    MD_TRY(conv(View{a.e2, 128, 0}, 128, View{a.eb, 128, 0}, 128, m2, batch, u->Wc[3], u->Bc[3], 1, s, zv(a.zb, 128)));
    MD_TRY(up(View{a.eb, 128, 0}, 128, m2, View{a.s1, 128, 0}, 64, m1, batch, u->Wu[0], u->Bu[0], s));  // -> s1[0:64]
    MD_TRY(conv(View{a.s1, 128, 0}, 128, View{a.d1, 64, 0}, 64, m1, batch, u->Wc[4], u->Bc[4], 1, s, zv(a.zd1, 64)));
    MD_TRY(up(View{a.d1, 64, 0}, 64, m1, View{a.s0, 64, 0}, 32, n, batch, u->Wu[1], u->Bu[1], s));      // -> s0[0:32]
    MD_TRY(conv(View{a.s0, 64, 0}, 64, View{a.d0, 32, 0}, 32, n, batch, u->Wc[5], u->Bc[5], 1, s, zv(a.zd0, 32)));
    MD_TRY(conv(View{a.d0, 32, 0}, 32, View{Y, 1, 0}, 1, n, batch, u->Wc[6], u->Bc[6], 0, s));
    return MD_OK;
}

md_status check_shape(const char* who, int n, int batch) {
    if (n < 4 || n > 1024 || batch < 1) { md_set_error("%s: n=%d (needs 4..1024), batch=%d", who, n, batch); return MD_ERR_ARG; }
    return MD_OK;
}

}  // namespace

extern "C" md_status md_unet_forward(md_unet* u, int n, int batch, const float* X, float* Y, md_stream stream) {
    if (!u || !X || !Y) { md_set_error("md_unet_forward: NULL argument"); return MD_ERR_ARG; }
    MD_TRY(check_shape("md_unet_forward", n, batch));
    cudaStream_t s = (cudaStream_t)stream;
    Acts a;
    MD_TRY(layout(u, n, batch, false, &a, s));
    return forward_pass(u, n, batch, X, Y, a, false, s);
}

extern "C" md_status md_unet_backward(md_unet* u, int n, int batch, const float* X, const float* dY, float* dparams,
                                      float* dX, md_stream stream) {
    if (!u || !X || !dY || !dparams) { md_set_error("md_unet_backward: NULL argument"); return MD_ERR_ARG; }
    MD_TRY(check_shape("md_unet_backward", n, batch));
    cudaStream_t s = (cudaStream_t)stream;
    if (!u->wt_ok) {
        for (int l = 0; l < UN_CONVS; ++l) {
            const long long cnt = 27LL * kConv[l][0] * kConv[l][1];
            k_un_flip<<<blocks(cnt, 256), 256, 0, s>>>(u->Wc[l], kConv[l][1], kConv[l][0], u->Wt[l]);
            MD_CHECK_LAUNCH();
        }
        u->wt_ok = true;
    }
    Acts a;
    MD_TRY(layout(u, n, batch, true, &a, s));
    const int m1 = n / 2, m2 = m1 / 2;
    // the recomputed output itself is not needed: it lands in dd0, which the
    // output layer's input gradient overwrites below
    MD_TRY(forward_pass(u, n, batch, X, a.dd0, a, true, s));
    // parameter gradients at the parameters' offsets
    float *gWc[UN_CONVS], *gBc[UN_CONVS], *gWu[UN_UPS], *gBu[UN_UPS];
    for (int l = 0; l < UN_CONVS; ++l) { gWc[l] = dparams + (u->Wc[l] - u->params); gBc[l] = dparams + (u->Bc[l] - u->params); }
    for (int l = 0; l < UN_UPS; ++l) { gWu[l] = dparams + (u->Wu[l] - u->params); gBu[l] = dparams + (u->Bu[l] - u->params); }
    MD_CUDA(cudaMemsetAsync(dparams, 0, sizeof(float) * (size_t)u->nparams, s));
    const View dy{const_cast<float*>(dY), 1, 0};
    // output layer
    MD_TRY(wgrad(dy, 1, View{a.d0, 32, 0}, 32, n, batch, gWc[6], gBc[6], s));
    MD_TRY(conv(dy, 1, View{a.dd0, 32, 0}, 32, n, batch, u->Wt[6], nullptr, 0, s));
    MD_TRY(gelu_back(View{a.dd0, 32, 0}, View{a.zd0, 32, 0}, 32, n, batch, s));
    // decoder level 0: conv 64 -> 32 on [up0 | e0]
    MD_TRY(wgrad(View{a.dd0, 32, 0}, 32, View{a.s0, 64, 0}, 64, n, batch, gWc[5], gBc[5], s));
    MD_TRY(conv(View{a.dd0, 32, 0}, 32, View{a.ds0, 64, 0}, 64, n, batch, u->Wt[5], nullptr, 0, s));
    MD_TRY(up_back(View{a.ds0, 64, 0}, 32, n, View{a.d1, 64, 0}, 64, m1, batch, u->Wu[1], View{a.dd1, 64, 0}, gWu[1],
                   gBu[1], s));
    MD_TRY(gelu_back(View{a.dd1, 64, 0}, View{a.zd1, 64, 0}, 64, m1, batch, s));
    // decoder level 1: conv 128 -> 64 on [up1 | e1]
    MD_TRY(wgrad(View{a.dd1, 64, 0}, 64, View{a.s1, 128, 0}, 128, m1, batch, gWc[4], gBc[4], s));
    MD_TRY(conv(View{a.dd1, 64, 0}, 64, View{a.ds1, 128, 0}, 128, m1, batch, u->Wt[4], nullptr, 0, s));
    MD_TRY(up_back(View{a.ds1, 128, 0}, 64, m1, View{a.eb, 128, 0}, 128, m2, batch, u->Wu[0], View{a.deb, 128, 0},
                   gWu[0], gBu[0], s));
    MD_TRY(gelu_back(View{a.deb, 128, 0}, View{a.zb, 128, 0}, 128, m2, batch, s));
    // bottleneck and level-2 encoder
    MD_TRY(wgrad(View{a.deb, 128, 0}, 128, View{a.e2, 128, 0}, 128, m2, batch, gWc[3], gBc[3], s));
    MD_TRY(conv(View{a.deb, 128, 0}, 128, View{a.de2, 128, 0}, 128, m2, batch, u->Wt[3], nullptr, 0, s));
    MD_TRY(gelu_back(View{a.de2, 128, 0}, View{a.z2, 128, 0}, 128, m2, batch, s));
    MD_TRY(wgrad(View{a.de2, 128, 0}, 128, View{a.p1, 64, 0}, 64, m2, batch, gWc[2], gBc[2], s));
    MD_TRY(conv(View{a.de2, 128, 0}, 128, View{a.dp1, 64, 0}, 64, m2, batch, u->Wt[2], nullptr, 0, s));
    // level-1 encoder: its gradient is the skip's (ds1[64:128]) plus the pooled path's
    const View de1{a.ds1, 128, 64};
    MD_TRY(pool_back(View{a.dp1, 64, 0}, View{a.s1, 128, 64}, 64, m1, de1, m2, batch, s));
    MD_TRY(gelu_back(de1, View{a.z1, 64, 0}, 64, m1, batch, s));
    MD_TRY(wgrad(de1, 64, View{a.p0, 32, 0}, 32, m1, batch, gWc[1], gBc[1], s));
    MD_TRY(conv(de1, 64, View{a.dp0, 32, 0}, 32, m1, batch, u->Wt[1], nullptr, 0, s));
    // level-0 encoder: skip (ds0[32:64]) plus the pooled path
    const View de0{a.ds0, 64, 32};
    MD_TRY(pool_back(View{a.dp0, 32, 0}, View{a.s0, 64, 32}, 32, n, de0, m1, batch, s));
    MD_TRY(gelu_back(de0, View{a.z0, 32, 0}, 32, n, batch, s));
    MD_TRY(wgrad(de0, 32, View{const_cast<float*>(X), 2, 0}, 2, n, batch, gWc[0], gBc[0], s));
    if (dX) MD_TRY(conv(de0, 32, View{dX, 2, 0}, 2, n, batch, u->Wt[0], nullptr, 0, s));
    return MD_OK;
}
