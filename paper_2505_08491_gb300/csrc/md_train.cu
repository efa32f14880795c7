// Unsupervised training of the preconditioner network (Section 3.2, eq.
// (risk) and (trained_preconditioner); the squared residual loss of Section
// 5.1), written on the library's own kernels:
//
//   per sample (instance A = K + beta M, residual r = [r0; r1]):
//     z1 = B11^{-1} r1,  l = beta Pi^T W Psi z1,  b0 = r0 + l,  s = ||b0||,
//     Y = N([r0/s, l/s, d_h]),  y = Y on interior nodes (0 on Dirichlet ones),
//     L = || C y / alpha - b0 / s ||^2  (= ||C z0 - b0||^2 / ||b0||^2 with
//     z0 = (s/alpha) y, C = K00 + beta Pi^T W Pi),
//     dL/dy = (2/alpha) C (C y / alpha - b0/s)  (C symmetric).
//   Minibatch mean; backward through the six layers (input gradients with
//   the flipped, transposed kernels times GELU'(z); weight gradients as
//   sums over grid rows of dZ (x) shifted activations); AdamW on FP32
//   master weights, BF16 copies re-packed after every step.
//
// C y is the operator apply of the whole system on [y; 0]: its grid part is
// K00 y + beta Pi^T W Pi y = C y.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <random>

#include "md_cnn.h"
#include "md_common.cuh"
#include "md_conv_tc.h"

md_status launch_prec_input(const Tables& T, const InstDesc* d, const long long* off, const float* v, float* z,
                            KState* st, int ninst, int max_n1, double* part, cudaStream_t s);

namespace {
const int kCin[MD_CNN_LAYERS] = {3, 32, 32, 32, 32, 32};
const int kCout[MD_CNN_LAYERS] = {32, 32, 32, 32, 32, 1};

size_t host_w_off(int l) {
    size_t o = 0;
    for (int i = 0; i < l; ++i) o += (size_t)kCout[i] * kCin[i] * 27 + kCout[i];
    return o;
}

__device__ __forceinline__ void unpack8(const uint4& r, float* x) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&r);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float2 f = __bfloat1622float2(h[k]);
        x[2 * k] = f.x;
        x[2 * k + 1] = f.y;
    }
}
__device__ __forceinline__ uint4 pack8(const float* v) {
    uint4 r;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&r);
#pragma unroll
    for (int k = 0; k < 4; ++k) h[k] = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
    return r;
}
}  // namespace

// ---- input gradient of a layer (CUDA cores) ------------------------------------
// dA[p][c] = sum_t sum_o Wt[t][o][c] dZ[p + off_t][o]  (flipped, transposed
// kernel: the adjoint of the forward correlation), then
//   MODE 0: dZ_prev[p][c] = dA[p][c] * GELU'(Z_prev[p][c])  (BF16 out)
//   MODE 1: dX[sample][c][n] = dA (FP32, c < 3; the network input gradient)
template <int CIN8, int COUT, int MODE>
__global__ void __launch_bounds__(128) k_dgrad(const __nv_bfloat16* __restrict__ dz, const long long* __restrict__ dz_off,
                                               const __nv_bfloat16* __restrict__ Wt, const __nv_bfloat16* __restrict__ zprev,
                                               __nv_bfloat16* __restrict__ out, const long long* __restrict__ out_off,
                                               float* __restrict__ dx, const Seg* __restrict__ seg,
                                               const int* __restrict__ Ns) {
    constexpr int CIN = CIN8 * 8;
    constexpr int NW = 27 * CIN * COUT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __nv_bfloat16* sw = reinterpret_cast<__nv_bfloat16*>(smem_raw);
    for (int i = threadIdx.x; i < NW; i += blockDim.x) sw[i] = Wt[i];
    __syncthreads();
    const Seg sg = seg[blockIdx.x];
    const int N = Ns[sg.inst], M = N + 1;
    const long long Pd = N + 3, P = Pd * Pd * Pd;
    const __nv_bfloat16* zi = dz + dz_off[sg.inst];
    for (int n = sg.begin + threadIdx.x; n < sg.end; n += blockDim.x) {
        const int i = n % M, r = n / M, j = r % M, k = r / M;
        const long long p = (i + 1) + Pd * ((j + 1) + Pd * (k + 1));
        float acc[COUT];
#pragma unroll
        for (int c = 0; c < COUT; ++c) acc[c] = 0.f;
        for (int tap = 0; tap < 27; ++tap) {
            const int dzz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dxx = tap % 3 - 1;
            const long long q = p + dxx + Pd * (dy + Pd * dzz);
#pragma unroll
            for (int c8 = 0; c8 < CIN8; ++c8) {
                float x[8];
                unpack8(*reinterpret_cast<const uint4*>(zi + (c8 * P + q) * 8), x);
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const __nv_bfloat16* wr = sw + ((size_t)tap * CIN + c8 * 8 + e) * COUT;
#pragma unroll
                    for (int c = 0; c < COUT; c += 8) {
                        float wv[8];
                        unpack8(*reinterpret_cast<const uint4*>(wr + c), wv);
#pragma unroll
                        for (int u = 0; u < 8; ++u) acc[c + u] = fmaf(wv[u], x[e], acc[c + u]);
                    }
                }
            }
        }
        if (MODE == 0) {
            const __nv_bfloat16* zp = zprev + out_off[sg.inst];
            __nv_bfloat16* o = out + out_off[sg.inst];
#pragma unroll
            for (int c8 = 0; c8 < COUT / 8; ++c8) {
                float zz[8], g[8];
                unpack8(*reinterpret_cast<const uint4*>(zp + (c8 * P + p) * 8), zz);
#pragma unroll
                for (int e = 0; e < 8; ++e) g[e] = acc[c8 * 8 + e] * gelu_grad_fast(zz[e]);
                *reinterpret_cast<uint4*>(o + (c8 * P + p) * 8) = pack8(g);
            }
        } else {
            const long long n3 = (long long)M * M * M;
            float* d = dx + (long long)sg.inst * 3 * n3;
            for (int c = 0; c < 3; ++c) d[c * n3 + n] = acc[c];
        }
    }
}

// ---- weight gradient of a layer (CUDA cores) -------------------------------------
// dW[o][c][t] = sum_p dZ[p][o] A[p + off_t][c],  db[o] = sum_p dZ[p][o], over
// the padded rows of the planes holding grid nodes (dZ is zero on halo rows).
// Each block accumulates its tiles of 128 rows; partials are summed in block
// order by k_wgrad_reduce (deterministic).
struct RowTile { int inst, p0; };

template <int CIN8, int COUT>
__global__ void __launch_bounds__(256) k_wgrad(const __nv_bfloat16* __restrict__ act, const long long* __restrict__ act_off,
                                               const __nv_bfloat16* __restrict__ dz, const long long* __restrict__ dz_off,
                                               const int* __restrict__ Ns, const RowTile* __restrict__ tiles, int ntiles,
                                               float* __restrict__ part) {
    constexpr int CIN = CIN8 * 8;
    constexpr int ZC8 = COUT >= 8 ? COUT / 8 : 1;
    constexpr int NPAIR = CIN * COUT;
    constexpr int PPT = NPAIR >= 256 ? NPAIR / 256 : 1;   // (c, o) pairs per thread
    constexpr int NSTRIDE = 27 * CIN * COUT + COUT;
    __shared__ float sz[128][ZC8 * 8];
    __shared__ float sa[128][CIN];
    const int tid = threadIdx.x;
    const bool active = tid < (NPAIR >= 256 ? 256 : NPAIR);
    // pair p -> (c, o): PPT consecutive o for one c
    const int c = active ? (tid * PPT) / COUT : 0;
    const int o0 = active ? (tid * PPT) % COUT : 0;
    float acc[27][PPT];
    float bacc[PPT];
#pragma unroll
    for (int t = 0; t < 27; ++t)
#pragma unroll
        for (int k = 0; k < PPT; ++k) acc[t][k] = 0.f;
#pragma unroll
    for (int k = 0; k < PPT; ++k) bacc[k] = 0.f;
    for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
        const RowTile T = tiles[ti];
        const long long Pd = Ns[T.inst] + 3, P = Pd * Pd * Pd;
        const __nv_bfloat16* zi = dz + dz_off[T.inst];
        const __nv_bfloat16* ai = act + act_off[T.inst];
        __syncthreads();
        for (int e = tid; e < 128 * ZC8; e += blockDim.x) {
            const int r = e / ZC8, c8 = e % ZC8;
            float v[8];
            unpack8(*reinterpret_cast<const uint4*>(zi + ((long long)c8 * P + T.p0 + r) * 8), v);
#pragma unroll
            for (int u = 0; u < 8; ++u) sz[r][c8 * 8 + u] = v[u];
        }
        __syncthreads();
        if (active && c == 0)
            for (int r = 0; r < 128; ++r)
#pragma unroll
                for (int k = 0; k < PPT; ++k) bacc[k] += sz[r][o0 + k];
#pragma unroll
        for (int t = 0; t < 27; ++t) {
            const long long off = (t % 3 - 1) + Pd * ((t / 3) % 3 - 1 + Pd * (t / 9 - 1));
            __syncthreads();
            for (int e = tid; e < 128 * CIN8; e += blockDim.x) {
                const int r = e / CIN8, c8 = e % CIN8;
                float v[8];
                unpack8(*reinterpret_cast<const uint4*>(ai + ((long long)c8 * P + T.p0 + r + off) * 8), v);
#pragma unroll
                for (int u = 0; u < 8; ++u) sa[r][c8 * 8 + u] = v[u];
            }
            __syncthreads();
            if (active) {
                float a2[PPT];
#pragma unroll
                for (int k = 0; k < PPT; ++k) a2[k] = 0.f;
                for (int r = 0; r < 128; ++r) {
                    const float av = sa[r][c];
#pragma unroll
                    for (int k = 0; k < PPT; ++k) a2[k] = fmaf(av, sz[r][o0 + k], a2[k]);
                }
#pragma unroll
                for (int k = 0; k < PPT; ++k) acc[t][k] += a2[k];
            }
        }
    }
    if (!active) return;
    float* pb = part + (size_t)blockIdx.x * NSTRIDE;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int o = o0 + k;
#pragma unroll
        for (int t = 0; t < 27; ++t) pb[((size_t)o * CIN + c) * 27 + t] = acc[t][k];
        if (c == 0) pb[27 * CIN * COUT + o] = bacc[k];
    }
}

// grad[l's block of the flat layout] = scale * sum over blocks of the partials
// (padded input channels dropped)
__global__ void k_wgrad_reduce(const float* __restrict__ part, int nblk, int cin_pad, int cin, int cout, float scale,
                               float* __restrict__ grad) {
    const int nstride = 27 * cin_pad * cout + cout;
    const int nout = cout * cin * 27 + cout;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nout; idx += gridDim.x * blockDim.x) {
        int src;
        if (idx < cout * cin * 27) {
            const int o = idx / (cin * 27), rem = idx % (cin * 27), c = rem / 27, t = rem % 27;
            src = (o * cin_pad + c) * 27 + t;
        } else {
            src = 27 * cin_pad * cout + (idx - cout * cin * 27);
        }
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += part[(size_t)b * nstride + src];
        grad[idx] = (float)(scale * s);
    }
}

// ---- loss pieces -------------------------------------------------------------------
// mask Dirichlet nodes of the grid part of per-slot vectors
__device__ __forceinline__ bool is_bd(int n, int N) {
    const int M = N + 1, i = n % M, r = n / M, j = r % M, k = r / M;
    return i == 0 || i == N || j == 0 || j == N || k == 0 || k == N;
}

__global__ void k_mask_grid(const Seg* __restrict__ seg, const InstDesc* __restrict__ D, const long long* __restrict__ off,
                            float* v, int zero_1d) {
    const Seg sg = seg[blockIdx.x];
    const InstDesc& d = D[sg.inst];
    float* vi = v + off[sg.inst];
    for (int e = sg.begin + threadIdx.x; e < sg.end; e += blockDim.x) {
        if (e >= d.n3) { if (zero_1d) vi[e] = 0.f; continue; }
        if (!d.natural && is_bd(e, d.N)) vi[e] = 0.f;
    }
}

// res = C y / alpha - (r0 + l) / s on interior nodes (0 elsewhere, 1D part 0);
// loss[slot] += sum res^2
__global__ void k_train_res(const Seg* __restrict__ seg, const InstDesc* __restrict__ D, const long long* __restrict__ off,
                            const float* __restrict__ cy, const float* __restrict__ r, const KState* __restrict__ st,
                            float* res, double* loss) {
    __shared__ double sh[32];
    const Seg sg = seg[blockIdx.x];
    const InstDesc& d = D[sg.inst];
    const long long o = off[sg.inst];
    const double s = st[sg.inst].s;
    const float inv_a = (float)(1.0 / d.alpha), inv_s = s > 0 ? (float)(1.0 / s) : 0.f;
    double acc = 0.0;
    for (int e = sg.begin + threadIdx.x; e < sg.end; e += blockDim.x) {
        float v = 0.f;
        if (e < d.n3 && (d.natural || !is_bd(e, d.N))) v = cy[o + e] * inv_a - (r[o + e] + d.lift32[e]) * inv_s;
        res[o + e] = v;
        acc += (double)v * v;
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        atomicAdd(&loss[sg.inst], t);
    }
}

// dY (network output gradient) = scale * (C res) on interior nodes, packed
// as channel 0 of a dx-paired one-chunk BF16 padded buffer
__global__ void k_train_dy(const Seg* __restrict__ seg, const InstDesc* __restrict__ D, const long long* __restrict__ off,
                           const float* __restrict__ cres, float scale, __nv_bfloat16* __restrict__ dy,
                           const long long* __restrict__ dy_off) {
    const Seg sg = seg[blockIdx.x];
    const InstDesc& d = D[sg.inst];
    const int N = d.N, M = N + 1;
    const long long Pd = N + 3;
    for (int n = sg.begin + threadIdx.x; n < sg.end; n += blockDim.x) {
        const int i = n % M, r = n / M, j = r % M, k = r / M;
        const long long p = (i + 1) + Pd * ((j + 1) + Pd * (k + 1));
        float own[3] = {0.f, 0.f, 0.f}, nx[3] = {0.f, 0.f, 0.f};
        if (d.natural || !is_bd(n, N)) own[0] = scale * cres[off[sg.inst] + n] / (float)d.alpha;
        if (i < N && (d.natural || !is_bd(n + 1, N))) nx[0] = scale * cres[off[sg.inst] + n + 1] / (float)d.alpha;
        store_dx_pair(dy + dy_off[sg.inst] + p * 8, own, nx, i == 0);
    }
}

// raw dY (FP32 grid per sample) -> dx-paired one-chunk BF16 padded buffer
__global__ void k_pack_dy_raw(const Seg* __restrict__ seg, const int* __restrict__ Ns, const float* __restrict__ dY,
                              __nv_bfloat16* __restrict__ dy, const long long* __restrict__ dy_off) {
    const Seg sg = seg[blockIdx.x];
    const int N = Ns[sg.inst], M = N + 1;
    const long long Pd = N + 3, n3 = (long long)M * M * M;
    for (int n = sg.begin + threadIdx.x; n < sg.end; n += blockDim.x) {
        const int i = n % M, r = n / M, j = r % M, k = r / M;
        const long long p = (i + 1) + Pd * ((j + 1) + Pd * (k + 1));
        const float own[3] = {dY[sg.inst * n3 + n], 0.f, 0.f};
        const float nx[3] = {i < N ? dY[sg.inst * n3 + n + 1] : 0.f, 0.f, 0.f};
        store_dx_pair(dy + dy_off[sg.inst] + p * 8, own, nx, i == 0);
    }
}

__global__ void k_set_active(KState* st, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) st[i].active = 1;
}

// AdamW (decoupled weight decay on weights, not biases)
__global__ void k_adamw(float* w, const float* g, float* m, float* v, const unsigned char* is_weight, int n, float lr,
                        float b1, float b2, float eps, float wd, float bc1, float bc2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float mh = mi / bc1, vh = vi / bc2;
        float wi = w[i];
        if (is_weight[i]) wi -= lr * wd * wi;
        w[i] = wi - lr * mh / (sqrtf(vh) + eps);
    }
}

// ---------------------------------------------------------------------------
// host side
struct TrainWork {
    int B = 0, N = 0;
    std::vector<void*> allocs;
    CnnWork* cw = nullptr;
    __nv_bfloat16* A[MD_CNN_LAYERS] = {};  // A[1..5]
    __nv_bfloat16* Z[MD_CNN_LAYERS] = {};  // Z[1..5]
    __nv_bfloat16 *dza = nullptr, *dzb = nullptr, *dy1 = nullptr;
    RowTile* tiles = nullptr;
    int ntiles = 0, wblocks = 0;
    float* part = nullptr;
    float* grad = nullptr;                 // MD_CNN_NPARAMS
    float* zero_bias = nullptr;            // 32 zeros: the adjoint convolutions have no bias
    // solve-side (training samples with operators)
    long long stride = 0;                  // per-slot vector stride (n3 + max n1)
    float *rv = nullptr, *yv = nullptr, *cy = nullptr, *res = nullptr, *cres = nullptr;
    long long* voff = nullptr;
    InstDesc* d = nullptr;
    KState* st = nullptr;
    double* loss = nullptr;
    double* part3 = nullptr;               // partial sums of ||r0||^2
    int max_n1 = 0;
    std::vector<float*> scratch;           // per slot: t32 (nq), lift (n3), ltouch (ntouch)
};

static void train_work_destroy(TrainWork* t) {
    if (!t) return;
    cnn_work_destroy(t->cw);
    dev_free_all(&t->allocs);
    delete t;
}

// B slots of grid N; max_n1/max_nq/max_touch size the per-slot scratch
static md_status train_work_create(int B, int N, int max_n1, int max_nq, int max_touch, TrainWork** out) {
    TrainWork* t = new TrainWork();
    t->B = B;
    t->N = N;
    md_status st = cnn_work_create(std::vector<int>(B, N), &t->cw);
    if (st != MD_OK) { delete t; return st; }
    auto chk = [&](md_status s2) { if (st == MD_OK) st = s2; };
    const long long Pd = N + 3, P = Pd * Pd * Pd;
    const size_t ab_elems = (size_t)(2 * CNN_MARGIN_ROWS + 4 * P * B) * 8;
    const size_t x0_elems = (size_t)(2 * CNN_MARGIN_ROWS + P * B) * 8;
    for (int l = 1; l < MD_CNN_LAYERS; ++l) {
        chk(dev_alloc(&t->allocs, &t->A[l], ab_elems));
        chk(dev_alloc(&t->allocs, &t->Z[l], ab_elems));
    }
    chk(dev_alloc(&t->allocs, &t->dza, ab_elems));
    chk(dev_alloc(&t->allocs, &t->dzb, ab_elems));
    chk(dev_alloc(&t->allocs, &t->dy1, x0_elems));
    std::vector<RowTile> tiles;
    for (int i = 0; i < B; ++i)
        for (long long p = Pd * Pd; p < (N + 2) * Pd * Pd; p += 128) tiles.push_back({i, (int)p});
    t->ntiles = (int)tiles.size();
    t->wblocks = std::max(1, std::min(t->ntiles, 2 * t->cw->nsm));
    chk(dev_upload(&t->allocs, &t->tiles, tiles.data(), tiles.size()));
    chk(dev_alloc(&t->allocs, &t->part, (size_t)t->wblocks * (27 * 32 * 32 + 32), false));
    chk(dev_alloc(&t->allocs, &t->grad, (size_t)MD_CNN_NPARAMS));
    chk(dev_alloc(&t->allocs, &t->zero_bias, 32));
    if (max_n1 >= 0) {
        const long long n3 = (long long)(N + 1) * (N + 1) * (N + 1);
        t->stride = n3 + max_n1;
        std::vector<long long> off(B);
        for (int i = 0; i < B; ++i) off[i] = i * t->stride;
        chk(dev_upload(&t->allocs, &t->voff, off.data(), off.size()));
        chk(dev_alloc(&t->allocs, &t->rv, (size_t)(B * t->stride)));
        chk(dev_alloc(&t->allocs, &t->yv, (size_t)(B * t->stride)));
        chk(dev_alloc(&t->allocs, &t->cy, (size_t)(B * t->stride)));
        chk(dev_alloc(&t->allocs, &t->res, (size_t)(B * t->stride)));
        chk(dev_alloc(&t->allocs, &t->cres, (size_t)(B * t->stride)));
        chk(dev_alloc(&t->allocs, &t->d, (size_t)B));
        chk(dev_alloc(&t->allocs, &t->st, (size_t)B));
        chk(dev_alloc(&t->allocs, &t->loss, (size_t)B));
        // per block of the n3 table (||r0||^2) or of the touched-node table (the lift)
        chk(dev_alloc(&t->allocs, &t->part3, (size_t)B * (n3 / 256 + 2) * MD_MAXR));
        t->max_n1 = max_n1;
        for (int i = 0; i < B && st == MD_OK; ++i) {
            float *a = nullptr, *b = nullptr, *c = nullptr;
            chk(dev_alloc(&t->allocs, &a, (size_t)max_nq));
            chk(dev_alloc(&t->allocs, &b, (size_t)n3));
            chk(dev_alloc(&t->allocs, &c, (size_t)std::max(max_touch, 1)));
            t->scratch.push_back(a);
            t->scratch.push_back(b);
            t->scratch.push_back(c);
        }
    }
    if (st != MD_OK) { train_work_destroy(t); return st; }
    *out = t;
    return MD_OK;
}

template <int CIN8, int COUT, int MODE>
static md_status launch_dgrad(const TrainWork* t, const __nv_bfloat16* dz, const long long* dz_off,
                              const __nv_bfloat16* Wt, const __nv_bfloat16* zprev, __nv_bfloat16* out, float* dx,
                              cudaStream_t s) {
    const size_t smem = (size_t)27 * CIN8 * 8 * COUT * sizeof(__nv_bfloat16);
    auto kern = k_dgrad<CIN8, COUT, MODE>;
    MD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<t->cw->nodes.nblocks, 128, smem, s>>>(dz, dz_off, Wt, zprev, out, t->cw->off_ab, dx, t->cw->nodes.seg, t->cw->N);
    MD_CHECK_LAUNCH();
    return MD_OK;
}

template <int CIN8, int COUT>
static md_status launch_wgrad(TrainWork* t, const __nv_bfloat16* act, const long long* act_off,
                              const __nv_bfloat16* dz, const long long* dz_off, int layer, float scale, cudaStream_t s) {
    k_wgrad<CIN8, COUT><<<t->wblocks, 256, 0, s>>>(act, act_off, dz, dz_off, t->cw->N, t->tiles, t->ntiles, t->part);
    MD_CHECK_LAUNCH();
    k_wgrad_reduce<<<64, 256, 0, s>>>(t->part, t->wblocks, CIN8 * 8, kCin[layer], kCout[layer], scale,
                                      t->grad + host_w_off(layer));
    MD_CHECK_LAUNCH();
    return MD_OK;
}

// Input gradient of layer l (1-5) on the tensor cores: the tcgen05
// convolution of the forward pass run as the adjoint (flipped, transposed
// weights, no bias; the last layer's 1 -> 32 adjoint as the first layer's
// kind) with the epilogue dZ_prev = dA * GELU'(Z_prev).
static md_status launch_dgrad_tc(const md_cnn* c, TrainWork* t, int l, const __nv_bfloat16* dz, const long long* dz_off,
                                 const __nv_bfloat16* zprev, __nv_bfloat16* out, cudaStream_t s) {
    CnnWork* w = t->cw;
    TcArgs a{};
    a.Ns = w->N;
    a.sched = TcSched{w->all_inst, w->all_pre, w->all_count};
    a.W = w->W;
    a.NS = w->NS;
    a.err = w->err;
    a.io = OutIO{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    a.mode = CONV_RAW;
    a.in = dz;
    a.in_off = dz_off;
    a.out = out;
    a.out_off = w->off_ab;
    a.wimg = c->wtmma + c->wtmma_off[l];
    a.bias = t->zero_bias;
    a.cout = 32;
    a.zprev = zprev;
    a.dgrad = 1;
    return tc_launch(l == MD_CNN_LAYERS - 1 ? 1 : 0, w->tps, a, w->ngroups, s);
}

// Backward from dZ6 (in t->dy1) through all layers; gradient into t->grad
// (scaled by `scale`); dX (FP32 raw layout) when dx != NULL.  Input gradients
// of layers 1-5 on the tensor cores with the tensor-core engine, weight
// gradients on CUDA cores.
static md_status backward_all(const md_cnn* c, TrainWork* t, float scale, float* dx, cudaStream_t s) {
    CnnWork* w = t->cw;
    const bool tc = c->engine == 0;
    // layer 5 (32 -> 1)
    MD_TRY((launch_wgrad<4, 1>(t, t->A[5], w->off_ab, t->dy1, w->off_x0, 5, scale, s)));
    if (tc) MD_TRY(launch_dgrad_tc(c, t, 5, t->dy1, w->off_x0, t->Z[5], t->dza, s));
    else MD_TRY((launch_dgrad<1, 32, 0>(t, t->dy1, w->off_x0, c->wt + c->wt_off[5], t->Z[5], t->dza, nullptr, s)));
    __nv_bfloat16* cur = t->dza;
    __nv_bfloat16* nxt = t->dzb;
    for (int l = 4; l >= 1; --l) {
        MD_TRY((launch_wgrad<4, 32>(t, t->A[l], w->off_ab, cur, w->off_ab, l, scale, s)));
        if (tc) MD_TRY(launch_dgrad_tc(c, t, l, cur, w->off_ab, t->Z[l], nxt, s));
        else MD_TRY((launch_dgrad<4, 32, 0>(t, cur, w->off_ab, c->wt + c->wt_off[l], t->Z[l], nxt, nullptr, s)));
        std::swap(cur, nxt);
    }
    MD_TRY((launch_wgrad<1, 32>(t, w->x0, w->off_x0, cur, w->off_ab, 0, scale, s)));
    if (dx) MD_TRY((launch_dgrad<4, 8, 1>(t, cur, w->off_ab, c->wt + c->wt_off[0], nullptr, nullptr, dx, s)));
    return MD_OK;
}

// ---- raw backward (autograd) ------------------------------------------------------------
extern "C" md_status md_cnn_backward(const md_cnn* c, int n_nodes_edge, int batch, const float* X, const float* dY,
                                     float* dparams, float* dX, md_stream stream) {
    if (!c || !X || !dY || !dparams || n_nodes_edge < 2 || batch < 1) { md_set_error("md_cnn_backward: bad argument"); return MD_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    TrainWork* t = nullptr;
    MD_TRY(train_work_create(batch, n_nodes_edge - 1, -1, 0, 0, &t));
    md_status st = MD_OK;
    const long long n3 = (long long)n_nodes_edge * n_nodes_edge * n_nodes_edge;
    std::vector<long long> off(batch);
    for (int i = 0; i < batch; ++i) off[i] = i * n3;
    long long* doff = nullptr;
    float* ytmp = nullptr;
    st = dev_upload(&t->allocs, &doff, off.data(), off.size());
    if (st == MD_OK) st = dev_alloc(&t->allocs, &ytmp, (size_t)(batch * n3), false);
    if (st == MD_OK) st = cnn_pack_raw(t->cw, X, s);
    OutIO io{ytmp, doff, nullptr, nullptr, nullptr, nullptr};
    if (st == MD_OK) st = cnn_forward_train(c, t->cw, t->A, t->Z, io, s);
    if (st == MD_OK) {
        k_pack_dy_raw<<<t->cw->nodes.nblocks, 128, 0, s>>>(t->cw->nodes.seg, t->cw->N, dY, t->dy1, t->cw->off_x0);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = md_cuda_status(e, "k_pack_dy_raw", __FILE__, __LINE__);
    }
    if (st == MD_OK) st = backward_all(c, t, 1.0f, dX, s);
    if (st == MD_OK) {
        cudaError_t e = cudaMemcpyAsync(dparams, t->grad, sizeof(float) * MD_CNN_NPARAMS, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = md_cuda_status(e, "md_cnn_backward", __FILE__, __LINE__);
    }
    train_work_destroy(t);
    return st;
}

// ---- training on instances ------------------------------------------------------------------
// One minibatch: loss (sum over slots written to loss_out) and gradient of
// the mean loss in t->grad.
static md_status minibatch(const md_cnn* c, TrainWork* t, const std::vector<const md_op*>& ops,
                           const std::vector<const float*>& rs, double* loss_out, cudaStream_t s) {
    const int B = (int)ops.size();
    // per-slot descriptors with private scratch
    std::vector<InstDesc> desc(B);
    std::vector<const InstDesc*> ptrs(B);
    for (int i = 0; i < B; ++i) {
        desc[i] = ops[i]->h;
        desc[i].t32 = t->scratch[3 * i];
        desc[i].lift32 = t->scratch[3 * i + 1];
        desc[i].ltouch32 = t->scratch[3 * i + 2];
        ptrs[i] = &desc[i];
    }
    std::vector<void*> tmp;
    Tables T;
    MD_TRY(build_tables(ptrs, &T, &tmp));
    md_status st = MD_OK;
    auto run = [&]() -> md_status {
        MD_CUDA(cudaMemcpyAsync(t->d, desc.data(), sizeof(InstDesc) * B, cudaMemcpyHostToDevice, s));
        for (int i = 0; i < B; ++i) {
            MD_CUDA(cudaMemsetAsync(desc[i].lift32, 0, sizeof(float) * desc[i].n3, s));
            MD_CUDA(cudaMemcpyAsync(t->rv + i * t->stride, rs[i], sizeof(float) * desc[i].n, cudaMemcpyDeviceToDevice, s));
        }
        MD_CUDA(cudaMemsetAsync(t->loss, 0, sizeof(double) * B, s));
        k_mask_grid<<<T.vec.nblocks, MD_TB, 0, s>>>(T.vec.seg, t->d, t->voff, t->rv, 0);
        k_set_active<<<(B + 31) / 32, 32, 0, s>>>(t->st, B);
        MD_CHECK_LAUNCH();
        // preconditioner input: ||r0||^2, 1D solve + lift, s, packed X
        MD_TRY(launch_prec_input(T, t->d, t->voff, t->rv, t->yv, t->st, B, t->max_n1, t->part3, s));
        MD_TRY(cnn_pack_prec(t->cw, t->d, t->rv, t->voff, t->st, t->yv, s));  // y is overwritten by the raw forward
        OutIO io{t->yv, t->voff, nullptr, nullptr, nullptr, nullptr};
        MD_TRY(cnn_forward_train(c, t->cw, t->A, t->Z, io, s));
        k_mask_grid<<<T.vec.nblocks, MD_TB, 0, s>>>(T.vec.seg, t->d, t->voff, t->yv, 1);
        MD_CHECK_LAUNCH();
        MD_TRY(launch_apply(T, t->d, B, MD_FP32, t->yv, t->voff, t->cy, s));
        k_train_res<<<T.vec.nblocks, MD_TB, 0, s>>>(T.vec.seg, t->d, t->voff, t->cy, t->rv, t->st, t->res, t->loss);
        MD_CHECK_LAUNCH();
        MD_TRY(launch_apply(T, t->d, B, MD_FP32, t->res, t->voff, t->cres, s));
        k_train_dy<<<t->cw->nodes.nblocks, 128, 0, s>>>(t->cw->nodes.seg, t->d, t->voff, t->cres, 2.0f / B, t->dy1,
                                                         t->cw->off_x0);
        MD_CHECK_LAUNCH();
        MD_TRY(backward_all(c, t, 1.0f, nullptr, s));
        std::vector<double> l(B);
        MD_CUDA(cudaMemcpyAsync(l.data(), t->loss, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
        MD_CUDA(cudaStreamSynchronize(s));
        *loss_out = std::accumulate(l.begin(), l.end(), 0.0);
        return MD_OK;
    };
    st = run();
    dev_free_all(&tmp);
    return st;
}

static md_status check_samples(int count, const md_op* const* ops, const float* const* r) {
    if (count < 1 || !ops || !r) { md_set_error("training: no samples"); return MD_ERR_ARG; }
    for (int i = 0; i < count; ++i)
        if (!ops[i] || !r[i]) { md_set_error("training: sample %d has a NULL operator or residual", i); return MD_ERR_ARG; }
    return MD_OK;
}

extern "C" md_status md_train_loss(const md_cnn* c, int count, const md_op* const* ops, const float* const* r,
                                   double* loss, float* dparams, md_stream stream) {
    if (!c || !loss) { md_set_error("md_train_loss: NULL argument"); return MD_ERR_ARG; }
    MD_TRY(check_samples(count, ops, r));
    const int N = ops[0]->h.N;
    int max_n1 = 0, max_nq = 0, max_t = 0;
    for (int i = 0; i < count; ++i) {
        if (ops[i]->h.N != N) { md_set_error("md_train_loss: samples of one call share the grid size"); return MD_ERR_ARG; }
        max_n1 = std::max(max_n1, ops[i]->h.n1);
        max_nq = std::max(max_nq, ops[i]->h.nq);
        max_t = std::max(max_t, ops[i]->h.ntouch);
    }
    cudaStream_t s = (cudaStream_t)stream;
    TrainWork* t = nullptr;
    MD_TRY(train_work_create(count, N, max_n1, max_nq, max_t, &t));
    std::vector<const md_op*> vo(ops, ops + count);
    std::vector<const float*> vr(r, r + count);
    double L = 0.0;
    md_status st = minibatch(c, t, vo, vr, &L, s);
    if (st == MD_OK) {
        *loss = L / count;
        if (dparams) {
            cudaError_t e = cudaMemcpy(dparams, t->grad, sizeof(float) * MD_CNN_NPARAMS, cudaMemcpyDeviceToDevice);
            if (e != cudaSuccess) st = md_cuda_status(e, "md_train_loss", __FILE__, __LINE__);
        }
    }
    train_work_destroy(t);
    return st;
}

// ---- the U-net's training loss (the same risk, Section 3.2 eq. (risk)) ----
// Input X = [b0 / s, d] (the U-net's two channels: the 3D block's right-hand
// side b0 = r0 + l scaled by s = ||b0||, and the distance field), output y;
// z0 = (s / alpha) y; loss ||C y / alpha - b0 / s||^2 over the unknown rows.

__global__ void k_unet_pack(const Seg* __restrict__ seg, const InstDesc* __restrict__ D, const long long* __restrict__ off,
                            const float* __restrict__ r, const KState* __restrict__ st, float* __restrict__ X) {
    const Seg sg = seg[blockIdx.x];
    const InstDesc& d = D[sg.inst];
    const long long n3 = d.n3, o = off[sg.inst];
    const double s = st[sg.inst].s;
    const float inv_s = s > 0 ? (float)(1.0 / s) : 0.f;
    float* x = X + (long long)sg.inst * 2 * n3;
    for (int e = sg.begin + threadIdx.x; e < sg.end; e += blockDim.x) {
        x[e] = (r[o + e] + d.lift32[e]) * inv_s;
        x[n3 + e] = d.dist[e];
    }
}

// the network output into the instance vector's 3D part (1D part zero)
__global__ void k_unet_scatter(const Seg* __restrict__ seg, const InstDesc* __restrict__ D,
                               const long long* __restrict__ off, const float* __restrict__ Y, float* __restrict__ v) {
    const Seg sg = seg[blockIdx.x];
    const InstDesc& d = D[sg.inst];
    const float* y = Y + (long long)sg.inst * d.n3;
    for (int e = sg.begin + threadIdx.x; e < sg.end; e += blockDim.x) v[off[sg.inst] + e] = e < d.n3 ? y[e] : 0.f;
}

// dY = scale (C res) / alpha on the unknown grid nodes, 0 elsewhere
__global__ void k_unet_dy(const Seg* __restrict__ seg, const InstDesc* __restrict__ D, const long long* __restrict__ off,
                          const float* __restrict__ cres, float scale, float* __restrict__ dY) {
    const Seg sg = seg[blockIdx.x];
    const InstDesc& d = D[sg.inst];
    float* g = dY + (long long)sg.inst * d.n3;
    for (int e = sg.begin + threadIdx.x; e < sg.end; e += blockDim.x)
        g[e] = (d.natural || !is_bd(e, d.N)) ? scale * cres[off[sg.inst] + e] / (float)d.alpha : 0.f;
}

extern "C" md_status md_unet_train_loss(md_unet* u, int count, const md_op* const* ops, const float* const* r,
                                        double* loss, float* dparams, md_stream stream) {
    if (!u || !loss) { md_set_error("md_unet_train_loss: NULL argument"); return MD_ERR_ARG; }
    MD_TRY(check_samples(count, ops, r));
    const int N = ops[0]->h.N;
    int max_n1 = 0, max_nq = 0, max_t = 0;
    for (int i = 0; i < count; ++i) {
        if (ops[i]->h.N != N) { md_set_error("md_unet_train_loss: samples of one call share the grid size"); return MD_ERR_ARG; }
        max_n1 = std::max(max_n1, ops[i]->h.n1);
        max_nq = std::max(max_nq, ops[i]->h.nq);
        max_t = std::max(max_t, ops[i]->h.ntouch);
    }
    if (N + 1 < 4) { md_set_error("md_unet_train_loss: grids of at least 4^3 nodes"); return MD_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    TrainWork* t = nullptr;
    MD_TRY(train_work_create(count, N, max_n1, max_nq, max_t, &t));
    const int B = count;
    const long long n3 = (long long)(N + 1) * (N + 1) * (N + 1);
    std::vector<InstDesc> desc(B);
    std::vector<const InstDesc*> ptrs(B);
    for (int i = 0; i < B; ++i) {
        desc[i] = ops[i]->h;
        desc[i].t32 = t->scratch[3 * i];
        desc[i].lift32 = t->scratch[3 * i + 1];
        desc[i].ltouch32 = t->scratch[3 * i + 2];
        ptrs[i] = &desc[i];
    }
    std::vector<void*> tmp;
    float *X = nullptr, *Y = nullptr, *dY = nullptr;
    Tables T;
    md_status st = build_tables(ptrs, &T, &tmp);
    if (st == MD_OK) st = dev_alloc(&tmp, &X, (size_t)(2 * n3 * B), false);
    if (st == MD_OK) st = dev_alloc(&tmp, &Y, (size_t)(n3 * B), false);
    if (st == MD_OK) st = dev_alloc(&tmp, &dY, (size_t)(n3 * B), false);
    auto run = [&]() -> md_status {
        MD_CUDA(cudaMemcpyAsync(t->d, desc.data(), sizeof(InstDesc) * B, cudaMemcpyHostToDevice, s));
        for (int i = 0; i < B; ++i) {
            MD_CUDA(cudaMemsetAsync(desc[i].lift32, 0, sizeof(float) * desc[i].n3, s));
            MD_CUDA(cudaMemcpyAsync(t->rv + i * t->stride, r[i], sizeof(float) * desc[i].n, cudaMemcpyDeviceToDevice, s));
        }
        MD_CUDA(cudaMemsetAsync(t->loss, 0, sizeof(double) * B, s));
        k_mask_grid<<<T.vec.nblocks, MD_TB, 0, s>>>(T.vec.seg, t->d, t->voff, t->rv, 0);
        k_set_active<<<(B + 31) / 32, 32, 0, s>>>(t->st, B);
        MD_CHECK_LAUNCH();
        // ||r0||, the 1D solve and its lift l, s = ||r0 + l||
        MD_TRY(launch_prec_input(T, t->d, t->voff, t->rv, t->yv, t->st, B, t->max_n1, t->part3, s));
        k_unet_pack<<<T.n3.nblocks, MD_TB, 0, s>>>(T.n3.seg, t->d, t->voff, t->rv, t->st, X);
        MD_CHECK_LAUNCH();
        MD_TRY(md_unet_forward(u, N + 1, B, X, Y, (md_stream)s));
        k_unet_scatter<<<T.vec.nblocks, MD_TB, 0, s>>>(T.vec.seg, t->d, t->voff, Y, t->yv);
        k_mask_grid<<<T.vec.nblocks, MD_TB, 0, s>>>(T.vec.seg, t->d, t->voff, t->yv, 1);
        MD_CHECK_LAUNCH();
        MD_TRY(launch_apply(T, t->d, B, MD_FP32, t->yv, t->voff, t->cy, s));
        k_train_res<<<T.vec.nblocks, MD_TB, 0, s>>>(T.vec.seg, t->d, t->voff, t->cy, t->rv, t->st, t->res, t->loss);
        MD_CHECK_LAUNCH();
        MD_TRY(launch_apply(T, t->d, B, MD_FP32, t->res, t->voff, t->cres, s));
        k_unet_dy<<<T.n3.nblocks, MD_TB, 0, s>>>(T.n3.seg, t->d, t->voff, t->cres, 2.0f / B, dY);
        MD_CHECK_LAUNCH();
        if (dparams) MD_TRY(md_unet_backward(u, N + 1, B, X, dY, dparams, nullptr, (md_stream)s));
        std::vector<double> l(B);
        MD_CUDA(cudaMemcpyAsync(l.data(), t->loss, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
        MD_CUDA(cudaStreamSynchronize(s));
        *loss = std::accumulate(l.begin(), l.end(), 0.0) / B;
        return MD_OK;
    };
    if (st == MD_OK) st = run();
    dev_free_all(&tmp);
    train_work_destroy(t);
    return st;
}

extern "C" md_status md_train(md_cnn* c, const md_train_cfg* cfg) {
    if (!c || !cfg) { md_set_error("md_train: NULL argument"); return MD_ERR_ARG; }
    if (cfg->n_ops < 1 || !cfg->ops || cfg->n_samples < 1 || !cfg->sample_op || !cfg->sample_r || cfg->epochs < 1 ||
        cfg->batch < 1) {
        md_set_error("md_train: bad configuration"); return MD_ERR_ARG;
    }
    for (int i = 0; i < cfg->n_samples; ++i)
        if (cfg->sample_op[i] < 0 || cfg->sample_op[i] >= cfg->n_ops || !cfg->ops[cfg->sample_op[i]] || !cfg->sample_r[i]) {
            md_set_error("md_train: sample %d is invalid", i); return MD_ERR_ARG;
        }
    // group samples by grid size
    std::vector<int> Ns;
    for (int i = 0; i < cfg->n_ops; ++i) Ns.push_back(cfg->ops[i]->h.N);
    std::sort(Ns.begin(), Ns.end());
    Ns.erase(std::unique(Ns.begin(), Ns.end()), Ns.end());
    std::vector<std::vector<int>> groups(Ns.size());
    for (int i = 0; i < cfg->n_samples; ++i) {
        const int N = cfg->ops[cfg->sample_op[i]]->h.N;
        groups[std::lower_bound(Ns.begin(), Ns.end(), N) - Ns.begin()].push_back(i);
    }
    int max_n1 = 0, max_nq = 0, max_t = 0;
    for (int i = 0; i < cfg->n_ops; ++i) {
        max_n1 = std::max(max_n1, cfg->ops[i]->h.n1);
        max_nq = std::max(max_nq, cfg->ops[i]->h.nq);
        max_t = std::max(max_t, cfg->ops[i]->h.ntouch);
    }
    const int B = cfg->batch;
    std::vector<TrainWork*> works(Ns.size(), nullptr);
    md_status st = MD_OK;
    for (size_t gi = 0; gi < Ns.size() && st == MD_OK; ++gi)
        st = train_work_create(B, Ns[gi], max_n1, max_nq, max_t, &works[gi]);
    // optimizer state (device) and master weights
    std::vector<void*> opt;
    float *w = nullptr, *m = nullptr, *v = nullptr;
    unsigned char* isw = nullptr;
    std::vector<unsigned char> hisw(MD_CNN_NPARAMS, 0);
    for (int l = 0; l < MD_CNN_LAYERS; ++l)
        for (size_t k = 0; k < (size_t)kCout[l] * kCin[l] * 27; ++k) hisw[host_w_off(l) + k] = 1;
    if (st == MD_OK) st = dev_upload(&opt, &w, c->host.data(), c->host.size());
    if (st == MD_OK) st = dev_alloc(&opt, &m, (size_t)MD_CNN_NPARAMS);
    if (st == MD_OK) st = dev_alloc(&opt, &v, (size_t)MD_CNN_NPARAMS);
    if (st == MD_OK) st = dev_upload(&opt, &isw, hisw.data(), hisw.size());
    cudaStream_t s = nullptr;
    if (st == MD_OK) {
        cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e != cudaSuccess) st = md_cuda_status(e, "cudaStreamCreate", __FILE__, __LINE__);
    }
    std::mt19937_64 rng(cfg->seed);
    // steps per epoch: full minibatches of each group
    long long steps_per_epoch = 0;
    for (auto& g : groups) steps_per_epoch += (long long)g.size() / B;
    if (st == MD_OK && steps_per_epoch == 0) { md_set_error("md_train: fewer samples than one minibatch"); st = MD_ERR_ARG; }
    const long long total_steps = steps_per_epoch * cfg->epochs;
    long long step = 0;
    std::vector<float> hw(MD_CNN_NPARAMS);
    for (int ep = 0; ep < cfg->epochs && st == MD_OK; ++ep) {
        // batches: shuffle within groups, then interleave the groups' batches
        std::vector<std::pair<int, std::vector<int>>> batches;
        for (size_t gi = 0; gi < groups.size(); ++gi) {
            std::vector<int> idx = groups[gi];
            std::shuffle(idx.begin(), idx.end(), rng);
            for (size_t b0 = 0; b0 + B <= idx.size(); b0 += B)
                batches.push_back({(int)gi, std::vector<int>(idx.begin() + b0, idx.begin() + b0 + B)});
        }
        std::shuffle(batches.begin(), batches.end(), rng);
        double ep_loss = 0.0;
        long long ep_n = 0;
        for (auto& bt : batches) {
            std::vector<const md_op*> bo;
            std::vector<const float*> br;
            for (int i : bt.second) {
                bo.push_back(cfg->ops[cfg->sample_op[i]]);
                br.push_back(cfg->sample_r[i]);
            }
            double L = 0.0;
            st = minibatch(c, works[bt.first], bo, br, &L, s);
            if (st != MD_OK) break;
            if (!std::isfinite(L)) { md_set_error("md_train: loss is not finite at step %lld", step); st = MD_ERR_NAN; break; }
            ep_loss += L;
            ep_n += B;
            // cosine learning rate from lr to lr_min over all steps
            const double frac = total_steps > 1 ? (double)step / (double)(total_steps - 1) : 1.0;
            const double lr = cfg->lr_min + 0.5 * (cfg->lr - cfg->lr_min) * (1.0 + std::cos(M_PI * frac));
            ++step;
            const float bc1 = (float)(1.0 - std::pow(cfg->beta1, (double)step));
            const float bc2 = (float)(1.0 - std::pow(cfg->beta2, (double)step));
            k_adamw<<<128, 256, 0, s>>>(w, works[bt.first]->grad, m, v, isw, MD_CNN_NPARAMS, (float)lr, (float)cfg->beta1,
                                        (float)cfg->beta2, (float)cfg->eps, (float)cfg->weight_decay, bc1, bc2);
            cudaError_t e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaMemcpyAsync(hw.data(), w, sizeof(float) * MD_CNN_NPARAMS, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) { st = md_cuda_status(e, "md_train step", __FILE__, __LINE__); break; }
            c->host = hw;
            st = cnn_upload(c);
            if (st != MD_OK) break;
        }
        if (st == MD_OK && cfg->loss_history) cfg->loss_history[ep] = ep_n ? ep_loss / ep_n : 0.0;
    }
    if (s) cudaStreamDestroy(s);
    for (auto* t : works) train_work_destroy(t);
    dev_free_all(&opt);
    return st;
}

// ---- optimizer state for training loops driven from outside (data-parallel
// training: each process computes its gradient with md_train_loss, the
// processes average them, and every process applies the same step)
struct md_opt {
    std::vector<void*> allocs;
    float *w = nullptr, *m = nullptr, *v = nullptr;  // FP32 master weights, AdamW moments
    unsigned char* isw = nullptr;                    // weight (1) or bias (0): decay on weights only
    long long step = 0;
};

extern "C" void md_opt_destroy(md_opt* o) {
    if (!o) return;
    dev_free_all(&o->allocs);
    delete o;
}

extern "C" md_status md_opt_create(const md_cnn* c, md_opt** out) {
    if (!c || !out) { md_set_error("md_opt_create: NULL argument"); return MD_ERR_ARG; }
    *out = nullptr;
    md_opt* o = new md_opt();
    std::vector<unsigned char> hisw(MD_CNN_NPARAMS, 0);
    for (int l = 0; l < MD_CNN_LAYERS; ++l)
        for (size_t k = 0; k < (size_t)kCout[l] * kCin[l] * 27; ++k) hisw[host_w_off(l) + k] = 1;
    md_status st = dev_upload(&o->allocs, &o->w, c->host.data(), c->host.size());
    if (st == MD_OK) st = dev_alloc(&o->allocs, &o->m, (size_t)MD_CNN_NPARAMS);
    if (st == MD_OK) st = dev_alloc(&o->allocs, &o->v, (size_t)MD_CNN_NPARAMS);
    if (st == MD_OK) st = dev_upload(&o->allocs, &o->isw, hisw.data(), hisw.size());
    if (st != MD_OK) { md_opt_destroy(o); return st; }
    *out = o;
    return MD_OK;
}

extern "C" md_status md_opt_step(md_opt* o, md_cnn* c, const float* grad, double lr, double beta1, double beta2,
                                 double eps, double weight_decay, md_stream stream) {
    if (!o || !c || !grad) { md_set_error("md_opt_step: NULL argument"); return MD_ERR_ARG; }
    if (!(lr >= 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0)) {
        md_set_error("md_opt_step: bad hyper-parameters");
        return MD_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    o->step += 1;
    const float bc1 = (float)(1.0 - std::pow(beta1, (double)o->step));
    const float bc2 = (float)(1.0 - std::pow(beta2, (double)o->step));
    k_adamw<<<128, 256, 0, s>>>(o->w, grad, o->m, o->v, o->isw, MD_CNN_NPARAMS, (float)lr, (float)beta1, (float)beta2,
                                (float)eps, (float)weight_decay, bc1, bc2);
    MD_CHECK_LAUNCH();
    std::vector<float> hw(MD_CNN_NPARAMS);
    MD_CUDA(cudaMemcpyAsync(hw.data(), o->w, sizeof(float) * MD_CNN_NPARAMS, cudaMemcpyDeviceToHost, s));
    MD_CUDA(cudaStreamSynchronize(s));
    for (float x : hw)
        if (!std::isfinite(x)) { md_set_error("md_opt_step: a weight is not finite"); return MD_ERR_NAN; }
    c->host = hw;
    return cnn_upload(c);
}

// ---- the Krylov augmentation of the training set (Section 4.1.1) -----------------
// An orthonormal basis q_0 = b/||b||, q_1, ..., q_m of the Krylov space of the
// 3D block C started at b: q_{j+1} = C q_j orthogonalised against q_0..q_j by
// modified Gram-Schmidt, twice, and normalised; FP64 throughout.  C q is the
// 3D part of the operator apply with the 1D part of the input zero.  Sums are
// per block, then added in block order by every block that needs them.
#define KB_TB 256
#define KB_BLOCKS 120

__global__ void __launch_bounds__(KB_TB) k_kb_dot(const double* __restrict__ a, const double* __restrict__ b, int n,
                                                  double* part) {
    __shared__ double sh[KB_TB / 32];
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) acc += a[i] * b[i];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < KB_TB / 32; ++w) s += sh[w];
        part[blockIdx.x] = s;
    }
}

__device__ inline double kb_sum(const double* part, int nparts) {
    double s = 0.0;
    for (int k = 0; k < nparts; ++k) s += part[k];
    return s;
}

// w -= (q, w) q, with (q, w) from the partials of k_kb_dot
__global__ void __launch_bounds__(KB_TB) k_kb_axpy(const double* __restrict__ q, double* w, int n,
                                                   const double* __restrict__ part, int nparts) {
    const double c = kb_sum(part, nparts);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) w[i] -= c * q[i];
}

// q = w / ||w|| (||w||^2 from the partials); the 1D part of u is left zero
__global__ void __launch_bounds__(KB_TB) k_kb_scale(const double* __restrict__ w, double* q, int n,
                                                    const double* __restrict__ part, int nparts) {
    const double s = kb_sum(part, nparts);
    const double inv = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) q[i] = w[i] * inv;
}

__global__ void k_kb_cast_in(const float* __restrict__ b, double* w, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) w[i] = (double)b[i];
}
__global__ void k_kb_cast_out(const double* __restrict__ q, float* out, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = (float)q[i];
}

extern "C" md_status md_krylov_basis(const md_op* op, const float* b, int m, float* Q, md_stream stream) {
    if (!op || !b || !Q) { md_set_error("md_krylov_basis: NULL argument"); return MD_ERR_ARG; }
    if (m < 1 || m > 16) { md_set_error("md_krylov_basis: m = %d outside [1, 16]", m); return MD_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    const int n3 = op->h.n3;
    const long long n = op->h.n;
    std::vector<void*> tmp;
    double *q = nullptr, *u = nullptr, *w = nullptr, *part = nullptr;
    md_status st = dev_alloc(&tmp, &q, (size_t)(m + 1) * n3);
    if (st == MD_OK) st = dev_alloc(&tmp, &u, (size_t)n);  // [q_j ; 0]
    if (st == MD_OK) st = dev_alloc(&tmp, &w, (size_t)n);
    if (st == MD_OK) st = dev_alloc(&tmp, &part, (size_t)KB_BLOCKS);
    auto run = [&]() -> md_status {
        // q_0 = b / ||b||
        k_kb_cast_in<<<KB_BLOCKS, KB_TB, 0, s>>>(b, w, n3);
        k_kb_dot<<<KB_BLOCKS, KB_TB, 0, s>>>(w, w, n3, part);
        k_kb_scale<<<KB_BLOCKS, KB_TB, 0, s>>>(w, q, n3, part, KB_BLOCKS);
        MD_CHECK_LAUNCH();
        for (int j = 0; j < m; ++j) {
            MD_CUDA(cudaMemcpyAsync(u, q + (size_t)j * n3, sizeof(double) * n3, cudaMemcpyDeviceToDevice, s));
            MD_TRY(md_apply(op, MD_FP64, u, w, s));
            for (int pass = 0; pass < 2; ++pass)
                for (int i = 0; i <= j; ++i) {
                    const double* qi = q + (size_t)i * n3;
                    k_kb_dot<<<KB_BLOCKS, KB_TB, 0, s>>>(qi, w, n3, part);
                    k_kb_axpy<<<KB_BLOCKS, KB_TB, 0, s>>>(qi, w, n3, part, KB_BLOCKS);
                }
            k_kb_dot<<<KB_BLOCKS, KB_TB, 0, s>>>(w, w, n3, part);
            k_kb_scale<<<KB_BLOCKS, KB_TB, 0, s>>>(w, q + (size_t)(j + 1) * n3, n3, part, KB_BLOCKS);
            MD_CHECK_LAUNCH();
        }
        k_kb_cast_out<<<KB_BLOCKS, KB_TB, 0, s>>>(q, Q, (int)((m + 1) * (long long)n3));
        MD_CHECK_LAUNCH();
        MD_CUDA(cudaStreamSynchronize(s));
        return MD_OK;
    };
    if (st == MD_OK) st = run();
    dev_free_all(&tmp);
    return st;
}
