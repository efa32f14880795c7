// The preconditioner network: parameter storage, input packing and the
// convolution layers on CUDA cores (the reference path of the network and
// the one training uses for its backward pass).
//
// Layer l computes Y = b + sum_q W(q) X(p + q) over q in {-1,0,1}^3 with zero
// 'same' padding (the convolution of Section 4.2 in cross-correlation
// orientation), then GELU(x) = x Phi(x) for l < 5.  Weights and hidden
// activations are BF16, accumulation FP32.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <type_traits>

#include "md_cnn.h"
#include "md_common.cuh"
#include "md_conv_tc.h"

namespace {
const int kCin[MD_CNN_LAYERS] = {3, 32, 32, 32, 32, 32};
const int kCout[MD_CNN_LAYERS] = {32, 32, 32, 32, 32, 1};
const int kCinPad[MD_CNN_LAYERS] = {8, 32, 32, 32, 32, 32};

size_t host_w_off(int l) {
    size_t o = 0;
    for (int i = 0; i < l; ++i) o += (size_t)kCout[i] * kCin[i] * 27 + kCout[i];
    return o;
}

uint64_t fnv1a(const void* p, size_t n) {
    const unsigned char* c = (const unsigned char*)p;
    uint64_t h = 1469598103934665603ULL;
    for (size_t i = 0; i < n; ++i) { h ^= c[i]; h *= 1099511628211ULL; }
    return h;
}
}  // namespace

// ---- parameters --------------------------------------------------------------
unsigned long long md_next_cnn_uid() {
    static std::atomic<unsigned long long> next{1};
    return next.fetch_add(1);
}

md_status cnn_upload(md_cnn* c) {
    // packed weights per layer: [tap][cin_pad][cout] BF16 (RN), biases FP32
    std::vector<__nv_bfloat16> w;
    std::vector<float> b;
    for (int l = 0; l < MD_CNN_LAYERS; ++l) {
        c->w_off[l] = w.size();
        c->b_off[l] = b.size();
        const float* W = c->host.data() + host_w_off(l);
        const float* B = W + (size_t)kCout[l] * kCin[l] * 27;
        for (int tap = 0; tap < 27; ++tap)
            for (int ci = 0; ci < kCinPad[l]; ++ci)
                for (int co = 0; co < kCout[l]; ++co) {
                    float v = ci < kCin[l] ? W[((size_t)co * kCin[l] + ci) * 27 + tap] : 0.0f;
                    w.push_back(__float2bfloat16_rn(v));
                }
        for (int co = 0; co < kCout[l]; ++co) b.push_back(B[co]);
    }
    c->w_off[MD_CNN_LAYERS] = w.size();
    c->b_off[MD_CNN_LAYERS] = b.size();
    // tensor-core operand images: first layer kind 1, hidden kind 0, last kind 2
    std::vector<__nv_bfloat16> img, all;
    for (int l = 0; l < MD_CNN_LAYERS; ++l) {
        const int kind = l == 0 ? 1 : (l == MD_CNN_LAYERS - 1 ? 2 : 0);
        tc_weight_image(kind, c->host.data() + host_w_off(l), kCin[l], kCout[l], img);
        c->wmma_off[l] = all.size();
        all.insert(all.end(), img.begin(), img.end());
    }
    c->wmma_off[MD_CNN_LAYERS] = all.size();
    // input-gradient (transposed, flipped) weights of every layer:
    // Wt[tap'][c_out padded to >= 8][c_in padded to >= 8] = W[c_out][c_in][26 - tap']
    std::vector<__nv_bfloat16> wt;
    for (int l = 0; l < MD_CNN_LAYERS; ++l) {
        c->wt_off[l] = wt.size();
        const float* W = c->host.data() + host_w_off(l);
        const int cop = kCout[l] < 8 ? 8 : kCout[l], cip = kCin[l] < 8 ? 8 : kCin[l];
        for (int tp = 0; tp < 27; ++tp)
            for (int co = 0; co < cop; ++co)
                for (int ci = 0; ci < cip; ++ci) {
                    float v = (co < kCout[l] && ci < kCin[l]) ? W[((size_t)co * kCin[l] + ci) * 27 + (26 - tp)] : 0.0f;
                    wt.push_back(__float2bfloat16_rn(v));
                }
    }
    c->wt_off[MD_CNN_LAYERS] = wt.size();
    // tensor-core images of the adjoint convolutions of layers 1-5: weights
    // W'[o'][c'][tap] = W[c'][o'][26 - tap] (flipped and transposed); the last
    // layer's adjoint has one input channel (kind 1, as the first layer)
    std::vector<__nv_bfloat16> allt;
    c->wtmma_off[0] = 0;
    for (int l = 1; l < MD_CNN_LAYERS; ++l) {
        const int ci = kCin[l], co = kCout[l];  // forward: ci -> co; adjoint: co -> ci
        const float* W = c->host.data() + host_w_off(l);
        std::vector<float> Wa((size_t)ci * co * 27);
        for (int o2 = 0; o2 < ci; ++o2)
            for (int c2 = 0; c2 < co; ++c2)
                for (int tap = 0; tap < 27; ++tap)
                    Wa[((size_t)o2 * co + c2) * 27 + tap] = W[((size_t)c2 * ci + o2) * 27 + (26 - tap)];
        tc_weight_image(l == MD_CNN_LAYERS - 1 ? 1 : 0, Wa.data(), co, ci, img);
        c->wtmma_off[l] = allt.size();
        allt.insert(allt.end(), img.begin(), img.end());
    }
    c->wtmma_off[MD_CNN_LAYERS] = allt.size();
    // device buffers keep their size, so a network updated in place (training)
    // reuses its allocations
    auto put = [](auto** dst, const auto& v) -> md_status {
        using T = typename std::remove_reference<decltype(v)>::type::value_type;
        if (!*dst) {
            std::vector<void*> tmp;
            return dev_upload(&tmp, (T**)dst, v.data(), v.size());
        }
        MD_CUDA(cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
        return MD_OK;
    };
    MD_TRY(put(&c->w, w));
    MD_TRY(put(&c->b, b));
    MD_TRY(put(&c->wmma, all));
    MD_TRY(put(&c->wt, wt));
    MD_TRY(put(&c->wtmma, allt));
    return MD_OK;
}

extern "C" md_status md_cnn_set_engine(md_cnn* c, int engine) {
    if (!c || (engine != 0 && engine != 1)) { md_set_error("md_cnn_set_engine: bad argument"); return MD_ERR_ARG; }
    c->engine = engine;
    return MD_OK;
}

extern "C" md_status md_cnn_create(const float* host_params, long long n_params, md_cnn** out) {
    if (!out || !host_params) { md_set_error("md_cnn_create: NULL argument"); return MD_ERR_ARG; }
    *out = nullptr;
    if (n_params != MD_CNN_NPARAMS) { md_set_error("md_cnn_create: %lld parameters, expected %d", n_params, MD_CNN_NPARAMS); return MD_ERR_ARG; }
    for (long long i = 0; i < n_params; ++i)
        if (!std::isfinite(host_params[i])) { md_set_error("md_cnn_create: parameter %lld is not finite", i); return MD_ERR_NAN; }
    md_cnn* c = new md_cnn();
    c->host.assign(host_params, host_params + n_params);
    md_status st = cnn_upload(c);
    if (st != MD_OK) { md_cnn_destroy(c); return st; }
    *out = c;
    return MD_OK;
}

md_status cnn_set_params(md_cnn* c, const float* host_params) {
    c->host.assign(host_params, host_params + MD_CNN_NPARAMS);
    return cnn_upload(c);
}

extern "C" md_status md_cnn_get_params(const md_cnn* c, float* host_params, long long n_params) {
    if (!c || !host_params || n_params != MD_CNN_NPARAMS) { md_set_error("md_cnn_get_params: bad argument"); return MD_ERR_ARG; }
    memcpy(host_params, c->host.data(), sizeof(float) * MD_CNN_NPARAMS);
    return MD_OK;
}

extern "C" void md_cnn_destroy(md_cnn* c) {
    if (!c) return;
    if (c->w) cudaFree(c->w);
    if (c->b) cudaFree(c->b);
    if (c->wmma) cudaFree(c->wmma);
    if (c->wt) cudaFree(c->wt);
    if (c->wtmma) cudaFree(c->wtmma);
    delete c;
}

extern "C" md_status md_cnn_save(const md_cnn* c, const char* path) {
    if (!c || !path) { md_set_error("md_cnn_save: NULL argument"); return MD_ERR_ARG; }
    FILE* f = fopen(path, "wb");
    if (!f) { md_set_error("md_cnn_save: cannot open %s", path); return MD_ERR_IO; }
    const char magic[8] = {'M', 'D', 'C', 'N', 'N', '0', '0', '1'};
    int64_t n = MD_CNN_NPARAMS;
    uint64_t h = fnv1a(c->host.data(), sizeof(float) * n);
    bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(&n, 8, 1, f) == 1 &&
              fwrite(c->host.data(), sizeof(float), n, f) == (size_t)n && fwrite(&h, 8, 1, f) == 1;
    ok = (fclose(f) == 0) && ok;
    if (!ok) { md_set_error("md_cnn_save: write failed for %s", path); return MD_ERR_IO; }
    return MD_OK;
}

extern "C" md_status md_cnn_load(const char* path, md_cnn** out) {
    if (!path || !out) { md_set_error("md_cnn_load: NULL argument"); return MD_ERR_ARG; }
    *out = nullptr;
    FILE* f = fopen(path, "rb");
    if (!f) { md_set_error("md_cnn_load: cannot open %s", path); return MD_ERR_IO; }
    char magic[8];
    int64_t n = 0;
    uint64_t h = 0;
    std::vector<float> v;
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "MDCNN001", 8) == 0 && fread(&n, 8, 1, f) == 1 &&
              n == MD_CNN_NPARAMS;
    if (ok) {
        v.resize(n);
        ok = fread(v.data(), sizeof(float), n, f) == (size_t)n && fread(&h, 8, 1, f) == 1;
    }
    fclose(f);
    if (!ok) { md_set_error("md_cnn_load: %s is not a network file of %d parameters", path, MD_CNN_NPARAMS); return MD_ERR_IO; }
    if (fnv1a(v.data(), sizeof(float) * n) != h) { md_set_error("md_cnn_load: checksum mismatch in %s", path); return MD_ERR_IO; }
    return md_cnn_create(v.data(), n, out);
}

// ---- workspace -----------------------------------------------------------------
template <int CIN8, int COUT, bool LAST>
__global__ void k_conv_simt(const __nv_bfloat16* __restrict__, const long long* __restrict__, __nv_bfloat16* __restrict__,
                            const long long* __restrict__, const __nv_bfloat16* __restrict__, const float* __restrict__,
                            const Seg* __restrict__, const int* __restrict__, OutIO, int, __nv_bfloat16* __restrict__);

// Kernel attributes are set once, outside any stream capture.
static md_status cnn_prepare() {
    static bool done = false;
    if (done) return MD_OK;
    MD_CUDA(cudaFuncSetAttribute(k_conv_simt<1, 32, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 27 * 8 * 32 * 2));
    MD_CUDA(cudaFuncSetAttribute(k_conv_simt<4, 32, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 27 * 32 * 32 * 2));
    MD_CUDA(cudaFuncSetAttribute(k_conv_simt<4, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 27 * 32 * 1 * 2));
    done = true;
    return MD_OK;
}

md_status cnn_work_create(const std::vector<int>& Ns, CnnWork** out) {
    MD_TRY(cnn_prepare());
    CnnWork* w = new CnnWork();
    w->ninst = (int)Ns.size();
    w->hN = Ns;
    long long rx = CNN_MARGIN_ROWS, rab = CNN_MARGIN_ROWS, nodes = 0;
    std::vector<Seg> segs;
    std::vector<InstRange> ranges;
    int pd_max = 0;
    for (int n : Ns) pd_max = std::max(pd_max, n + 3);
    w->pd_max = pd_max;
    w->tps = 2;
    w->W = tc_window_rows(w->tps, pd_max);
    w->NS = tc_ring_slots(w->W);
    if (w->NS == 0) { delete w; md_set_error("grid too large for the tensor-core convolution windows"); return MD_ERR_ARG; }
    {
        int dev = 0, nsm = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && nsm > 0)
            w->nsm = nsm;
    }
    // per instance: columns of tps*126 in-plane rows, each walked over the N+1
    // padded planes [1, N+2) that hold grid nodes (the step order TcSched
    // describes); the schedule of a pass over every instance
    std::vector<long long> steps_i, all_pre;
    std::vector<int> all_inst;
    long long steps = 0;
    const int CH = 512;
    all_pre.push_back(0);
    for (int i = 0; i < w->ninst; ++i) {
        long long Pd = Ns[i] + 3, P = Pd * Pd * Pd;
        if (Pd + 1 + 256 + 8 > CNN_MARGIN_ROWS) { delete w; md_set_error("grid too large for the network workspace"); return MD_ERR_ARG; }
        w->h_off_x0.push_back(rx * 8);
        w->h_off_ab.push_back(rab * 8);
        rx += P;
        rab += 4 * P;
        int n3 = (Ns[i] + 1) * (Ns[i] + 1) * (Ns[i] + 1);
        nodes += n3;
        ranges.push_back({(int)segs.size(), 0});
        for (int b = 0; b < n3; b += CH) segs.push_back({i, 0, b, std::min(n3, b + CH)});
        ranges.back().count = (int)segs.size() - ranges.back().first;
        const long long cols = (Pd * Pd + 126LL * w->tps - 1) / (126LL * w->tps);
        steps_i.push_back(cols * (Ns[i] + 1));
        steps += steps_i.back();
        all_inst.push_back(i);
        all_pre.push_back(steps);
    }
    w->ngroups = (int)std::max(1LL, std::min<long long>(w->nsm, steps));
    rx += CNN_MARGIN_ROWS;
    rab += CNN_MARGIN_ROWS;
    w->total_nodes = nodes;
    md_status st = MD_OK;
    auto chk = [&](md_status s) { if (st == MD_OK) st = s; };
    chk(tc_prepare(w->W, w->tps));
    chk(dev_upload(&w->allocs, &w->N, Ns.data(), Ns.size()));
    chk(dev_upload(&w->allocs, &w->steps, steps_i.data(), steps_i.size()));
    chk(dev_upload(&w->allocs, &w->all_inst, all_inst.data(), all_inst.size()));
    chk(dev_upload(&w->allocs, &w->all_pre, all_pre.data(), all_pre.size()));
    chk(dev_upload(&w->allocs, &w->all_count, &w->ninst, 1));
    chk(dev_alloc(&w->allocs, &w->run_inst, (size_t)w->ninst));
    chk(dev_alloc(&w->allocs, &w->run_pre, (size_t)w->ninst + 1));
    chk(dev_alloc(&w->allocs, &w->run_count, 1));
    chk(dev_alloc(&w->allocs, &w->err, 1));
    chk(dev_upload(&w->allocs, &w->off_x0, w->h_off_x0.data(), w->h_off_x0.size()));
    chk(dev_upload(&w->allocs, &w->off_ab, w->h_off_ab.data(), w->h_off_ab.size()));
    chk(dev_alloc(&w->allocs, &w->x0, (size_t)rx * 8));
    chk(dev_alloc(&w->allocs, &w->a, (size_t)rab * 8));
    chk(dev_alloc(&w->allocs, &w->b, (size_t)rab * 8));
    w->nodes.nblocks = (int)segs.size();
    w->nodes.hrange = ranges;
    chk(dev_upload(&w->allocs, &w->nodes.seg, segs.data(), segs.size()));
    chk(dev_upload(&w->allocs, &w->nodes.range, ranges.data(), ranges.size()));
    if (st != MD_OK) { cnn_work_destroy(w); return st; }
    *out = w;
    return MD_OK;
}

// The plane steps of every instance for `tps` tiles per plane step (columns
// of tps*126 in-plane rows, each walked over the N+1 planes with grid nodes).
static void tc_steps(const std::vector<int>& Ns, int tps, std::vector<long long>& steps_i, std::vector<long long>& pre) {
    steps_i.clear();
    pre.assign(1, 0);
    for (int n : Ns) {
        const long long Pd = n + 3;
        const long long cols = (Pd * Pd + 126LL * tps - 1) / (126LL * tps);
        steps_i.push_back(cols * (n + 1));
        pre.push_back(pre.back() + steps_i.back());
    }
}

md_status cnn_work_set_tps(CnnWork* w, int tps) {
    if (tps != 1 && tps != 2) { md_set_error("tiles per plane step must be 1 or 2"); return MD_ERR_ARG; }
    const int W = tc_window_rows(tps, w->pd_max), NS = tc_ring_slots(W);
    if (NS == 0) { md_set_error("grid too large for the tensor-core convolution windows"); return MD_ERR_ARG; }
    std::vector<long long> steps_i, pre;
    tc_steps(w->hN, tps, steps_i, pre);
    MD_TRY(tc_prepare(W, tps));
    MD_CUDA(cudaMemcpy(w->steps, steps_i.data(), sizeof(long long) * steps_i.size(), cudaMemcpyHostToDevice));
    MD_CUDA(cudaMemcpy(w->all_pre, pre.data(), sizeof(long long) * pre.size(), cudaMemcpyHostToDevice));
    w->tps = tps;
    w->W = W;
    w->NS = NS;
    w->ngroups = (int)std::max(1LL, std::min<long long>(w->nsm, pre.back()));
    return MD_OK;
}

// Autotuning of the tiles per plane step: a forward pass of the network over
// every grid of the workspace (raw output into `out` at `off`) timed with
// each choice; the faster one is kept.  us[0], us[1]: microseconds per pass
// with 1 and 2 tiles per step.
md_status cnn_autotune_tps(const md_cnn* c, CnnWork* w, float* out, const long long* off, double* us) {
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    MD_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    md_status st = MD_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = MD_ERR_CUDA;
    OutIO io{out, off, nullptr, nullptr, nullptr, nullptr};
    int best = 2;
    double best_us = 1e300;
    for (int tps = 2; tps >= 1 && st == MD_OK; --tps) {
        st = cnn_work_set_tps(w, tps);
        if (st != MD_OK) { us[tps - 1] = -1.0; st = MD_OK; (void)cudaGetLastError(); continue; }
        st = cnn_forward_layers(c, w, io, CONV_RAW, s);
        if (st == MD_OK && cudaEventRecord(e0, s) != cudaSuccess) st = MD_ERR_CUDA;
        for (int r = 0; r < 2 && st == MD_OK; ++r) st = cnn_forward_layers(c, w, io, CONV_RAW, s);
        if (st == MD_OK && cudaEventRecord(e1, s) != cudaSuccess) st = MD_ERR_CUDA;
        float ms = 0.f;
        if (st == MD_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            st = MD_ERR_CUDA;
        if (st != MD_OK) break;
        us[tps - 1] = 1e3 * ms / 2;
        if (us[tps - 1] < best_us) { best_us = us[tps - 1]; best = tps; }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    int err = 0;
    if (st == MD_OK && cudaMemcpy(&err, w->err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && err) {
        md_set_error("a convolution timed out while tuning");
        st = MD_ERR_TIMEOUT;
    }
    if (st != MD_OK) return st == MD_ERR_CUDA ? md_cuda_status(cudaGetLastError(), "conv autotune", __FILE__, __LINE__) : st;
    return cnn_work_set_tps(w, best);
}

void cnn_work_destroy(CnnWork* w) {
    if (!w) return;
    dev_free_all(&w->allocs);
    delete w;
}

// ---- kernels ---------------------------------------------------------------------

__device__ inline void unpack8(const uint4& r, float (&x)[8]) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&r);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float2 f = __bfloat1622float2(h[k]);
        x[2 * k] = f.x;
        x[2 * k + 1] = f.y;
    }
}

__device__ inline uint4 pack8(const float* v) {
    uint4 r;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&r);
#pragma unroll
    for (int k = 0; k < 4; ++k) h[k] = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
    return r;
}

// One thread per grid node, all output channels in registers.
template <int CIN8, int COUT, bool LAST>
__global__ void __launch_bounds__(128) k_conv_simt(const __nv_bfloat16* __restrict__ in, const long long* __restrict__ in_off,
                                                   __nv_bfloat16* __restrict__ outb, const long long* __restrict__ out_off,
                                                   const __nv_bfloat16* __restrict__ W, const float* __restrict__ Bias,
                                                   const Seg* __restrict__ seg, const int* __restrict__ Ns, OutIO io, int mode,
                                                   __nv_bfloat16* __restrict__ zsave) {
    constexpr int CIN = CIN8 * 8;
    constexpr int NW = 27 * CIN * COUT;
    if (!cnn_runs(io.st, seg[blockIdx.x].inst)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __nv_bfloat16* sw = reinterpret_cast<__nv_bfloat16*>(smem_raw);
    for (int i = threadIdx.x; i < NW; i += blockDim.x) sw[i] = W[i];
    __syncthreads();
    const Seg sg = seg[blockIdx.x];
    const int N = Ns[sg.inst], M = N + 1;
    const long long Pd = N + 3, P = Pd * Pd * Pd;
    const __nv_bfloat16* xi = in + in_off[sg.inst];
    for (int n = sg.begin + threadIdx.x; n < sg.end; n += blockDim.x) {
        const int i = n % M, r = n / M, j = r % M, k = r / M;
        const long long p = (i + 1) + Pd * ((j + 1) + Pd * (k + 1));
        float acc[COUT];
#pragma unroll
        for (int co = 0; co < COUT; ++co) acc[co] = Bias[co];
        for (int tap = 0; tap < 27; ++tap) {
            const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
            const long long q = p + dx + Pd * (dy + Pd * dz);
#pragma unroll
            for (int c = 0; c < CIN8; ++c) {
                const uint4 raw = *reinterpret_cast<const uint4*>(xi + (c * P + q) * 8);
                float x[8];
                unpack8(raw, x);
#pragma unroll
                for (int ci = 0; ci < 8; ++ci) {
                    const __nv_bfloat16* wr = sw + ((size_t)tap * CIN + c * 8 + ci) * COUT;
                    if (COUT % 8 == 0) {
#pragma unroll
                        for (int co = 0; co < COUT; co += 8) {
                            float wv[8];
                            unpack8(*reinterpret_cast<const uint4*>(wr + co), wv);
#pragma unroll
                            for (int e = 0; e < 8; ++e) acc[co + e] = fmaf(wv[e], x[ci], acc[co + e]);
                        }
                    } else {
#pragma unroll
                        for (int co = 0; co < COUT; ++co) acc[co] = fmaf(__bfloat162float(wr[co]), x[ci], acc[co]);
                    }
                }
            }
        }
        if (!LAST) {
            __nv_bfloat16* o = outb + out_off[sg.inst];
#pragma unroll
            for (int c = 0; c < COUT / 8; ++c) {
                float v[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) v[e] = gelu_fast(acc[c * 8 + e]);
                *reinterpret_cast<uint4*>(o + (c * P + p) * 8) = pack8(v);
                if (zsave) *reinterpret_cast<uint4*>(zsave + out_off[sg.inst] + (c * P + p) * 8) = pack8(acc + c * 8);
            }
        } else {
            float* o = io.out + io.off[sg.inst];
            if (mode == CONV_PREC) {
                // Dirichlet nodes were written by the input pack (z0 = v0); with
                // natural conditions on the cube every node is the network's
                const bool bd = !io.D[sg.inst].natural && (i == 0 || i == N || j == 0 || j == N || k == 0 || k == N);
                const double s = io.st[sg.inst].s;
                const float scale = (float)(s / io.D[sg.inst].alpha);
                if (!bd) o[n] = scale * acc[0];
            } else {
                o[n] = acc[0];
            }
        }
    }
}

template <int CIN8, int COUT, bool LAST>
static md_status launch_conv(const __nv_bfloat16* in, const long long* in_off, __nv_bfloat16* outb,
                             const long long* out_off, const __nv_bfloat16* W, const float* B, const CnnWork* w,
                             const OutIO& io, int mode, cudaStream_t s, __nv_bfloat16* zsave = nullptr) {
    const size_t smem = (size_t)27 * CIN8 * 8 * COUT * sizeof(__nv_bfloat16);
    auto kern = k_conv_simt<CIN8, COUT, LAST>;
    kern<<<w->nodes.nblocks, 128, smem, s>>>(in, in_off, outb, out_off, W, B, w->nodes.seg, w->N, io, mode, zsave);
    MD_CHECK_LAUNCH();
    return MD_OK;
}

// The plane steps of the instances that run the network in this application
// (cnn_runs), in instance order, for the tensor-core launches (TcSched): one
// block scans the per-instance step counts.  Instance i is handled by thread
// i / per, per = ceil(ninst / blockDim.x).
__global__ void __launch_bounds__(1024) k_conv_sched(const KState* __restrict__ st, int ninst,
                                                     const long long* __restrict__ steps, int* __restrict__ act_inst,
                                                     long long* __restrict__ act_pre, int* __restrict__ count) {
    __shared__ int wn[32];
    __shared__ long long ws[32];
    const int per = (ninst + blockDim.x - 1) / blockDim.x;
    const int i0 = min(ninst, (int)threadIdx.x * per), i1 = min(ninst, i0 + per);
    int n = 0;
    long long sum = 0;
    for (int i = i0; i < i1; ++i)
        if (cnn_runs(st, i)) { ++n; sum += steps[i]; }
    // inclusive scan of (n, sum) over the block: within warps, then over warp totals
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int xn = n;
    long long xs = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int yn = __shfl_up_sync(0xffffffffu, xn, o);
        const long long ys = __shfl_up_sync(0xffffffffu, xs, o);
        if (lane >= o) { xn += yn; xs += ys; }
    }
    if (lane == 31) { wn[warp] = xn; ws[warp] = xs; }
    __syncthreads();
    if (warp == 0) {
        int tn = lane < nw ? wn[lane] : 0;
        long long ts = lane < nw ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int yn = __shfl_up_sync(0xffffffffu, tn, o);
            const long long ys = __shfl_up_sync(0xffffffffu, ts, o);
            if (lane >= o) { tn += yn; ts += ys; }
        }
        if (lane < nw) { wn[lane] = tn; ws[lane] = ts; }
    }
    __syncthreads();
    // exclusive offsets of this thread's instances
    int a = xn - n + (warp > 0 ? wn[warp - 1] : 0);
    long long p = xs - sum + (warp > 0 ? ws[warp - 1] : 0);
    for (int i = i0; i < i1; ++i)
        if (cnn_runs(st, i)) {
            act_inst[a] = i;
            act_pre[a] = p;
            ++a;
            p += steps[i];
        }
    if (threadIdx.x == blockDim.x - 1) {
        act_pre[a] = p;  // a = the count of running instances, p = their steps
        *count = a;
    }
}

static md_status tc_forward_layers(const md_cnn* c, CnnWork* w, const OutIO& io, ConvOut last, cudaStream_t s,
                                   unsigned long long* stamp0, unsigned long long* stamp1) {
    TcArgs a{};
    int grid = w->ngroups;
    if (io.st) {
        // inside a solve: only the instances still running the network, spread
        // over one CTA per SM
        k_conv_sched<<<1, 1024, 0, s>>>(io.st, w->ninst, w->steps, w->run_inst, w->run_pre, w->run_count);
        MD_CHECK_LAUNCH();
        a.sched = TcSched{w->run_inst, w->run_pre, w->run_count};
        grid = w->nsm;
    } else {
        a.sched = TcSched{w->all_inst, w->all_pre, w->all_count};
    }
    a.Ns = w->N;
    a.W = w->W;
    a.NS = w->NS;
    a.io = io;
    a.mode = (int)last;
    a.err = w->err;
    // layer 0: x0 (one chunk) -> a
    a.in = w->x0; a.in_off = w->off_x0; a.out = w->a; a.out_off = w->off_ab;
    a.wimg = c->wmma + c->wmma_off[0]; a.bias = c->b + c->b_off[0]; a.cout = 32;
    MD_TRY(tc_launch(1, w->tps, a, grid, s));
    __nv_bfloat16* src = w->a;
    __nv_bfloat16* dst = w->b;
    if (stamp0) k_stamp<<<1, 1, 0, s>>>(stamp0);
    for (int l = 1; l <= 4; ++l) {
        a.in = src; a.in_off = w->off_ab; a.out = dst; a.out_off = w->off_ab;
        a.wimg = c->wmma + c->wmma_off[l]; a.bias = c->b + c->b_off[l]; a.cout = 32;
        MD_TRY(tc_launch(0, w->tps, a, grid, s));
        std::swap(src, dst);
    }
    if (stamp1) k_stamp<<<1, 1, 0, s>>>(stamp1);
    a.in = src; a.in_off = w->off_ab; a.out = nullptr; a.out_off = nullptr;
    a.wimg = c->wmma + c->wmma_off[5]; a.bias = c->b + c->b_off[5]; a.cout = 1;
    MD_TRY(tc_launch(2, w->tps, a, grid, s));
    return MD_OK;
}

// Forward pass keeping every activation: A[l] (l = 1..5) the GELU outputs,
// Z[l] the pre-activations (BF16, 4 chunks, layout of w->a), x0 the input;
// the last layer writes y (FP32 grid, + io.off) as CONV_RAW.
md_status cnn_forward_train(const md_cnn* c, CnnWork* w, __nv_bfloat16* const* A, __nv_bfloat16* const* Z,
                            const OutIO& io, cudaStream_t s) {
    const __nv_bfloat16* src = w->x0;
    const long long* src_off = w->off_x0;
    for (int l = 0; l < MD_CNN_LAYERS; ++l) {
        const bool last = l == MD_CNN_LAYERS - 1;
        if (c->engine == 0) {
            TcArgs a{};
            a.Ns = w->N; a.sched = TcSched{w->all_inst, w->all_pre, w->all_count}; a.W = w->W; a.NS = w->NS; a.err = w->err;
            a.io = io; a.mode = CONV_RAW;
            a.in = src; a.in_off = src_off;
            a.out = last ? nullptr : A[l + 1]; a.out_off = w->off_ab;
            a.zsave = last ? nullptr : Z[l + 1];
            a.wimg = c->wmma + c->wmma_off[l]; a.bias = c->b + c->b_off[l]; a.cout = last ? 1 : 32;
            MD_TRY(tc_launch(l == 0 ? 1 : (last ? 2 : 0), w->tps, a, w->ngroups, s));
        } else {
            const __nv_bfloat16* W = c->w + c->w_off[l];
            const float* B = c->b + c->b_off[l];
            if (l == 0) {
                MD_TRY((launch_conv<1, 32, false>(src, src_off, A[1], w->off_ab, W, B, w, io, 0, s, Z[1])));
            } else if (!last) {
                MD_TRY((launch_conv<4, 32, false>(src, src_off, A[l + 1], w->off_ab, W, B, w, io, 0, s, Z[l + 1])));
            } else {
                MD_TRY((launch_conv<4, 1, true>(src, src_off, nullptr, nullptr, W, B, w, io, CONV_RAW, s)));
            }
        }
        if (!last) { src = A[l + 1]; src_off = w->off_ab; }
    }
    return MD_OK;
}

md_status cnn_forward_layers(const md_cnn* c, CnnWork* w, const OutIO& io, ConvOut last, cudaStream_t s,
                             unsigned long long* stamp0, unsigned long long* stamp1) {
    if (c->engine == 0) return tc_forward_layers(c, w, io, last, s, stamp0, stamp1);
    const __nv_bfloat16* W = c->w;
    const float* B = c->b;
    MD_TRY((launch_conv<1, 32, false>(w->x0, w->off_x0, w->a, w->off_ab, W + c->w_off[0], B + c->b_off[0], w, io, 0, s)));
    __nv_bfloat16* src = w->a;
    __nv_bfloat16* dst = w->b;
    if (stamp0) k_stamp<<<1, 1, 0, s>>>(stamp0);
    for (int l = 1; l <= 4; ++l) {
        MD_TRY((launch_conv<4, 32, false>(src, w->off_ab, dst, w->off_ab, W + c->w_off[l], B + c->b_off[l], w, io, 0, s)));
        std::swap(src, dst);
    }
    if (stamp1) k_stamp<<<1, 1, 0, s>>>(stamp1);
    MD_TRY((launch_conv<4, 1, true>(src, w->off_ab, nullptr, nullptr, W + c->w_off[5], B + c->b_off[5], w, io, (int)last, s)));
    return MD_OK;
}

// ---- input packing -------------------------------------------------------------------
// Network input X = [v0 / s, l / s, d] in the dx-paired one-chunk BF16
// layout (store_dx_pair); and the
// preconditioner output on Dirichlet nodes, z0 = v0 (the last layer writes
// the interior nodes only).
__global__ void k_pack_prec(const Seg* __restrict__ seg, const int* __restrict__ Ns, const InstDesc* __restrict__ D,
                            const float* __restrict__ v, const long long* __restrict__ voff, const KState* __restrict__ st,
                            __nv_bfloat16* __restrict__ x0, const long long* __restrict__ x0off, float* __restrict__ z,
                            int use_lift) {
    const Seg sg = seg[blockIdx.x];
    if (!cnn_runs(st, sg.inst)) return;
    const InstDesc& d = D[sg.inst];
    const int N = Ns[sg.inst], M = N + 1;
    const long long Pd = N + 3;
    const double s = st[sg.inst].s;
    const float sf = (float)s;
    const float* vi = v + voff[sg.inst];
    __nv_bfloat16* xo = x0 + x0off[sg.inst];
    auto chan = [&](int m, float (&c)[3]) {
        c[0] = s > 0.0 ? vi[m] / sf : 0.f;
        c[1] = (s > 0.0 && use_lift) ? d.lift32[m] / sf : 0.f;
        c[2] = d.dist[m];
    };
    for (int n = sg.begin + threadIdx.x; n < sg.end; n += blockDim.x) {
        const int i = n % M, r = n / M, j = r % M, k = r / M;
        const long long p = (i + 1) + Pd * ((j + 1) + Pd * (k + 1));
        float own[3], nx[3] = {0.f, 0.f, 0.f};
        chan(n, own);
        if (i < N) chan(n + 1, nx);
        store_dx_pair(xo + p * 8, own, nx, i == 0);
        if (!d.natural && (i == 0 || i == N || j == 0 || j == N || k == 0 || k == N)) z[voff[sg.inst] + n] = vi[n];
    }
}

md_status cnn_pack_prec(CnnWork* w, const InstDesc* D, const float* v, const long long* voff, const KState* st,
                        float* z, cudaStream_t s, bool use_lift) {
    k_pack_prec<<<w->nodes.nblocks, 128, 0, s>>>(w->nodes.seg, w->N, D, v, voff, st, w->x0, w->off_x0, z, use_lift ? 1 : 0);
    MD_CHECK_LAUNCH();
    return MD_OK;
}

__global__ void k_pack_raw(const Seg* __restrict__ seg, const int* __restrict__ Ns, const float* __restrict__ X,
                           __nv_bfloat16* __restrict__ x0, const long long* __restrict__ x0off) {
    const Seg sg = seg[blockIdx.x];
    const int N = Ns[sg.inst], M = N + 1;
    const long long Pd = N + 3, n3 = (long long)M * M * M;
    const float* xi = X + (long long)sg.inst * 3 * n3;
    __nv_bfloat16* xo = x0 + x0off[sg.inst];
    for (int n = sg.begin + threadIdx.x; n < sg.end; n += blockDim.x) {
        const int i = n % M, r = n / M, j = r % M, k = r / M;
        const long long p = (i + 1) + Pd * ((j + 1) + Pd * (k + 1));
        const float own[3] = {xi[n], xi[n3 + n], xi[2 * n3 + n]};
        float nx[3] = {0.f, 0.f, 0.f};
        if (i < N) {
            nx[0] = xi[n + 1];
            nx[1] = xi[n3 + n + 1];
            nx[2] = xi[2 * n3 + n + 1];
        }
        store_dx_pair(xo + p * 8, own, nx, i == 0);
    }
}

md_status cnn_pack_raw(CnnWork* w, const float* X, cudaStream_t s) {
    k_pack_raw<<<w->nodes.nblocks, 128, 0, s>>>(w->nodes.seg, w->N, X, w->x0, w->off_x0);
    MD_CHECK_LAUNCH();
    return MD_OK;
}

// ---- raw forward API -----------------------------------------------------------------
extern "C" md_status md_cnn_forward(const md_cnn* c, int n_nodes_edge, int batch, const float* X, float* Y, md_stream s) {
    if (!c || !X || !Y || n_nodes_edge < 2 || batch < 1) { md_set_error("md_cnn_forward: bad argument"); return MD_ERR_ARG; }
    std::vector<int> Ns(batch, n_nodes_edge - 1);
    CnnWork* w = nullptr;
    MD_TRY(cnn_work_create(Ns, &w));
    std::vector<long long> off(batch);
    const long long n3 = (long long)n_nodes_edge * n_nodes_edge * n_nodes_edge;
    for (int i = 0; i < batch; ++i) off[i] = i * n3;
    long long* doff = nullptr;
    md_status st = dev_upload(&w->allocs, &doff, off.data(), off.size());
    OutIO io{Y, doff, nullptr, nullptr, nullptr, nullptr};
    if (st == MD_OK) st = cnn_pack_raw(w, X, (cudaStream_t)s);
    if (st == MD_OK) st = cnn_forward_layers(c, w, io, CONV_RAW, (cudaStream_t)s);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)s);
    int err = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&err, w->err, sizeof(int), cudaMemcpyDeviceToHost);
    cnn_work_destroy(w);
    if (st == MD_OK && e != cudaSuccess) st = md_cuda_status(e, "md_cnn_forward", __FILE__, __LINE__);
    if (st == MD_OK && err) { md_set_error("md_cnn_forward: a convolution timed out"); st = MD_ERR_TIMEOUT; }
    return st;
}
