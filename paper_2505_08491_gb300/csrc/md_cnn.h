// Network workspace and convolution launches (internal).
#pragma once
#include "md_internal.h"

// Activation layout: per instance a zero-haloed padded grid of P = Pd^3 rows,
// Pd = N + 3, row p = (i+1) + Pd((j+1) + Pd(k+1)) for grid node (i,j,k);
// channels in chunks of 8: element (chunk c, row p, lane l) at
// (c * P + p) * 8 + l.  Halo rows are never written and stay zero, which is
// the zero 'same' padding of every layer.  Each buffer has a zero margin of
// CNN_MARGIN_ROWS rows before the first and after the last instance, which
// the tensor-core windows of halo-only tiles may read.  The one exception to
// zero halo rows is the dx-paired one-chunk layout below.
#define CNN_MARGIN_ROWS 8192

#ifdef __CUDACC__
// One-chunk inputs of the first layer's kind (the network input X0, and the
// last layer's adjoint input dY in training) are stored dx-paired: row p holds
// the node's channels (at most 3) in lanes 0-2 and those of the next node
// along x in lanes 3-5 (zero past the grid row's end), lanes 6-7 zero, so that
// one 8-lane chunk carries two dx taps of the convolution; the halo row just
// before the first node of every grid row holds that node's channels in lanes
// 3-5.  rowp: the node's row; first: the node starts its grid row (i = 0).
__device__ __forceinline__ void store_dx_pair(__nv_bfloat16* rowp, const float (&own)[3], const float (&next)[3],
                                              bool first) {
    uint4 r;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&r);
    h[0] = __floats2bfloat162_rn(own[0], own[1]);
    h[1] = __floats2bfloat162_rn(own[2], next[0]);
    h[2] = __floats2bfloat162_rn(next[1], next[2]);
    h[3] = __floats2bfloat162_rn(0.f, 0.f);
    *reinterpret_cast<uint4*>(rowp) = r;
    if (first) {
        h[0] = __floats2bfloat162_rn(0.f, 0.f);
        h[1] = __floats2bfloat162_rn(0.f, own[0]);
        h[2] = __floats2bfloat162_rn(own[1], own[2]);
        *reinterpret_cast<uint4*>(rowp - 8) = r;
    }
}
#endif
struct CnnWork {
    int ninst = 0;
    std::vector<void*> allocs;
    std::vector<int> hN;
    int* N = nullptr;              // device, per instance
    // tensor-core path: z-walking work units of tps*126 in-plane rows,
    // window rows W, NS ring slots.  The plane steps of a launch are split
    // evenly over its CTAs (TcSched): every instance (all_*, ngroups CTAs) for
    // a pass without solver state, or the instances that still run the
    // network (run_*, written on the device before each application, nsm
    // CTAs), so that a solve whose instances have mostly converged still
    // spreads the rest over every SM.
    long long* steps = nullptr;    // device, per instance: plane steps (columns x (N+1))
    int* all_inst = nullptr;
    long long* all_pre = nullptr;
    int* all_count = nullptr;
    int* run_inst = nullptr;
    long long* run_pre = nullptr;
    int* run_count = nullptr;
    int ngroups = 1, tps = 2, W = 0, NS = 0, nsm = 148, pd_max = 0;
    int* err = nullptr;            // set by a timed-out wait in a conv kernel
    __nv_bfloat16* x0 = nullptr;   // 1 chunk, dx-paired (store_dx_pair)
    __nv_bfloat16* a = nullptr;    // 4 chunks
    __nv_bfloat16* b = nullptr;    // 4 chunks
    long long* off_x0 = nullptr;   // per instance, element offset into x0
    long long* off_ab = nullptr;   // per instance, element offset into a / b
    std::vector<long long> h_off_x0, h_off_ab;
    Table nodes;                   // grid-node ranges per instance
    long long total_nodes = 0;
};

md_status cnn_work_create(const std::vector<int>& Ns, CnnWork** out);
void cnn_work_destroy(CnnWork* w);
// tiles per plane step of the tensor-core convolutions (1 or 2), and its
// autotuning by timed forward passes (us[0], us[1]: per pass with 1 and 2)
md_status cnn_work_set_tps(CnnWork* w, int tps);
struct md_cnn;
md_status cnn_autotune_tps(const md_cnn* c, CnnWork* w, float* out, const long long* off, double* us);

// Output handling of the last layer.
enum ConvOut {
    CONV_PREC = 1,     // z0 = (s / alpha) y on interior nodes, v0 on Dirichlet nodes
    CONV_RAW = 2       // y (FP32) at the grid node
};

struct OutIO {
    float* out;                // instance i's 3D part starts at out + off[i]
    const long long* off;
    const float* vin;          // CONV_PREC: preconditioner input (Dirichlet copy), + vin_off[i]
    const long long* vin_off;
    const KState* st;          // CONV_PREC: st[i].s
    const InstDesc* D;         // CONV_PREC: D[i].alpha
};

md_status cnn_forward_layers(const md_cnn* c, CnnWork* w, const OutIO& io, ConvOut last, cudaStream_t s,
                             unsigned long long* stamp0 = nullptr, unsigned long long* stamp1 = nullptr);
md_status cnn_forward_train(const md_cnn* c, CnnWork* w, __nv_bfloat16* const* A, __nv_bfloat16* const* Z,
                            const OutIO& io, cudaStream_t s);
md_status cnn_upload(md_cnn* c);
// X0 = [v0 / s, l / s, d] from a preconditioner input (instance 3D part at v + voff[i])
// use_lift = false: the lifted-1D channel is zero (block lower-triangular order)
md_status cnn_pack_prec(CnnWork* w, const InstDesc* D, const float* v, const long long* voff, const KState* st,
                        float* z, cudaStream_t s, bool use_lift = true);
// X0 from a raw channel-major FP32 input (sample, channel, z, y, x)
md_status cnn_pack_raw(CnnWork* w, const float* X, cudaStream_t s);
