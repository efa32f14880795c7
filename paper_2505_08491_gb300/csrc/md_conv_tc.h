// Tensor-core (tcgen05) convolution launches (internal).
#pragma once
#include <vector>

#include "md_cnn.h"

// One work unit: in-plane rows [s0, s0 + TPS*126) of one instance, walked
// over padded planes [z0, z1) (TPS = 128-lane tiles per plane step, each
// yielding 126 rows).
struct TcUnit { int inst, s0, z0, z1; };

// The plane steps one launch works on.  The instances that run are listed in
// instance order, act_inst[a] for a < *count; instance act_inst[a] owns the
// steps [act_pre[a], act_pre[a + 1]): its columns of TPS*126 in-plane rows in
// order (column c starts at in-plane row c TPS 126), each walked over the N+1
// padded planes [1, N+2) that hold grid nodes.  CTA b of a grid of G takes
// the steps [S b / G, S (b + 1) / G), S = act_pre[*count], cut at column
// ends into units, so every CTA walks the same number of plane steps
// whichever instances run.
struct TcSched {
    const int* act_inst;
    const long long* act_pre;
    const int* count;
};

#define TC_EPI_CH 8                          // output channels per epilogue thread
#define TC_EPI_GROUPS (32 / TC_EPI_CH)       // channel groups
#define TC_EPI_WARPS (4 * TC_EPI_GROUPS)     // epilogue warps: 4 TMEM lane quarters x channel groups
#define TC_MMA_WARPS 2                       // MMA issuers: warp 1 and the last warp, one tile of a step each
#define TC_MMA2_WARP (2 + TC_EPI_WARPS)      // warp index of the second issuer
#define TC_THREADS (32 * (1 + TC_MMA_WARPS + TC_EPI_WARPS))  // + producer warp
#define TC_TPS_MAX 2                         // tiles per plane step (epilogue exchange buffers)
#define TC_NBUF_MAX 8                        // deepest accumulator ring (last layer)

struct TcArgs {
    const __nv_bfloat16* in;     // activation buffer (chunk-major padded layout)
    const long long* in_off;     // per instance element offset
    __nv_bfloat16* out;          // next activation buffer (hidden layers)
    const long long* out_off;
    const int* Ns;               // per instance grid size N
    TcSched sched;               // the plane steps of this launch and their split over the CTAs
    int W;                       // rows per (window, chunk) region in shared memory
    int NS;                      // ring slots
    const __nv_bfloat16* wimg;   // weight image in operand layout
    const float* bias;
    int cout;                    // real output channels
    OutIO io;                    // last layer output / instance gating
    int mode;                    // ConvOut of the last layer
    int* err;                    // set on a timed-out wait
    __nv_bfloat16* zsave;        // optional pre-activation copy (hidden layers, layout of out)
    // input gradient (training's backward): the layer runs the adjoint
    // convolution (weights flipped and transposed in wimg, zero bias) and the
    // epilogue multiplies by GELU'(zprev), the previous layer's saved
    // pre-activation (layout of out), instead of applying GELU
    const __nv_bfloat16* zprev;
    int dgrad;
};

__host__ __device__ constexpr int tc_wimg_bytes(int kind) {
    return kind == 1 ? 3 * 3 * 2 * 32 * 16 : (kind == 2 ? 3 * 4 * 16 * 16 : 9 * 4 * 96 * 16);
}
// rows one window copy holds: TPS tiles 126 rows apart, 128 rows each, read
// at dy offsets 0..2 Pd from the window start, plus 8 rows of slack (the
// first layer's window starts one row early and reads up to 2 rows past the
// last tile's dy = +1 rows: its dx = +1 chunk)
__host__ __device__ constexpr int tc_window_load_rows(int tps, int pd) { return (tps - 1) * 126 + 128 + 2 * pd + 8; }
__host__ __device__ constexpr int tc_align(int b) { return (b + 1023) & ~1023; }

int tc_smem_bytes(int kind, int W, int ns);
int tc_ring_slots(int W);
int tc_window_rows(int tps, int pd_max);
md_status tc_prepare(int W, int tps);
md_status tc_launch(int kind, int tps, const TcArgs& a, int grid, cudaStream_t s);
void tc_weight_image(int kind, const float* W, int cin, int cout, std::vector<__nv_bfloat16>& img);
