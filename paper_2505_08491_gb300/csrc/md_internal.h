// Internal declarations of the md library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/md.h"

#define MD_KMAX 64              // largest FGMRES restart length
#define MD_MAXR (MD_KMAX + 4)   // reduction values per block
#define MD_TB 256               // threads per block of the streaming kernels
#define MD_INNER_MAX 4          // most inner FGMRES steps of the 3D block solve

// ---------------------------------------------------------------------------
// error handling
void md_set_error(const char* fmt, ...);
md_status md_cuda_status(cudaError_t e, const char* what, const char* file, int line);

#define MD_CUDA(call)                                                              \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) return md_cuda_status(e_, #call, __FILE__, __LINE__); \
    } while (0)
#define MD_TRY(call)                      \
    do {                                  \
        md_status s_ = (call);            \
        if (s_ != MD_OK) return s_;       \
    } while (0)
#define MD_CHECK_LAUNCH() MD_CUDA(cudaGetLastError())

// ---------------------------------------------------------------------------
// One assembled instance, as the kernels see it.  All pointers are device
// pointers owned by the md_op.
struct InstDesc {
    int N, n3, n1, nq, ntouch, nsegs;
    int natural;      // 1: natural (Neumann) conditions on the cube faces, no Dirichlet rows
    long long n;
    double h, beta, alpha;
    double st64[4];   // K00 (+ sigma mass) stencil by offset class: centre, face, edge, corner
    float st32[4];
    double ms64[4];   // Q1 mass stencil (load vector)
    // Pi, row per quadrature point: columns = grid nodes, values = averaging weights
    const int* pi_ptr; const int* pi_col; const double* pi_v64; const float* pi_v32;
    // per quadrature point: 1D element end nodes and P1 values there
    const int* qa; const int* qb;
    const double* psa64; const double* psb64; const float* psa32; const float* psb32;
    // Pi^T W, row per touched grid node: entries (q, Pi[q,n] w_q); rows ordered
    // by stencil tile (below), and by node within a tile
    const int* tn_node; const int* tn_ptr; const int* tn_q; const double* tn_v64; const float* tn_v32;
    // stencil tiles of the operator apply: tz planes x ty rows x all N+1
    // columns of the grid, numbered zt * nyt + yt (ntiles of them); the rows
    // of Pi^T W of tile b are tile_tptr[b] .. tile_tptr[b+1] - 1.  mdiv =
    // ceil(2^32 / (N+1)) divides by N+1 with one multiply-high (exact for
    // dividends below 2^20).
    int ty, tz, nyt, ntiles;
    unsigned int mdiv;
    const int* tile_tptr;
    // 1D rows: kappa K1 (CSR) and Psi^T W (entries (q, psi w_q))
    const int* k1_ptr; const int* k1_col; const double* k1_v64; const float* k1_v32;
    const int* pw_ptr; const int* pw_q; const double* pw_v64; const float* pw_v32;
    const double* load1;      // int_Lambda psi_i ds (0 on 1D Dirichlet nodes)
    // the known 1D Dirichlet values moved to the right-hand side: b0 += rhs0,
    // b1 += rhs1 (b1 = u_d on those nodes); nullptr without 1D Dirichlet nodes
    const double* rhs0; const double* rhs1;
    // tree LDL^T of B11 in elimination order (children before parents)
    const int* tr_order; const int* tr_parent;
    // level schedule of its sweeps: nodes by height above the leaves in
    // lv_up[lvu_ptr[h] .. lvu_ptr[h+1]) (a node's children are lower), the
    // children of node i in ch_idx[ch_ptr[i] .. ch_ptr[i+1]); nodes by depth
    // below the roots in lv_dn[lvd_ptr[k] .. lvd_ptr[k+1])
    int nlvu, nlvd;
    const int* lvu_ptr; const int* lv_up; const int* ch_ptr; const int* ch_idx; const int* lvd_ptr; const int* lv_dn;
    const double* tr_l64; const double* tr_dinv64; const float* tr_l32; const float* tr_dinv32;
    // per grid / per dof
    const float* dist;      // n3
    const double* dinv64;   // n, 1 / diag(A)
    const float* dinv32;
    const float* sminv32;   // n3, the Jacobi smoother's row scaling rho_i / c_ii (md_apply.cu)
    const double* segs;     // nsegs * 6 segment end points (distance field)
    // scratch owned by the op
    double* t64; float* t32;  // nq
    float* lift32;            // n3, zero except touched nodes
    float* ltouch32;          // ntouch
};

// A block of a batched launch: instance, work kind, [begin, end) range.
struct Seg { int inst, kind, begin, end; };
// Blocks of one instance inside a table.
struct InstRange { int first, count; };

struct Table {
    Seg* seg = nullptr;         // device
    InstRange* range = nullptr; // device, per instance
    int nblocks = 0;
    std::vector<InstRange> hrange;
    int smem32 = 0, smem64 = 0; // dynamic shared memory of its launch (stencil tiles), FP32 / FP64
};

// Tables for the launches of a set of instances.
struct Tables {
    Table apply_a;   // kind 1: averaging gather t = Pi u0 - Psi u1 over nq
    Table apply_b;   // kind 4: stencil tile with its Pi^T W t rows ; kind 3: 1D rows over n1
    Table vec;       // kind 0: ranges over n (whole instance vector)
    Table n3;        // kind 0: ranges over n3
    Table touch;     // kind 0: ranges over ntouch
};

// ---------------------------------------------------------------------------
// handles
struct md_op {
    InstDesc h;                  // host copy of the descriptor (device pointers)
    InstDesc* d = nullptr;       // device copy
    std::vector<void*> allocs;   // device allocations to free
    int n_touch_nodes = 0;
    Tables tabs;                 // launch tables of this instance alone
    long long* off0 = nullptr;   // device {0}
    md_batch* solver_cache[3] = {nullptr, nullptr, nullptr};
    int solver_cache_restart[3] = {0, 0, 0};
    const md_cnn* solver_cache_cnn = nullptr;
};

struct CnnLayer { int cin, cout, cin_pad; };

unsigned long long md_next_cnn_uid();  // process-wide counter (md_cnn.cu)

struct md_cnn {
    // identity of this network for captured graphs: a handle address can be
    // reused by a later network, a uid is never reused
    unsigned long long uid = md_next_cnn_uid();
    std::vector<float> host;     // FP32 master copy (MD_CNN_NPARAMS)
    __nv_bfloat16* w = nullptr;  // device packed weights, per layer [tap][cout][cin_pad]
    float* b = nullptr;          // device biases, per layer [cout]
    size_t w_off[MD_CNN_LAYERS + 1];
    size_t b_off[MD_CNN_LAYERS + 1];
    // tcgen05 operand images of the weights (md_conv_tc.cu)
    __nv_bfloat16* wmma = nullptr;
    size_t wmma_off[MD_CNN_LAYERS + 1];
    int engine = 0;              // 0: tensor cores (tcgen05), 1: CUDA cores
    // input-gradient weights (training): per layer [tap'][c_out pad][c_in]
    __nv_bfloat16* wt = nullptr;
    size_t wt_off[MD_CNN_LAYERS + 1];
    // tcgen05 operand images of the adjoint convolutions (layers 1-5; the
    // flipped, transposed kernels: hidden 32 -> 32 and the last layer's 1 -> 32)
    __nv_bfloat16* wtmma = nullptr;
    size_t wtmma_off[MD_CNN_LAYERS + 1];
};

// Per-instance Krylov state (device).
struct KState {
    double H[(MD_KMAX + 1) * MD_KMAX];   // Hessenberg, column j at H[j * (KMAX+1)]
    double cs[MD_KMAX], sn[MD_KMAX];
    double g[MD_KMAX + 1];
    double y[MD_KMAX];
    double sig[MD_KMAX + 1];             // 1 / ||V_j||: v_j = sig_j V_j
    double coef[MD_KMAX + 1];            // update coefficients of the running pass
    double wn2_before;                   // ||W||^2 before orthogonalisation
    double bnorm, beta, relres, est;
    double s2_touch, s, v3n2;            // preconditioner input norm pieces
    double tol, inner_tol;
    double rho, alpha_cg, pq;            // CG scalars
    unsigned long long t_start, t_done;  // globaltimer stamps
    double relres_prev;                  // true relative residual at the previous restart
    int j, m, active, converged, iters, reorth, nan_seen, fallback, maxit, cycle_iters, stalls;
    int fb_iter;                         // iteration at which the Jacobi fallback began
    // inner FGMRES steps of the 3D block solve: Hessenberg (column j at
    // iH[j * (MD_INNER_MAX + 1)]), Gram-Schmidt coefficients, solution, ||b0||
    double iH[(MD_INNER_MAX + 1) * MD_INNER_MAX];
    double icoef[MD_INNER_MAX + 1];
    double iy[MD_INNER_MAX];
    double ib0;
    unsigned int counter[12];            // last-block counters per reduction kernel
};

// Per-instance results written when an instance finishes: iterations,
// iterations preconditioned by the network (all of them unless the instance
// fell back to Jacobi), true relative residual, seconds from solve start.
struct ResOut {
    int* iters;
    int* net_iters;
    double* relres;
    double* time;
};

// An instance runs the network in this launch: inside its cycle and not
// switched to the Jacobi fallback.
__host__ __device__ inline bool cnn_runs(const KState* st, int inst) {
    return !st || (st[inst].active && !st[inst].fallback);
}

// Stencil tile shape of the operator apply for grid N: ty rows of all N+1
// columns (at most 256 columns, one per thread) and tz planes, such that the
// FP64 input tile with its halo and the output tile fit 64 KB of shared memory
// (tiles twice as large measured slower on the mixed batch).
void apply_tile_shape(int N, int* ty, int* tz);
int apply_tile_smem(int N, int ty, int tz, int elem_bytes);
md_status apply_prepare(int smem32, int smem64);

// Problem-size independent kernel launches (md_apply.cu)
struct KState;
// gate: 0 all instances, 1 active ones (inside a cycle), 2 unfinished ones
md_status launch_apply(const Tables& T, const InstDesc* d, int ninst, md_prec prec, const void* u,
                       const long long* off, void* y, cudaStream_t s, const KState* st = nullptr, int gate = 0);
md_status launch_rhs(const md_op* op, const double* f, double g, double* b, cudaStream_t s);
md_status launch_dist(md_op* op, cudaStream_t s);
md_status launch_dinv_fill(md_op* op, const std::vector<double>& touch_diag, const std::vector<double>& touch_rowsum,
                           const std::vector<double>& d1, cudaStream_t s);

// Tables (md_tables.cpp)
// vec_chunk: elements per block of the streaming vector kernels.  The Krylov
// kernels of FGMRES carry per-block fixed costs (a reduction per basis
// vector, the last-block combine) and prefer long chunks; the CG kernels
// stream one or two vectors and prefer more, shorter blocks.
#define MD_VEC_CHUNK_FGMRES 8192
#define MD_VEC_CHUNK_CG 2048
md_status build_tables(const std::vector<const InstDesc*>& insts, Tables* T, std::vector<void*>* allocs,
                       int vec_chunk = MD_VEC_CHUNK_FGMRES);
void free_tables(Tables* T);

// device memory helpers
template <class T>
md_status dev_upload(std::vector<void*>* allocs, T** dst, const T* src, size_t count) {
    *dst = nullptr;
    if (count == 0) count = 1;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) { md_set_error("cudaMalloc(%zu) failed: %s", count * sizeof(T), cudaGetErrorString(e)); return MD_ERR_OOM; }
    allocs->push_back(p);
    if (src) {
        e = cudaMemcpy(p, src, count * sizeof(T), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return md_cuda_status(e, "cudaMemcpy", __FILE__, __LINE__);
    }
    *dst = (T*)p;
    return MD_OK;
}
template <class T>
md_status dev_alloc(std::vector<void*>* allocs, T** dst, size_t count, bool zero = true) {
    MD_TRY(dev_upload<T>(allocs, dst, nullptr, count));
    if (zero) MD_CUDA(cudaMemset(*dst, 0, (count ? count : 1) * sizeof(T)));
    return MD_OK;
}
void dev_free_all(std::vector<void*>* allocs);

// preconditioner / network (md_prec.cu, md_cnn.cu)
struct CnnWork;
md_status cnn_work_create(const std::vector<const InstDesc*>& insts, CnnWork** out);
void cnn_work_destroy(CnnWork* w);
