// Batched Krylov solvers: flexible GMRES(k) with the block preconditioner
// (Section 4, eq. (twosteps)) and Jacobi-CG, for one or many instances.
//
// FGMRES, right preconditioned, per instance:
//   cycle: r = b - A x (FP64), beta = ||r||, V_0 = r (FP32), v_0 = V_0/||V_0||
//     for j: Z_j = P(V_j); W = A Z_j;                       (FP32)
//            h_ij = (w, v_i) by classical Gram-Schmidt on the stored,
//            unnormalised V_i (v_i = sig_i V_i, P positively homogeneous so
//            z_j = sig_j Z_j), a second pass when ||w|| drops below half;
//            Givens rotations on the FP64 Hessenberg, estimate |g_{j+1}|;
//     x += sum_j y_j sig_j Z_j with H y = g (FP64 x, FP32 correction).
// Every kernel runs across all instances; an instance leaves the cycle when
// its estimate reaches max(tol ||b||, 1e-5 beta) (FP32 vectors cannot carry
// the residual further within one cycle), and the restart's FP64 residual
// decides convergence.  One restart cycle is captured as a CUDA graph.
//
// Jacobi-CG: FP64 conjugate gradients with M = diag(A)^{-1}; stops on the
// recursive residual, then reports the true one.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "md_cnn.h"
#include "md_common.cuh"

#define INNER_REL 1e-5
#define STAGNATION_MIN_ITERS 10
// threads of the per-instance tree solve + lift: the lift walks the touched grid
// nodes with dependent loads, so it wants many threads in flight
#define TREE_TB 1024
// elements per thread and loop trip of the CG streaming kernels
#define CG_U 4

// Control block of one batched solve, on the device: the limits the host
// writes before launching the solve graph, what the graph counts while it
// runs, and (when profiling) the summed device time of its sections.
struct SolveCtl {
    double tol;
    int maxit;
    int max_cycles;
    int cycles;                        // restart cycles (CG: chunks of iterations) run
    int pad;
    unsigned long long kernels;        // kernels run by the loop (slots, restarts, chunks)
    unsigned long long t_prec, t_conv, t_apply, t_arn, t_restart;  // ns summed over slots / restarts
    unsigned long long slots, conv_groups;
    unsigned long long stamp[8];
};

struct md_batch {
    int ninst = 0;
    md_solver solver = MD_SOLVER_FGMRES_JACOBI;
    int k = 30;
    const md_cnn* cnn = nullptr;
    std::vector<const md_op*> ops;
    std::vector<InstDesc> hdesc;
    InstDesc* d = nullptr;
    std::vector<void*> allocs;
    Tables tabs;
    std::vector<long long> hoff;
    long long* off = nullptr;
    long long total = 0;
    double *x = nullptr, *b = nullptr, *y64 = nullptr, *r64 = nullptr, *p64 = nullptr;
    float *V = nullptr, *Z = nullptr;
    KState* st = nullptr;
    double* part = nullptr;
    int* ndone = nullptr;
    ResOut res{};
    int max_n1 = 0, max_nq = 0;
    CnnWork* cw = nullptr;
    // the whole solve as one executable graph, driven on the device: the
    // set-up kernels, then a WHILE node over restart cycles (CG: chunks of
    // iterations) whose body, for FGMRES, runs every iteration slot under an
    // IF node that skips it once no instance iterates in the cycle
    cudaStream_t cap = nullptr, cap_body = nullptr;  // capture streams (solve, loop body)
    cudaGraphExec_t solve_graph = nullptr;
    long long init_kernels = 0;          // kernels of the set-up part (the rest are counted on the device)
    int host_loop = 0;                   // 1: the host-driven loop below instead of solve_graph
    cudaGraphExec_t init_graph = nullptr, cycle_graph = nullptr;
    long long cycle_kernels = 0;
    SolveCtl* ctl = nullptr;             // device: limits of this solve, counters, profile sums
    SolveCtl* h_ctl = nullptr;           // pinned host copy
    int if_mode = -1;                    // 2: one graph per solve, 3: the host-driven loop
    md_tuning_t tuning{};                // choices of the autotuner at creation
    int prec_order = 0;                  // 0: block upper-triangular (the paper's), 1: lower
    int graph_prec_order = 0;
    int inner_m = 0;                     // inner FGMRES steps of the 3D block solve (0: one network application)
    int graph_inner_m = 0;
    float *iV = nullptr, *iZ = nullptr;  // their basis (MD_INNER_MAX + 1) and directions (MD_INNER_MAX), x total
    int smooth_nu = 0;                   // Jacobi sweeps before and after the network (0: none)
    float smooth_omega = 1.f;            // their damping
    int graph_smooth_nu = 0;
    float graph_smooth_omega = 1.f;
    unsigned long long graph_cnn_uid = 0;  // network the graph was captured with (0: none)
    // the U-net as the 3D block solve (md_batch_set_unet; uniform grid size un):
    // its input (ninst x 2 x un^3) and output (ninst x un^3)
    md_unet* unet = nullptr;
    const md_unet* graph_unet = nullptr;
    float *ux = nullptr, *uy = nullptr;
    int un = 0;
    bool graph_prof = false;
    int graph_engine = -1;
    long long graph_kernels = 0;
    std::vector<double> last_times;
    // instrumentation
    bool profiling = false;
    md_batch_stats_t stats{};
};

// Device timestamps of the profiled sections (SolveCtl::stamp): per iteration
// slot (reused by every slot, which run in order), then the restart.
enum { ST_PRE0 = 0, ST_CONV0, ST_CONV1, ST_APPLY0, ST_APPLY1, ST_ARN1, ST_REST0, ST_REST1, ST_COUNT };

static unsigned long long* stamp_at(md_batch* B, int which) {
    if (!B->profiling) return nullptr;
    return &B->ctl->stamp[which];
}
static void stamp(unsigned long long* at, cudaStream_t s) {
    if (at) k_stamp<<<1, 1, 0, s>>>(at);
}

// ---------------------------------------------------------------------------
// reduction helper: each block writes R partials; the last block of the
// instance sums them in block order (deterministic) into out[0..R)
template <int MAXV>
__device__ inline void reduce_values(double* vals, int count, double* part, int blk, const InstRange& rg,
                                     unsigned int* counter, double* out, double* sh) {
    // vals: per-thread values [count] in registers/local; reduce in block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int r = 0; r < count; ++r) {
        double x = warp_sum(vals[r]);
        if (lane == 0) sh[r * 32 + warp] = x;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < count; r += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += sh[r * 32 + w];
        part[(size_t)blk * MD_MAXR + r] = s;
    }
    __syncthreads();
    bool last = last_block_arrive(counter, rg.count);
    out[0] = last ? 1.0 : 0.0;
    if (!last) return;
    for (int r = threadIdx.x; r < count; r += blockDim.x) {
        double s = 0.0;
        for (int b2 = rg.first; b2 < rg.first + rg.count; ++b2) s += part[(size_t)b2 * MD_MAXR + r];
        sh[r] = s;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
__global__ void k_init_state(KState* st, int ninst, const SolveCtl* ctl, int* ndone) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *ndone = 0;
    if (i >= ninst) return;
    KState& S = st[i];
    S.tol = ctl->tol; S.maxit = ctl->maxit; S.iters = 0; S.converged = 0; S.active = 0; S.j = 0; S.m = 0;
    S.reorth = 0; S.nan_seen = 0; S.fallback = 0; S.bnorm = 0; S.relres = 1; S.cycle_iters = -1; S.stalls = 0;
    S.fb_iter = 0; S.relres_prev = 1.0;
    S.inner_tol = INNER_REL;
    S.t_start = globaltimer();
    S.t_done = 0;
    for (int c = 0; c < 12; ++c) S.counter[c] = 0;
}

// ---- the solve loop's conditions, set on the device (conditional graph nodes)
// WHILE over cycles: another restart cycle (CG: chunk) while an instance is
// unfinished and the cycle limit is not reached.  At the end of a cycle
// (end_of_cycle = 1) it also counts the cycle, the nk kernels of the loop
// body outside the iteration slots and, when profiling, the restart's time.
__global__ void k_loop_cond(SolveCtl* ctl, const int* ndone, int ninst, cudaGraphConditionalHandle hw,
                            unsigned long long nk, int end_of_cycle, int prof) {
    if (end_of_cycle) {
        ctl->cycles += 1;
        ctl->kernels += nk;
        if (prof) ctl->t_restart += ctl->stamp[ST_REST1] - ctl->stamp[ST_REST0];
    }
    cudaGraphSetConditional(hw, (*ndone < ninst && ctl->cycles < ctl->max_cycles) ? 1u : 0u);
}

// End of a cycle of the host-driven loop: count it and, when profiling, add
// the restart's time.
__global__ void k_cycle_count(SolveCtl* ctl, int prof) {
    ctl->cycles += 1;
    if (prof) ctl->t_restart += ctl->stamp[ST_REST1] - ctl->stamp[ST_REST0];
}

// After an iteration slot: count it and, when profiling, add its section times.
__global__ void k_slot_count(SolveCtl* ctl, int prof) {
    ctl->slots += 1;
    if (prof) {
        const unsigned long long* t = ctl->stamp;
        ctl->t_prec += t[ST_APPLY0] - t[ST_PRE0];
        ctl->t_conv += t[ST_CONV1] - t[ST_CONV0];
        ctl->t_apply += t[ST_APPLY1] - t[ST_APPLY0];
        ctl->t_arn += t[ST_ARN1] - t[ST_APPLY1];
    }
}

// sum of b^2 -> bnorm ; kind: FP64 batched vector
__global__ void __launch_bounds__(MD_TB) k_norm_b(const Seg* __restrict__ seg, const InstRange* __restrict__ rng,
                                                  const long long* __restrict__ off, const double* __restrict__ b,
                                                  KState* st, double* part) {
    __shared__ double sh[32 * 4];
    const Seg sg = seg[blockIdx.x];
    const double* bi = b + off[sg.inst];
    double v[1] = {0.0};
    for (int e = sg.begin + threadIdx.x; e < sg.end; e += blockDim.x) v[0] += bi[e] * bi[e];
    double flag;
    reduce_values<1>(v, 1, part, blockIdx.x, rng[sg.inst], &st[sg.inst].counter[0], &flag, sh);
    if (flag == 1.0 && threadIdx.x == 0) st[sg.inst].bnorm = sqrt(sh[0]);
}

// the instance's preconditioner becomes Jacobi for the rest of its solve
__device__ inline void set_fallback(KState& S) {
    if (!S.fallback) {
        S.fallback = 1;
        S.fb_iter = S.iters;
    }
}

__device__ inline void mark_done(KState& S, int* ndone, ResOut res, int inst) {
    S.active = 0;
    S.converged = S.relres <= S.tol ? 1 : 0;
    S.t_done = globaltimer();
    S.m = 0;
    res.iters[inst] = S.iters;
    res.net_iters[inst] = S.fallback ? S.fb_iter : S.iters;
    res.relres[inst] = S.relres;
    res.time[inst] = (double)(S.t_done - S.t_start) * 1e-9;
    atomicAdd(ndone, 1);
}

// FGMRES restart: r = b - y (y = A x in FP64), V_0 = r in FP32
__global__ void __launch_bounds__(MD_TB) k_resid(const Seg* __restrict__ seg, const InstRange* __restrict__ rng,
                                                 const long long* __restrict__ off, const InstDesc* __restrict__ D,
                                                 const double* __restrict__ b, const double* __restrict__ y, float* V0,
                                                 KState* st, double* part, int* ndone, ResOut res, int k) {
    __shared__ double sh[32 * 4];
    const Seg sg = seg[blockIdx.x];
    KState& S = st[sg.inst];
    if (S.t_done) return;  // finished instances skip
    const long long o = off[sg.inst];
    const int n3 = D[sg.inst].n3;
    double v[3] = {0.0, 0.0, 0.0};
    for (int e = sg.begin + threadIdx.x; e < sg.end; e += blockDim.x) {
        const double r = b[o + e] - y[o + e];
        const float rf = (float)r;
        V0[o + e] = rf;
        v[0] += r * r;
        v[1] += (double)rf * rf;
        if (e < n3) v[2] += (double)rf * rf;
    }
    double flag;
    reduce_values<3>(v, 3, part, blockIdx.x, rng[sg.inst], &S.counter[1], &flag, sh);
    if (flag == 1.0 && threadIdx.x == 0) {
        S.beta = sqrt(sh[0]);
        S.relres = S.bnorm > 0 ? S.beta / S.bnorm : 0.0;
        S.m = 0;
        S.j = 0;
        // a cycle that made no iteration (breakdown) counts as a stall; three
        // stalls in a row, or a non-finite residual, end the instance unconverged
        if (S.cycle_iters == 0) S.stalls += 1;
        else if (S.cycle_iters > 0) S.stalls = 0;
        // a cycle that did not halve the true residual -- a full one of
        // STAGNATION_MIN_ITERS or more iterations, or one whose estimate
        // claimed convergence early -- shows that the network does not
        // precondition this instance, which continues under Jacobi
        const bool stagnated = S.cycle_iters > 0 && (S.cycle_iters >= STAGNATION_MIN_ITERS || S.cycle_iters < k) &&
                               S.relres > 0.5 * S.relres_prev;
        S.relres_prev = S.relres;
        if (S.relres <= S.tol || S.iters >= S.maxit || S.stalls >= 3 || !isfinite(S.relres)) {
            mark_done(S, ndone, res, sg.inst);
        } else {
            if (stagnated) set_fallback(S);
            S.active = 1;
            S.g[0] = S.beta;
            S.sig[0] = 1.0 / sqrt(sh[1]);
            S.v3n2 = sh[2];
        }
    }
}

// W (= V_{j+1} slot) dots: d_i = (W, V_i), i <= j, and ||W||^2.  JB >= j + 1
// bounds the basis length at compile time: every thread keeps the products of
// its elements with all basis vectors in registers, so the loads of all V_i
// are independent and in flight together (one memory-bound pass over the
// data), and the block reduces once at the end.
template <int JB>
__global__ void __launch_bounds__(MD_TB) k_dots(const Seg* __restrict__ seg, const InstRange* __restrict__ rng,
                                                const long long* __restrict__ off, const float* __restrict__ V,
                                                long long total, int j, int pass, KState* st, double* part) {
    constexpr int NW = MD_TB / 32;
    __shared__ double sh[(JB + 1) * NW];
    const Seg sg = seg[blockIdx.x];
    KState& S = st[sg.inst];
    if (!S.active || (pass == 1 && !S.reorth)) return;
    const long long o = off[sg.inst];
    const float* W = V + (long long)(j + 1) * total + o;
    const float* V0 = V + o;
    // U elements per thread and loop trip, so U x (j + 1) independent loads are
    // in flight before the first FMA needs one
    constexpr int U = JB <= 8 ? 4 : (JB <= 32 ? 2 : 1);
    float acc[JB + 1];
#pragma unroll
    for (int i = 0; i <= JB; ++i) acc[i] = 0.f;
    for (int e0 = sg.begin + threadIdx.x; e0 < sg.end; e0 += U * MD_TB) {
        float w[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * MD_TB;
            w[u] = e < sg.end ? W[e] : 0.f;
        }
        // all loads of the trip first: instructions issue in order, so an FMA
        // waiting on one load would hold back the loads behind it
        float x[JB][U];
#pragma unroll
        for (int i = 0; i < JB; ++i)
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = e0 + u * MD_TB;
                x[i][u] = (i <= j && e < sg.end) ? V0[(long long)i * total + e] : 0.f;
            }
#pragma unroll
        for (int i = 0; i < JB; ++i)
#pragma unroll
            for (int u = 0; u < U; ++u) acc[i] = fmaf(w[u], x[i][u], acc[i]);
#pragma unroll
        for (int u = 0; u < U; ++u) acc[JB] = fmaf(w[u], w[u], acc[JB]);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i <= JB; ++i) {
        if (i <= j || i == JB) {
            const double x = warp_sum((double)acc[i]);
            if (lane == 0) sh[i * NW + warp] = x;
        }
    }
    __syncthreads();
    const int cnt = j + 2;  // dots i = 0..j, then ||W||^2
    for (int r = threadIdx.x; r < cnt; r += blockDim.x) {
        const int src = r <= j ? r : JB;
        double s = 0.0;
        for (int w2 = 0; w2 < NW; ++w2) s += sh[src * NW + w2];
        part[(size_t)blockIdx.x * MD_MAXR + r] = s;
    }
    const InstRange rg = rng[sg.inst];
    if (!last_block_arrive(&S.counter[2], rg.count)) return;
    double* H = S.H + (size_t)j * (MD_KMAX + 1);
    for (int r = threadIdx.x; r < cnt; r += blockDim.x) {
        double s = 0.0;
        for (int b2 = rg.first; b2 < rg.first + rg.count; ++b2) s += part[(size_t)b2 * MD_MAXR + r];
        if (r <= j) {
            const double h = S.sig[j] * S.sig[r] * s;
            if (pass == 0) H[r] = h; else H[r] += h;
            S.coef[r] = S.sig[r] * S.sig[r] * s;
        } else if (pass == 0) {
            S.wn2_before = s;
        }
    }
}

// W -= sum_i coef_i V_i ; ||W||^2, ||W_3D||^2.  As k_dots: the basis length is
// bounded by JB at compile time so the loads of all V_i are issued together.
// In the first pass the same trip also forms the dots (W_new, V_i) of the
// second, re-orthogonalising pass from the V_i already in registers, so that
// pass needs no separate multi-dot over the basis: when ||W|| dropped below
// half of its length before the pass (the CGS2 condition), the last block
// adds them to column j of H and makes them the second pass's coefficients;
// otherwise it ends the step (H[j+1][j], sig_{j+1}).  The second pass
// (pass = 1, only where the condition fired) applies them and ends the step.
template <int JB, int PASS>
__global__ void __launch_bounds__(MD_TB) k_update(const Seg* __restrict__ seg, const InstRange* __restrict__ rng,
                                                  const long long* __restrict__ off, const InstDesc* __restrict__ D,
                                                  float* V, long long total, int j, KState* st, double* part) {
    constexpr int NW = MD_TB / 32;
    constexpr int pass = PASS;
    __shared__ double sh[(JB + 2) * NW];
    __shared__ float sc[JB];
    const Seg sg = seg[blockIdx.x];
    KState& S = st[sg.inst];
    if (!S.active || (pass == 1 && !S.reorth)) return;
    for (int i = threadIdx.x; i < JB; i += blockDim.x) sc[i] = i <= j ? (float)S.coef[i] : 0.f;
    __syncthreads();
    const long long o = off[sg.inst];
    const int n3 = D[sg.inst].n3;
    float* W = V + (long long)(j + 1) * total + o;
    const float* V0 = V + o;
    constexpr int U = JB <= 8 ? 4 : (JB <= 16 ? 2 : 1);
    // the second pass forms no dots (compiled without their registers)
    constexpr bool dots2 = PASS == 0;
    float a = 0.f, a3 = 0.f;
    float acc[JB];
#pragma unroll
    for (int i = 0; i < JB; ++i) acc[i] = 0.f;
    for (int e0 = sg.begin + threadIdx.x; e0 < sg.end; e0 += U * MD_TB) {
        float w[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * MD_TB;
            w[u] = e < sg.end ? W[e] : 0.f;
        }
        float x[JB][U];
#pragma unroll
        for (int i = 0; i < JB; ++i)
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = e0 + u * MD_TB;
                x[i][u] = (i <= j && e < sg.end) ? V0[(long long)i * total + e] : 0.f;
            }
#pragma unroll
        for (int i = 0; i < JB; ++i)
#pragma unroll
            for (int u = 0; u < U; ++u) w[u] = fmaf(-sc[i], x[i][u], w[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * MD_TB;
            if (e < sg.end) {
                W[e] = w[u];
                a = fmaf(w[u], w[u], a);
                if (e < n3) a3 = fmaf(w[u], w[u], a3);
            }
        }
        if (dots2) {
            // out-of-range lanes hold w = x = 0 and add nothing
#pragma unroll
            for (int i = 0; i < JB; ++i)
#pragma unroll
                for (int u = 0; u < U; ++u) acc[i] = fmaf(w[u], x[i][u], acc[i]);
        }
    }
    // block sums: slots 0, 1 = ||W||^2, ||W_3D||^2; 2 + i = (W, V_i), i <= j
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cnt = dots2 ? j + 3 : 2;
    {
        const double x0 = warp_sum((double)a), x1 = warp_sum((double)a3);
        if (lane == 0) { sh[warp] = x0; sh[NW + warp] = x1; }
    }
    if (dots2) {
#pragma unroll
        for (int i = 0; i < JB; ++i) {
            if (i <= j) {
                const double x = warp_sum((double)acc[i]);
                if (lane == 0) sh[(2 + i) * NW + warp] = x;
            }
        }
    }
    __syncthreads();
    for (int r = threadIdx.x; r < cnt; r += blockDim.x) {
        double sum = 0.0;
        for (int w2 = 0; w2 < NW; ++w2) sum += sh[r * NW + w2];
        part[(size_t)blockIdx.x * MD_MAXR + r] = sum;
    }
    const InstRange rg = rng[sg.inst];
    if (!last_block_arrive(&S.counter[3], rg.count)) return;
    __shared__ double tot[2];
    for (int r = threadIdx.x; r < 2; r += blockDim.x) {
        double sum = 0.0;
        for (int b2 = rg.first; b2 < rg.first + rg.count; ++b2) sum += part[(size_t)b2 * MD_MAXR + r];
        tot[r] = sum;
    }
    __syncthreads();
    const double wn2 = tot[0];
    if (dots2 && wn2 < 0.25 * S.wn2_before && wn2 > 0.0) {
        // second pass: its dots are this launch's (W_new, V_i)
        double* H = S.H + (size_t)j * (MD_KMAX + 1);
        for (int r = 2 + threadIdx.x; r < cnt; r += blockDim.x) {
            double sum = 0.0;
            for (int b2 = rg.first; b2 < rg.first + rg.count; ++b2) sum += part[(size_t)b2 * MD_MAXR + r];
            const int i = r - 2;
            H[i] += S.sig[j] * S.sig[i] * sum;
            S.coef[i] = S.sig[i] * S.sig[i] * sum;
        }
        if (threadIdx.x == 0) {
            S.reorth = 1;
            S.wn2_before = wn2;
        }
    } else if (threadIdx.x == 0) {
        S.reorth = 0;
        S.H[(size_t)j * (MD_KMAX + 1) + j + 1] = S.sig[j] * sqrt(wn2);
        S.sig[j + 1] = wn2 > 0.0 ? 1.0 / sqrt(wn2) : 0.0;
        S.v3n2 = tot[1];
    }
}

// One Arnoldi step's Gram-Schmidt with the basis-length bound that covers
// j + 1 vectors: the multi-dot, the update (with the second pass's dots), and
// the second pass's update where the re-orthogonalisation condition fired.
template <int JB>
static void launch_gs_step(md_batch* B, int j, cudaStream_t s) {
    const Tables& T = B->tabs;
    k_dots<JB><<<T.vec.nblocks, MD_TB, 0, s>>>(T.vec.seg, T.vec.range, B->off, B->V, B->total, j, 0, B->st, B->part);
    k_update<JB, 0><<<T.vec.nblocks, MD_TB, 0, s>>>(T.vec.seg, T.vec.range, B->off, B->d, B->V, B->total, j, B->st,
                                                    B->part);
    k_update<JB, 1><<<T.vec.nblocks, MD_TB, 0, s>>>(T.vec.seg, T.vec.range, B->off, B->d, B->V, B->total, j, B->st,
                                                    B->part);
}
static void launch_gs(md_batch* B, int j, cudaStream_t s) {
    if (j < 8) launch_gs_step<8>(B, j, s);
    else if (j < 16) launch_gs_step<16>(B, j, s);
    else if (j < 24) launch_gs_step<24>(B, j, s);
    else if (j < 32) launch_gs_step<32>(B, j, s);
    else launch_gs_step<MD_KMAX>(B, j, s);
}

// Givens rotations, residual estimate, cycle exit; one thread per instance
__global__ void k_givens(KState* st, int ninst, int j, int k) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ninst) return;
    KState& S = st[i];
    if (!S.active) return;
    double* H = S.H + (size_t)j * (MD_KMAX + 1);
    const double hlast = H[j + 1];
    for (int r = 0; r < j; ++r) {
        const double t = S.cs[r] * H[r] + S.sn[r] * H[r + 1];
        H[r + 1] = -S.sn[r] * H[r] + S.cs[r] * H[r + 1];
        H[r] = t;
    }
    const double den = hypot(H[j], H[j + 1]);
    if (den == 0.0 || !isfinite(den)) {
        // breakdown: keep the columns before j; a preconditioner that gave no
        // usable direction (or a non-finite one) is replaced by Jacobi for the
        // rest of this instance's solve
        S.active = 0;
        S.nan_seen |= !isfinite(den);
        if (j == 0 || !isfinite(den)) set_fallback(S);
        return;
    }
    S.cs[j] = H[j] / den;
    S.sn[j] = H[j + 1] / den;
    H[j] = den;
    H[j + 1] = 0.0;
    S.g[j + 1] = -S.sn[j] * S.g[j];
    S.g[j] = S.cs[j] * S.g[j];
    S.est = fabs(S.g[j + 1]);
    S.iters += 1;
    S.m = j + 1;
    if (S.est <= S.tol * S.bnorm || S.est <= S.inner_tol * S.beta || S.iters >= S.maxit || j + 1 == k ||
        hlast == 0.0)
        S.active = 0;
}

// H y = g on the m columns of this cycle; coef_i = y_i sig_i
__global__ void k_lsq(KState* st, int ninst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ninst) return;
    KState& S = st[i];
    S.active = 0;
    S.cycle_iters = S.t_done ? 0 : S.m;
    if (S.t_done || S.m == 0) return;
    const int m = S.m;
    for (int r = m - 1; r >= 0; --r) {
        double s = S.g[r];
        for (int l = r + 1; l < m; ++l) s -= S.H[(size_t)l * (MD_KMAX + 1) + r] * S.y[l];
        S.y[r] = s / S.H[(size_t)r * (MD_KMAX + 1) + r];
    }
    for (int r = 0; r < m; ++r) S.coef[r] = S.y[r] * S.sig[r];
}

// x += sum_i coef_i Z_i  (FP32 correction, FP64 x)
__global__ void __launch_bounds__(MD_TB) k_xupd(const Seg* __restrict__ seg, const long long* __restrict__ off,
                                                const float* __restrict__ Z, long long total, double* x, const KState* st) {
    __shared__ float sc[MD_KMAX];
    const Seg sg = seg[blockIdx.x];
    const KState& S = st[sg.inst];
    if (S.t_done || S.m == 0) return;
    const int m = S.m;
    for (int i = threadIdx.x; i < m; i += blockDim.x) sc[i] = (float)S.coef[i];
    __syncthreads();
    const long long o = off[sg.inst];
    for (int e = sg.begin + threadIdx.x; e < sg.end; e += blockDim.x) {
        float c = 0.f;
        for (int i = 0; i < m; ++i) c = fmaf(sc[i], Z[(long long)i * total + o + e], c);
        x[o + e] += (double)c;
    }
}

// ---- preconditioner kernels ---------------------------------------------------
// Jacobi: Z = diag(A)^{-1} V
__global__ void __launch_bounds__(MD_TB) k_jacobi(const Seg* __restrict__ seg, const long long* __restrict__ off,
                                                  const InstDesc* __restrict__ D, const float* __restrict__ v, float* z,
                                                  const KState* st, int only_fallback) {
    const Seg sg = seg[blockIdx.x];
    if (st && (!st[sg.inst].active || (only_fallback && !st[sg.inst].fallback))) return;
    const long long o = off[sg.inst];
    const float* dinv = D[sg.inst].dinv32;
    for (int e = sg.begin + threadIdx.x; e < sg.end; e += blockDim.x) z[o + e] = dinv[e] * v[o + e];
}

// Shared memory of the tree kernels for n1 1D nodes: y, the factor l and
// 1/d (floats), the parents and the level schedule (ints): 10 n1 + 3 words.
__host__ __device__ inline size_t tree_smem_bytes(int n1) { return (10 * (size_t)n1 + 3) * 4; }

struct TreeSm {
    float *y, *sl, *sdi;
    int *spar, *lv_up, *ch_ptr, *ch_idx, *lv_dn, *lvu_ptr, *lvd_ptr;
};

// Carve the tree arrays out of `raw` and copy the factor and its schedule in.
__device__ inline TreeSm tree_load(unsigned char* raw, const InstDesc& d) {
    const int n1 = d.n1;
    TreeSm t;
    t.y = reinterpret_cast<float*>(raw);
    t.sl = t.y + n1;
    t.sdi = t.sl + n1;
    t.spar = reinterpret_cast<int*>(t.sdi + n1);
    t.lv_up = t.spar + n1;
    t.ch_ptr = t.lv_up + n1;
    t.ch_idx = t.ch_ptr + n1 + 1;
    t.lv_dn = t.ch_idx + n1;
    t.lvu_ptr = t.lv_dn + n1;
    t.lvd_ptr = t.lvu_ptr + n1 + 1;
    const int nch = d.ch_ptr[n1];
    for (int i = threadIdx.x; i < n1; i += blockDim.x) {
        t.sl[i] = d.tr_l32[i];
        t.sdi[i] = d.tr_dinv32[i];
        t.spar[i] = d.tr_parent[i];
        t.lv_up[i] = d.lv_up[i];
        t.lv_dn[i] = d.lv_dn[i];
    }
    for (int i = threadIdx.x; i <= n1; i += blockDim.x) t.ch_ptr[i] = d.ch_ptr[i];
    for (int i = threadIdx.x; i < nch; i += blockDim.x) t.ch_idx[i] = d.ch_idx[i];
    for (int i = threadIdx.x; i <= d.nlvu; i += blockDim.x) t.lvu_ptr[i] = d.lvu_ptr[i];
    for (int i = threadIdx.x; i <= d.nlvd; i += blockDim.x) t.lvd_ptr[i] = d.lvd_ptr[i];
    return t;
}

// Tree LDL^T solve in place on t.y (length n1, shared memory), level by
// level so that the whole block works on every sweep: forward (leaves to
// roots) by height, each node taking y_i -= sum over its children c of
// l_c y_c once all of them are final; the diagonal scaling; backward (roots
// to leaves) by depth, y_i -= l_i y_parent(i).  The caller synchronises the
// block after writing y.
__device__ inline void tree_solve_levels(const InstDesc& d, const TreeSm& t) {
    for (int h = 0; h < d.nlvu; ++h) {
        for (int k = t.lvu_ptr[h] + threadIdx.x; k < t.lvu_ptr[h + 1]; k += blockDim.x) {
            const int i = t.lv_up[k];
            float acc = t.y[i];
            for (int c = t.ch_ptr[i]; c < t.ch_ptr[i + 1]; ++c) {
                const int ch = t.ch_idx[c];
                acc -= t.sl[ch] * t.y[ch];
            }
            t.y[i] = acc;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < d.n1; i += blockDim.x) t.y[i] *= t.sdi[i];
    __syncthreads();
    for (int k = 1; k < d.nlvd; ++k) {
        for (int e = t.lvd_ptr[k] + threadIdx.x; e < t.lvd_ptr[k + 1]; e += blockDim.x) {
            const int i = t.lv_dn[e];
            t.y[i] -= t.sl[i] * t.y[t.spar[i]];
        }
        __syncthreads();
    }
}

// Lower block order: the network input scale is s = ||v0|| (no lifted 1D part).
__global__ void k_lower_setup(KState* st, int ninst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ninst) return;
    KState& S = st[i];
    if (!S.active || S.fallback) return;
    S.s2_touch = 0.0;
    S.s = S.v3n2 > 0.0 ? sqrt(S.v3n2) : 0.0;
}

// Lower block order, the averaging of the network's output at the quadrature
// points, t_q = (Pi z0)(q), into the instance's t scratch: one thread per
// point over the whole batch (the quadrature-point table of the apply).
__global__ void __launch_bounds__(MD_TB) k_gather_z0(const InstDesc* __restrict__ D, const Seg* __restrict__ seg,
                                                     const long long* __restrict__ off, const float* __restrict__ z,
                                                     const KState* st) {
    const Seg sg = seg[blockIdx.x];
    if (!cnn_runs(st, sg.inst)) return;
    const InstDesc& d = D[sg.inst];
    const float* z0 = z + off[sg.inst];
    for (int q = sg.begin + threadIdx.x; q < sg.end; q += blockDim.x)
        d.t32[q] = csr_row<float, float>(d.pi_col, d.pi_v32, d.pi_ptr[q], d.pi_ptr[q + 1], z0);
}

// Lower block order, 1D part after the network: z1 = B11^{-1} (v1 + beta Psi^T W Pi z0),
// i.e. v1 minus the 1-0 block of A applied to z0 (Pi z0 from k_gather_z0,
// then the Psi^T W rows, then the tree solve in shared memory).
__global__ void __launch_bounds__(TREE_TB) k_lower_1d(const InstDesc* __restrict__ D, const long long* __restrict__ off,
                                                      const float* __restrict__ v, float* z, const KState* st) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int inst = blockIdx.x;
    const KState& S = st[inst];
    if (!S.active || S.fallback) return;
    const InstDesc& d = D[inst];
    const int n1 = d.n1;
    const TreeSm tr = tree_load(smraw, d);
    float* y = tr.y;
    const float* t = d.t32;  // (Pi z0)(q), k_gather_z0
    const long long o = off[inst];
    const float beta = (float)d.beta;
    const float* v1 = v + o + d.n3;
    for (int i = threadIdx.x; i < n1; i += blockDim.x)
        y[i] = v1[i] + beta * csr_row<float, float>(d.pw_q, d.pw_v32, d.pw_ptr[i], d.pw_ptr[i + 1], t);
    __syncthreads();
    tree_solve_levels(d, tr);
    float* z1 = z + o + d.n3;
    for (int i = threadIdx.x; i < n1; i += blockDim.x) z1[i] = y[i];
}

// 1D block solve z1 = B11^{-1} v1 (tree LDL^T sweeps in shared memory), one
// block per instance.  It also sets the network's input scale to
// s = ||v0||, which k_lift then corrects for the lifted part.
__global__ void __launch_bounds__(TREE_TB) k_tree_1d(const InstDesc* __restrict__ D, const long long* __restrict__ off,
                                                 const float* __restrict__ v, float* z, KState* st) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int inst = blockIdx.x;
    KState& S = st[inst];
    if (!S.active || S.fallback) return;
    const InstDesc& d = D[inst];
    const int n1 = d.n1;
    const TreeSm tr = tree_load(smraw, d);
    float* y = tr.y;
    const long long o = off[inst];
    const float* v1 = v + o + d.n3;
    for (int i = threadIdx.x; i < n1; i += blockDim.x) y[i] = v1[i];
    __syncthreads();
    tree_solve_levels(d, tr);
    float* z1 = z + o + d.n3;
    for (int i = threadIdx.x; i < n1; i += blockDim.x) z1[i] = y[i];
    if (threadIdx.x == 0) {
        S.s2_touch = 0.0;
        S.s = S.v3n2 > 0.0 ? sqrt(S.v3n2) : 0.0;
    }
}

// The lift l = beta Pi^T W Psi z1 on the grid nodes the averaging reaches
// (z1 in z's 1D part), one thread per node over the whole batch (the
// touched-node table), into the instance's lift buffers; and the network's
// input scale s = ||v0 + l||: ||v0||^2 (st.v3n2) plus sum (2 v0 l + l^2)
// over those nodes, the last block of an instance storing s.
__global__ void __launch_bounds__(MD_TB) k_lift(const Seg* __restrict__ seg, const InstRange* __restrict__ rng,
                                                const long long* __restrict__ off, const InstDesc* __restrict__ D,
                                                const float* __restrict__ v, const float* __restrict__ z, KState* st,
                                                double* part) {
    __shared__ double sh[32 * 4];
    const Seg sg = seg[blockIdx.x];
    KState& S = st[sg.inst];
    if (!S.active || S.fallback) return;
    const InstDesc& d = D[sg.inst];
    const long long o = off[sg.inst];
    const float* z1 = z + o + d.n3;
    const float* v0 = v + o;
    const float beta = (float)d.beta;
    double vals[1] = {0.0};
    for (int idx = sg.begin + threadIdx.x; idx < sg.end; idx += blockDim.x) {
        float acc = 0.f;
        for (int jj = d.tn_ptr[idx]; jj < d.tn_ptr[idx + 1]; ++jj) {
            const int q = d.tn_q[jj];
            acc += d.tn_v32[jj] * (d.psa32[q] * z1[d.qa[q]] + d.psb32[q] * z1[d.qb[q]]);
        }
        const float l = beta * acc;
        const int node = d.tn_node[idx];
        d.ltouch32[idx] = l;
        d.lift32[node] = l;
        const float vv = v0[node];
        vals[0] += (double)(2.f * vv * l + l * l);
    }
    double flag;
    reduce_values<1>(vals, 1, part, blockIdx.x, rng[sg.inst], &S.counter[8], &flag, sh);
    if (flag == 1.0 && threadIdx.x == 0) {
        S.s2_touch = sh[0];
        const double s2 = S.v3n2 + sh[0];
        S.s = s2 > 0.0 ? sqrt(s2) : 0.0;
    }
}

// The 1D part of the block preconditioner in the upper order (z1 and the
// lift with the input scale) and in the lower order (z1 from the network's
// z0), for every instance that runs the network.
static md_status launch_upper_1d(const Tables& T, const InstDesc* d, const long long* off, int ninst, int max_n1,
                                 const float* v, float* z, KState* st, double* part, cudaStream_t s) {
    k_tree_1d<<<ninst, TREE_TB, tree_smem_bytes(max_n1), s>>>(d, off, v, z, st);
    MD_CHECK_LAUNCH();
    if (T.touch.nblocks > 0) {
        k_lift<<<T.touch.nblocks, MD_TB, 0, s>>>(T.touch.seg, T.touch.range, off, d, v, z, st, part);
        MD_CHECK_LAUNCH();
    }
    return MD_OK;
}

static md_status launch_lower_1d(md_batch* B, const float* v, float* z, cudaStream_t s);

// ---- Jacobi pre- and post-smoothing around the 3D solve (Section 5, 'Effect of
// pre- and post-smoothing') --------------------------------------------------------
// The 3D part of Z holds the smoothing iterate x.  Its 1D part holds z1 in the
// upper order, so the 3D part of A Z is C x - l, and zero in the lower order,
// where it is C x: in both orders the residual of the 3D solve, b0 - C x, is
// r0 - (A Z)_0, and one operator apply serves every sweep.

// The smoothing kernels stream three or four vectors over the long segments of
// the Krylov tables: each thread issues the loads of SM_U elements before any
// arithmetic, so a block keeps SM_U x 256 loads in flight per array.
#define SM_U 8

// D^{-1} below is the smoother's row scaling rho_i / c_ii (InstDesc::sminv32):
// 1 / c_ii on the stencil rows, less on rows the coupling makes heavy.
// First sweep from x = 0: x = omega D^{-1} b0 (b0 = r0 + l, or r0 in the lower
// order, which also clears the 1D part of Z).  Whole-vector segments.
__global__ void __launch_bounds__(MD_TB) k_smooth_first(const Seg* __restrict__ seg, const long long* __restrict__ off,
                                                        const InstDesc* __restrict__ D, const float* __restrict__ v,
                                                        float* z, const KState* st, float omega, int use_lift) {
    const Seg sg = seg[blockIdx.x];
    if (!cnn_runs(st, sg.inst)) return;
    const InstDesc& d = D[sg.inst];
    const long long o = off[sg.inst];
    const int n3 = d.n3;
    const float* vi = v + o;
    float* zi = z + o;
    for (int e0 = sg.begin + threadIdx.x; e0 < sg.end; e0 += SM_U * MD_TB) {
        float b[SM_U], w[SM_U];
#pragma unroll
        for (int u = 0; u < SM_U; ++u) {
            const int e = e0 + u * MD_TB;
            const bool in3 = e < sg.end && e < n3;
            b[u] = in3 ? vi[e] : 0.f;
            w[u] = in3 ? d.sminv32[e] : 0.f;
            if (in3 && use_lift) b[u] += d.lift32[e];
        }
#pragma unroll
        for (int u = 0; u < SM_U; ++u) {
            const int e = e0 + u * MD_TB;
            if (e >= sg.end) continue;
            if (e < n3) zi[e] = omega * w[u] * b[u];
            else if (!use_lift) zi[e] = 0.f;
        }
    }
}

// One sweep x += omega D^{-1} (r0 - (A Z)_0), az = A Z.  3D segments.
__global__ void __launch_bounds__(MD_TB) k_smooth_sweep(const Seg* __restrict__ seg, const long long* __restrict__ off,
                                                        const InstDesc* __restrict__ D, const float* __restrict__ v,
                                                        const float* __restrict__ az, float* z, const KState* st,
                                                        float omega) {
    const Seg sg = seg[blockIdx.x];
    if (!cnn_runs(st, sg.inst)) return;
    const long long o = off[sg.inst];
    const float* dinv = D[sg.inst].sminv32;
    const float* vi = v + o;
    const float* ai = az + o;
    float* zi = z + o;
    for (int e0 = sg.begin + threadIdx.x; e0 < sg.end; e0 += SM_U * MD_TB) {
        float r[SM_U], a[SM_U], w[SM_U], x[SM_U];
#pragma unroll
        for (int u = 0; u < SM_U; ++u) {
            const int e = e0 + u * MD_TB;
            const bool in = e < sg.end;
            r[u] = in ? vi[e] : 0.f;
            a[u] = in ? ai[e] : 0.f;
            w[u] = in ? dinv[e] : 0.f;
            x[u] = in ? zi[e] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < SM_U; ++u) {
            const int e = e0 + u * MD_TB;
            if (e < sg.end) zi[e] = x[u] + omega * w[u] * (r[u] - a[u]);
        }
    }
}

// Input of the network correction, in place over t = A Z: the 3D residual
// res = r0 - (A Z)_0 = b0 - C x goes to the network as [(res - l)/s, l/s, d]
// (the lifted part keeps its own channel; l = 0 in the lower order), with
// s = ||res||.  3D segments; the last block of an instance stores s.
__global__ void __launch_bounds__(MD_TB) k_smooth_resid(const Seg* __restrict__ seg, const InstRange* __restrict__ rng,
                                                        const long long* __restrict__ off,
                                                        const InstDesc* __restrict__ D, const float* __restrict__ v,
                                                        float* t, KState* st, double* part, int use_lift) {
    __shared__ double sh[32 * 4];
    const Seg sg = seg[blockIdx.x];
    if (!cnn_runs(st, sg.inst)) return;
    KState& S = st[sg.inst];
    const InstDesc& d = D[sg.inst];
    const long long o = off[sg.inst];
    const float* vi = v + o;
    float* ti = t + o;
    float acc = 0.f;
    for (int e0 = sg.begin + threadIdx.x; e0 < sg.end; e0 += SM_U * MD_TB) {
        float r[SM_U], a[SM_U], l[SM_U];
#pragma unroll
        for (int u = 0; u < SM_U; ++u) {
            const int e = e0 + u * MD_TB;
            const bool in = e < sg.end;
            r[u] = in ? vi[e] : 0.f;
            a[u] = in ? ti[e] : 0.f;
            l[u] = (in && use_lift) ? d.lift32[e] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < SM_U; ++u) {
            const int e = e0 + u * MD_TB;
            const float res = r[u] - a[u];
            acc = fmaf(res, res, acc);
            if (e < sg.end) ti[e] = res - l[u];
        }
    }
    double vals[1] = {(double)acc};
    double flag;
    reduce_values<1>(vals, 1, part, blockIdx.x, rng[sg.inst], &S.counter[5], &flag, sh);
    if (flag == 1.0 && threadIdx.x == 0) S.s = sh[0] > 0.0 ? sqrt(sh[0]) : 0.0;
}

// x += the network's correction (3D segments).
__global__ void __launch_bounds__(MD_TB) k_smooth_add(const Seg* __restrict__ seg, const long long* __restrict__ off,
                                                      const float* __restrict__ t, float* z, const KState* st) {
    const Seg sg = seg[blockIdx.x];
    if (!cnn_runs(st, sg.inst)) return;
    const long long o = off[sg.inst];
    const float* ti = t + o;
    float* zi = z + o;
    for (int e0 = sg.begin + threadIdx.x; e0 < sg.end; e0 += SM_U * MD_TB) {
        float a[SM_U], x[SM_U];
#pragma unroll
        for (int u = 0; u < SM_U; ++u) {
            const int e = e0 + u * MD_TB;
            const bool in = e < sg.end;
            a[u] = in ? ti[e] : 0.f;
            x[u] = in ? zi[e] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < SM_U; ++u) {
            const int e = e0 + u * MD_TB;
            if (e < sg.end) zi[e] = x[u] + a[u];
        }
    }
}

// ---- the 3D block solve as m steps of flexible GMRES on C (Section 6: '3 steps
// of P-FGMRES' as the 3D solve of the block preconditioner) -------------------------
// Per instance, basis vectors iV_0..iV_m and directions iZ_j = N(iV_j), whole
// length; the 1D parts of iZ stay zero, so the operator apply gives C iZ_j in
// the 3D part.  iZ_0 is the network on the block's own input ([r0/s, l/s, d]),
// iV_0 = b0 / s; W = C iZ_j is orthogonalised against iV_0..iV_j by two
// classical Gram-Schmidt passes (FP64 sums per instance), iV_{j+1} = W / ||W||,
// and iZ_{j+1} is the network on [iV_{j+1}, 0, d].  After m steps
// z0 = sum_j y_j iZ_j, y the FP64 least-squares solution of min ||s e_1 - H y||.

// iV_0 = b0 / s (b0 = r0 + l, or r0 in the lower order), iZ_0 /= s, H = 0.
__global__ void __launch_bounds__(MD_TB) k_inner_start(const Seg* __restrict__ seg, const long long* __restrict__ off,
                                                       const InstDesc* __restrict__ D, const float* __restrict__ v,
                                                       float* iv0, float* iz0, KState* st, int use_lift) {
    const Seg sg = seg[blockIdx.x];
    if (!cnn_runs(st, sg.inst)) return;
    KState& S = st[sg.inst];
    const InstDesc& d = D[sg.inst];
    const long long o = off[sg.inst];
    const double s = S.s;
    const float inv = s > 0.0 ? (float)(1.0 / s) : 0.f;
    if (sg.begin == 0) {
        for (int i = threadIdx.x; i < (MD_INNER_MAX + 1) * MD_INNER_MAX; i += blockDim.x) S.iH[i] = 0.0;
        if (threadIdx.x == 0) S.ib0 = s;
    }
    for (int e0 = sg.begin + threadIdx.x; e0 < sg.end; e0 += SM_U * MD_TB) {
        float b[SM_U], z[SM_U];
#pragma unroll
        for (int u = 0; u < SM_U; ++u) {
            const int e = e0 + u * MD_TB;
            const bool in = e < sg.end;
            b[u] = in ? v[o + e] : 0.f;
            z[u] = in ? iz0[o + e] : 0.f;
            if (in && use_lift) b[u] += d.lift32[e];
        }
#pragma unroll
        for (int u = 0; u < SM_U; ++u) {
            const int e = e0 + u * MD_TB;
            if (e < sg.end) {
                iv0[o + e] = b[u] * inv;
                iz0[o + e] = z[u] * inv;
            }
        }
    }
}

// (W, iV_i) for i <= j over the 3D part, W = iV_{j+1}; the instance's last
// block stores them as this pass's coefficients and adds them to column j of H.
__global__ void __launch_bounds__(MD_TB) k_inner_dots(const Seg* __restrict__ seg, const InstRange* __restrict__ rng,
                                                      const long long* __restrict__ off, const float* __restrict__ iV,
                                                      long long total, int j, KState* st, double* part) {
    __shared__ double sh[32 * MD_INNER_MAX];
    const Seg sg = seg[blockIdx.x];
    if (!cnn_runs(st, sg.inst)) return;
    KState& S = st[sg.inst];
    const long long o = off[sg.inst];
    const float* W = iV + (long long)(j + 1) * total + o;
    const float* V0 = iV + o;
    constexpr int U = 2;
    float acc[MD_INNER_MAX];
#pragma unroll
    for (int i = 0; i < MD_INNER_MAX; ++i) acc[i] = 0.f;
    for (int e0 = sg.begin + threadIdx.x; e0 < sg.end; e0 += U * MD_TB) {
        float w[U], x[MD_INNER_MAX][U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * MD_TB;
            w[u] = e < sg.end ? W[e] : 0.f;
        }
#pragma unroll
        for (int i = 0; i < MD_INNER_MAX; ++i)
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = e0 + u * MD_TB;
                x[i][u] = (i <= j && e < sg.end) ? V0[(long long)i * total + e] : 0.f;
            }
#pragma unroll
        for (int i = 0; i < MD_INNER_MAX; ++i)
#pragma unroll
            for (int u = 0; u < U; ++u) acc[i] = fmaf(w[u], x[i][u], acc[i]);
    }
    double vals[MD_INNER_MAX];
#pragma unroll
    for (int i = 0; i < MD_INNER_MAX; ++i) vals[i] = (double)acc[i];
    double flag;
    reduce_values<MD_INNER_MAX>(vals, j + 1, part, blockIdx.x, rng[sg.inst], &S.counter[6], &flag, sh);
    if (flag == 1.0) {
        for (int r = threadIdx.x; r <= j; r += blockDim.x) {
            S.icoef[r] = sh[r];
            S.iH[(size_t)j * (MD_INNER_MAX + 1) + r] += sh[r];
        }
    }
}

// W -= sum_{i<=j} coef_i iV_i over the 3D part and ||W||^2; after the second
// pass the last block stores H[j+1, j] = ||W|| and sets the network's input
// scale to 1 for the normalised iV_{j+1}.
__global__ void __launch_bounds__(MD_TB) k_inner_update(const Seg* __restrict__ seg, const InstRange* __restrict__ rng,
                                                        const long long* __restrict__ off, float* iV, long long total,
                                                        int j, int pass, KState* st, double* part) {
    __shared__ double sh[32 * 4];
    __shared__ float sc[MD_INNER_MAX];
    const Seg sg = seg[blockIdx.x];
    if (!cnn_runs(st, sg.inst)) return;
    KState& S = st[sg.inst];
    if (threadIdx.x < MD_INNER_MAX) sc[threadIdx.x] = (int)threadIdx.x <= j ? (float)S.icoef[threadIdx.x] : 0.f;
    __syncthreads();
    const long long o = off[sg.inst];
    float* W = iV + (long long)(j + 1) * total + o;
    const float* V0 = iV + o;
    constexpr int U = 2;
    float a = 0.f;
    for (int e0 = sg.begin + threadIdx.x; e0 < sg.end; e0 += U * MD_TB) {
        float w[U], x[MD_INNER_MAX][U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * MD_TB;
            w[u] = e < sg.end ? W[e] : 0.f;
        }
#pragma unroll
        for (int i = 0; i < MD_INNER_MAX; ++i)
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = e0 + u * MD_TB;
                x[i][u] = (i <= j && e < sg.end) ? V0[(long long)i * total + e] : 0.f;
            }
#pragma unroll
        for (int i = 0; i < MD_INNER_MAX; ++i)
#pragma unroll
            for (int u = 0; u < U; ++u) w[u] = fmaf(-sc[i], x[i][u], w[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * MD_TB;
            if (e < sg.end) {
                W[e] = w[u];
                a = fmaf(w[u], w[u], a);
            }
        }
    }
    double vals[1] = {(double)a};
    double flag;
    reduce_values<1>(vals, 1, part, blockIdx.x, rng[sg.inst], &S.counter[7], &flag, sh);
    if (flag == 1.0 && threadIdx.x == 0 && pass == 1) {
        S.iH[(size_t)j * (MD_INNER_MAX + 1) + j + 1] = sqrt(sh[0]);
        S.s = 1.0;
    }
}

// iV_{j+1} = W / H[j+1, j] (zero after a breakdown).
__global__ void __launch_bounds__(MD_TB) k_inner_scale(const Seg* __restrict__ seg, const long long* __restrict__ off,
                                                       float* iV, long long total, int j, const KState* st) {
    const Seg sg = seg[blockIdx.x];
    if (!cnn_runs(st, sg.inst)) return;
    const double h = st[sg.inst].iH[(size_t)j * (MD_INNER_MAX + 1) + j + 1];
    const float inv = h > 0.0 ? (float)(1.0 / h) : 0.f;
    float* W = iV + (long long)(j + 1) * total + off[sg.inst];
    for (int e0 = sg.begin + threadIdx.x; e0 < sg.end; e0 += SM_U * MD_TB) {
        float w[SM_U];
#pragma unroll
        for (int u = 0; u < SM_U; ++u) {
            const int e = e0 + u * MD_TB;
            w[u] = e < sg.end ? W[e] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < SM_U; ++u) {
            const int e = e0 + u * MD_TB;
            if (e < sg.end) W[e] = w[u] * inv;
        }
    }
}

// Givens rotations on the (m+1) x m Hessenberg and back substitution for
// min ||s e_1 - H y||; one thread per instance.
__global__ void k_inner_lsq(KState* st, int ninst, int m) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ninst || !cnn_runs(st, i)) return;
    KState& S = st[i];
    double H[(MD_INNER_MAX + 1) * MD_INNER_MAX];
    double g[MD_INNER_MAX + 1], cs[MD_INNER_MAX], sn[MD_INNER_MAX];
    for (int r = 0; r < (MD_INNER_MAX + 1) * MD_INNER_MAX; ++r) H[r] = S.iH[r];
    for (int r = 0; r <= MD_INNER_MAX; ++r) g[r] = 0.0;
    g[0] = S.ib0;
    for (int j = 0; j < m; ++j) {
        double* col = H + j * (MD_INNER_MAX + 1);
        for (int r = 0; r < j; ++r) {
            const double t = cs[r] * col[r] + sn[r] * col[r + 1];
            col[r + 1] = -sn[r] * col[r] + cs[r] * col[r + 1];
            col[r] = t;
        }
        const double den = hypot(col[j], col[j + 1]);
        if (den > 0.0 && isfinite(den)) {
            cs[j] = col[j] / den;
            sn[j] = col[j + 1] / den;
        } else {
            cs[j] = 1.0;
            sn[j] = 0.0;
        }
        col[j] = cs[j] * col[j] + sn[j] * col[j + 1];
        col[j + 1] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
    }
    for (int r = m - 1; r >= 0; --r) {
        double t = g[r];
        for (int l = r + 1; l < m; ++l) t -= H[l * (MD_INNER_MAX + 1) + r] * S.iy[l];
        const double dgl = H[r * (MD_INNER_MAX + 1) + r];
        S.iy[r] = (dgl != 0.0 && isfinite(t / dgl)) ? t / dgl : 0.0;
    }
}

// z0 = sum_j y_j iZ_j (3D part).
__global__ void __launch_bounds__(MD_TB) k_inner_combine(const Seg* __restrict__ seg, const long long* __restrict__ off,
                                                         const float* __restrict__ iZ, long long total, float* z,
                                                         const KState* st, int m) {
    const Seg sg = seg[blockIdx.x];
    if (!cnn_runs(st, sg.inst)) return;
    const KState& S = st[sg.inst];
    float y[MD_INNER_MAX];
#pragma unroll
    for (int j = 0; j < MD_INNER_MAX; ++j) y[j] = j < m ? (float)S.iy[j] : 0.f;
    const long long o = off[sg.inst];
    for (int e0 = sg.begin + threadIdx.x; e0 < sg.end; e0 += 2 * MD_TB) {
        float x[MD_INNER_MAX][2];
#pragma unroll
        for (int j = 0; j < MD_INNER_MAX; ++j)
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int e = e0 + u * MD_TB;
                x[j][u] = (j < m && e < sg.end) ? iZ[(long long)j * total + o + e] : 0.f;
            }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int e = e0 + u * MD_TB;
            if (e >= sg.end) continue;
            float acc = 0.f;
#pragma unroll
            for (int j = 0; j < MD_INNER_MAX; ++j) acc = fmaf(y[j], x[j][u], acc);
            z[o + e] = acc;
        }
    }
}

// ||v0||^2 of a preconditioner input given from outside the solver
__global__ void __launch_bounds__(MD_TB) k_norm3(const Seg* __restrict__ seg, const InstRange* __restrict__ rng,
                                                 const long long* __restrict__ off, const float* __restrict__ v,
                                                 KState* st, double* part) {
    __shared__ double sh[32 * 4];
    const Seg sg = seg[blockIdx.x];
    KState& S = st[sg.inst];
    const float* vi = v + off[sg.inst];
    float a = 0.f;
    for (int e = sg.begin + threadIdx.x; e < sg.end; e += blockDim.x) a = fmaf(vi[e], vi[e], a);
    double vals[1] = {(double)a};
    double flag;
    reduce_values<1>(vals, 1, part, blockIdx.x, rng[sg.inst], &S.counter[4], &flag, sh);
    if (flag == 1.0 && threadIdx.x == 0) S.v3n2 = sh[0];
}

// ---- CG (FP64) -------------------------------------------------------------------
__global__ void __launch_bounds__(MD_TB) k_cg_init(const Seg* __restrict__ seg, const InstRange* __restrict__ rng,
                                                   const long long* __restrict__ off, const InstDesc* __restrict__ D,
                                                   const double* __restrict__ b, const double* __restrict__ y,
                                                   double* r, double* p, KState* st, double* part, int* ndone,
                                                   ResOut res) {
    __shared__ double sh[32 * 4];
    const Seg sg = seg[blockIdx.x];
    KState& S = st[sg.inst];
    const long long o = off[sg.inst];
    const double* dinv = D[sg.inst].dinv64;
    double v[2] = {0.0, 0.0};
    for (int e = sg.begin + threadIdx.x; e < sg.end; e += blockDim.x) {
        const double rr = b[o + e] - y[o + e];
        r[o + e] = rr;
        const double zz = dinv[e] * rr;
        p[o + e] = zz;
        v[0] += rr * zz;
        v[1] += rr * rr;
    }
    double flag;
    reduce_values<2>(v, 2, part, blockIdx.x, rng[sg.inst], &S.counter[1], &flag, sh);
    if (flag == 1.0 && threadIdx.x == 0) {
        S.rho = sh[0];
        S.relres = S.bnorm > 0 ? sqrt(sh[1]) / S.bnorm : 0.0;
        if (S.relres <= S.tol || S.iters >= S.maxit) mark_done(S, ndone, res, sg.inst);
        else S.active = 1;
    }
}

__global__ void __launch_bounds__(MD_TB) k_cg_alpha(const Seg* __restrict__ seg, const InstRange* __restrict__ rng,
                                                    const long long* __restrict__ off, const double* __restrict__ p,
                                                    const double* __restrict__ q, KState* st, double* part) {
    __shared__ double sh[32 * 4];
    const Seg sg = seg[blockIdx.x];
    KState& S = st[sg.inst];
    if (!S.active) return;
    const long long o = off[sg.inst];
    double v[1] = {0.0};
    // CG_U elements per thread and trip, loads before arithmetic (in-order issue)
    for (int e0 = sg.begin + threadIdx.x; e0 < sg.end; e0 += CG_U * MD_TB) {
        double pp[CG_U], qq[CG_U];
#pragma unroll
        for (int u = 0; u < CG_U; ++u) {
            const int e = e0 + u * MD_TB;
            pp[u] = e < sg.end ? p[o + e] : 0.0;
            qq[u] = e < sg.end ? q[o + e] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < CG_U; ++u) v[0] += pp[u] * qq[u];
    }
    double flag;
    reduce_values<1>(v, 1, part, blockIdx.x, rng[sg.inst], &S.counter[2], &flag, sh);
    if (flag == 1.0 && threadIdx.x == 0) {
        S.pq = sh[0];
        S.alpha_cg = S.rho / sh[0];
    }
}

__global__ void __launch_bounds__(MD_TB) k_cg_xr(const Seg* __restrict__ seg, const InstRange* __restrict__ rng,
                                                 const long long* __restrict__ off, const InstDesc* __restrict__ D,
                                                 double* x, double* r, const double* __restrict__ p,
                                                 const double* __restrict__ q, KState* st, double* part, int* ndone,
                                                 ResOut res) {
    __shared__ double sh[32 * 4];
    const Seg sg = seg[blockIdx.x];
    KState& S = st[sg.inst];
    if (!S.active) return;
    const long long o = off[sg.inst];
    const double a = S.alpha_cg;
    const double* dinv = D[sg.inst].dinv64;
    double v[2] = {0.0, 0.0};
    for (int e0 = sg.begin + threadIdx.x; e0 < sg.end; e0 += CG_U * MD_TB) {
        double xx[CG_U], pp[CG_U], rr0[CG_U], qq[CG_U], dd[CG_U];
#pragma unroll
        for (int u = 0; u < CG_U; ++u) {
            const int e = e0 + u * MD_TB;
            const bool in = e < sg.end;
            xx[u] = in ? x[o + e] : 0.0;
            pp[u] = in ? p[o + e] : 0.0;
            rr0[u] = in ? r[o + e] : 0.0;
            qq[u] = in ? q[o + e] : 0.0;
            dd[u] = in ? dinv[e] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < CG_U; ++u) {
            const int e = e0 + u * MD_TB;
            if (e < sg.end) {
                x[o + e] = xx[u] + a * pp[u];
                const double rr = rr0[u] - a * qq[u];
                r[o + e] = rr;
                v[0] += rr * (dd[u] * rr);
                v[1] += rr * rr;
            }
        }
    }
    double flag;
    reduce_values<2>(v, 2, part, blockIdx.x, rng[sg.inst], &S.counter[3], &flag, sh);
    if (flag == 1.0 && threadIdx.x == 0) {
        const double rho_new = sh[0];
        S.coef[0] = rho_new / S.rho;  // beta of the p update
        S.rho = rho_new;
        S.iters += 1;
        S.relres = S.bnorm > 0 ? sqrt(sh[1]) / S.bnorm : 0.0;
        if (S.relres <= S.tol || S.iters >= S.maxit || !isfinite(S.relres)) {
            S.active = 0;
            S.reorth = 1;  // marks "stopped, needs the true residual"
        }
    }
}

__global__ void __launch_bounds__(MD_TB) k_cg_p(const Seg* __restrict__ seg, const long long* __restrict__ off,
                                                const InstDesc* __restrict__ D, const double* __restrict__ r,
                                                double* p, const KState* st) {
    const Seg sg = seg[blockIdx.x];
    const KState& S = st[sg.inst];
    if (!S.active) return;
    const long long o = off[sg.inst];
    const double bc = S.coef[0];
    const double* dinv = D[sg.inst].dinv64;
    for (int e0 = sg.begin + threadIdx.x; e0 < sg.end; e0 += CG_U * MD_TB) {
        double dd[CG_U], rr[CG_U], pp[CG_U];
#pragma unroll
        for (int u = 0; u < CG_U; ++u) {
            const int e = e0 + u * MD_TB;
            const bool in = e < sg.end;
            dd[u] = in ? dinv[e] : 0.0;
            rr[u] = in ? r[o + e] : 0.0;
            pp[u] = in ? p[o + e] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < CG_U; ++u) {
            const int e = e0 + u * MD_TB;
            if (e < sg.end) p[o + e] = dd[u] * rr[u] + bc * pp[u];
        }
    }
}

// true residual after CG stopped: relres = ||b - A x|| / ||b||
__global__ void __launch_bounds__(MD_TB) k_cg_final(const Seg* __restrict__ seg, const InstRange* __restrict__ rng,
                                                    const long long* __restrict__ off, const double* __restrict__ b,
                                                    const double* __restrict__ y, KState* st, double* part, int* ndone,
                                                    ResOut res) {
    __shared__ double sh[32 * 4];
    const Seg sg = seg[blockIdx.x];
    KState& S = st[sg.inst];
    if (S.t_done || !S.reorth) return;
    const long long o = off[sg.inst];
    double v[1] = {0.0};
    for (int e = sg.begin + threadIdx.x; e < sg.end; e += blockDim.x) {
        const double rr = b[o + e] - y[o + e];
        v[0] += rr * rr;
    }
    double flag;
    reduce_values<1>(v, 1, part, blockIdx.x, rng[sg.inst], &S.counter[4], &flag, sh);
    if (flag == 1.0 && threadIdx.x == 0) {
        S.relres = S.bnorm > 0 ? sqrt(sh[0]) / S.bnorm : 0.0;
        S.reorth = 0;
        mark_done(S, ndone, res, sg.inst);
    }
}

// ---------------------------------------------------------------------------
// host side
static md_status launch_lower_1d(md_batch* B, const float* v, float* z, cudaStream_t s) {
    const Tables& T = B->tabs;
    k_gather_z0<<<T.apply_a.nblocks, MD_TB, 0, s>>>(B->d, T.apply_a.seg, B->off, z, B->st);
    MD_CHECK_LAUNCH();
    k_lower_1d<<<B->ninst, TREE_TB, tree_smem_bytes(B->max_n1), s>>>(B->d, B->off, v, z, B->st);
    MD_CHECK_LAUNCH();
    return MD_OK;
}

// The network preconditioner with smoothing (B->smooth_nu > 0):
//   x = S_J(C, b0, 0, nu);  x += N(b0 - C x);  z0 = S_J(C, b0, x, nu)
// tmp: a whole-length scratch vector (the apply output and the network's
// input and output).
static md_status launch_precond_smoothed(md_batch* B, const md_cnn* cnn, const float* vin, float* zout, float* tmp,
                                         cudaStream_t s, unsigned long long* e_conv0, unsigned long long* e_conv1) {
    const Tables& T = B->tabs;
    const bool lower = B->prec_order == 1;
    const float omega = B->smooth_omega;
    if (!lower) {
        MD_TRY(launch_upper_1d(T, B->d, B->off, B->ninst, B->max_n1, vin, zout, B->st, B->part, s));
    }
    k_smooth_first<<<T.vec.nblocks, MD_TB, 0, s>>>(T.vec.seg, B->off, B->d, vin, zout, B->st, omega, !lower);
    MD_CHECK_LAUNCH();
    auto sweep = [&]() -> md_status {
        MD_TRY(launch_apply(T, B->d, B->ninst, MD_FP32, zout, B->off, tmp, s, B->st, 1));
        k_smooth_sweep<<<T.n3.nblocks, MD_TB, 0, s>>>(T.n3.seg, B->off, B->d, vin, tmp, zout, B->st, omega);
        MD_CHECK_LAUNCH();
        return MD_OK;
    };
    for (int i = 1; i < B->smooth_nu; ++i) MD_TRY(sweep());
    MD_TRY(launch_apply(T, B->d, B->ninst, MD_FP32, zout, B->off, tmp, s, B->st, 1));
    k_smooth_resid<<<T.n3.nblocks, MD_TB, 0, s>>>(T.n3.seg, T.n3.range, B->off, B->d, vin, tmp, B->st, B->part,
                                                   !lower);
    MD_CHECK_LAUNCH();
    MD_TRY(cnn_pack_prec(B->cw, B->d, tmp, B->off, B->st, tmp, s, !lower));
    OutIO io{tmp, B->off, tmp, B->off, B->st, B->d};
    MD_TRY(cnn_forward_layers(cnn, B->cw, io, CONV_PREC, s, e_conv0, e_conv1));
    k_smooth_add<<<T.n3.nblocks, MD_TB, 0, s>>>(T.n3.seg, B->off, tmp, zout, B->st);
    MD_CHECK_LAUNCH();
    for (int i = 0; i < B->smooth_nu; ++i) MD_TRY(sweep());
    if (lower) {
        MD_TRY(launch_lower_1d(B, vin, zout, s));
    }
    return MD_OK;
}

// The network preconditioner with the 3D solve as B->inner_m inner FGMRES
// steps on C (kernels above).  The conv events bracket the first network
// application only.
static md_status launch_precond_inner(md_batch* B, const md_cnn* cnn, const float* vin, float* zout, cudaStream_t s,
                                      unsigned long long* e_conv0, unsigned long long* e_conv1) {
    const Tables& T = B->tabs;
    const bool lower = B->prec_order == 1;
    const long long tot = B->total;
    const int m = B->inner_m;
    if (lower) {
        k_lower_setup<<<(B->ninst + 31) / 32, 32, 0, s>>>(B->st, B->ninst);
    } else {
        MD_TRY(launch_upper_1d(T, B->d, B->off, B->ninst, B->max_n1, vin, zout, B->st, B->part, s));
    }
    MD_CHECK_LAUNCH();
    MD_TRY(cnn_pack_prec(B->cw, B->d, vin, B->off, B->st, B->iZ, s, !lower));
    OutIO io0{B->iZ, B->off, vin, B->off, B->st, B->d};
    MD_TRY(cnn_forward_layers(cnn, B->cw, io0, CONV_PREC, s, e_conv0, e_conv1));
    k_inner_start<<<T.n3.nblocks, MD_TB, 0, s>>>(T.n3.seg, B->off, B->d, vin, B->iV, B->iZ, B->st, !lower);
    MD_CHECK_LAUNCH();
    for (int j = 0; j < m; ++j) {
        float* Zj = B->iZ + (long long)j * tot;
        float* W = B->iV + (long long)(j + 1) * tot;
        MD_TRY(launch_apply(T, B->d, B->ninst, MD_FP32, Zj, B->off, W, s, B->st, 1));
        for (int pass = 0; pass < 2; ++pass) {
            k_inner_dots<<<T.n3.nblocks, MD_TB, 0, s>>>(T.n3.seg, T.n3.range, B->off, B->iV, tot, j, B->st, B->part);
            k_inner_update<<<T.n3.nblocks, MD_TB, 0, s>>>(T.n3.seg, T.n3.range, B->off, B->iV, tot, j, pass, B->st,
                                                           B->part);
            MD_CHECK_LAUNCH();
        }
        k_inner_scale<<<T.n3.nblocks, MD_TB, 0, s>>>(T.n3.seg, B->off, B->iV, tot, j, B->st);
        MD_CHECK_LAUNCH();
        if (j + 1 < m) {
            float* Zn = B->iZ + (long long)(j + 1) * tot;
            MD_TRY(cnn_pack_prec(B->cw, B->d, W, B->off, B->st, Zn, s, false));
            OutIO io{Zn, B->off, W, B->off, B->st, B->d};
            MD_TRY(cnn_forward_layers(cnn, B->cw, io, CONV_PREC, s));
        }
    }
    k_inner_lsq<<<(B->ninst + 31) / 32, 32, 0, s>>>(B->st, B->ninst, m);
    k_inner_combine<<<T.n3.nblocks, MD_TB, 0, s>>>(T.n3.seg, B->off, B->iZ, tot, zout, B->st, m);
    MD_CHECK_LAUNCH();
    if (lower) {
        MD_TRY(launch_lower_1d(B, vin, zout, s));
    }
    return MD_OK;
}

// The U-net's input [b0 / s, d] per instance (b0 = v0 + l in the upper
// order, v0 in the lower), as the network input pack does for the CNN.
__global__ void k_unet_in(const Seg* __restrict__ seg, const InstDesc* __restrict__ D, const long long* __restrict__ off,
                          const float* __restrict__ v, const KState* __restrict__ st, int use_lift, float* __restrict__ X) {
    const Seg sg = seg[blockIdx.x];
    if (!cnn_runs(st, sg.inst)) return;
    const InstDesc& d = D[sg.inst];
    const long long n3 = d.n3;
    const double s = st[sg.inst].s;
    const float inv_s = s > 0.0 ? (float)(1.0 / s) : 0.f;
    const float* vi = v + off[sg.inst];
    float* x = X + (long long)sg.inst * 2 * n3;
    for (int e = sg.begin + threadIdx.x; e < sg.end; e += blockDim.x) {
        x[e] = (vi[e] + (use_lift ? d.lift32[e] : 0.f)) * inv_s;
        x[n3 + e] = d.dist[e];
    }
}

// z0 = (s / alpha) y on the unknown grid nodes, v0 on Dirichlet nodes
__global__ void k_unet_out(const Seg* __restrict__ seg, const InstDesc* __restrict__ D, const long long* __restrict__ off,
                           const float* __restrict__ v, const KState* __restrict__ st, const float* __restrict__ Y,
                           float* __restrict__ z) {
    const Seg sg = seg[blockIdx.x];
    if (!cnn_runs(st, sg.inst)) return;
    const InstDesc& d = D[sg.inst];
    const float scale = (float)(st[sg.inst].s / d.alpha);
    const float* y = Y + (long long)sg.inst * d.n3;
    const long long o = off[sg.inst];
    const int M = d.N + 1;
    for (int e = sg.begin + threadIdx.x; e < sg.end; e += blockDim.x) {
        const int i = e % M, j = (e / M) % M, k = e / (M * M);
        const bool bd = !d.natural && (i == 0 || i == d.N || j == 0 || j == d.N || k == 0 || k == d.N);
        z[o + e] = bd ? v[o + e] : scale * y[e];
    }
}

static md_status launch_precond(md_batch* B, const md_cnn* cnn, const float* vin, float* zout, float* tmp,
                                cudaStream_t s, unsigned long long* e_conv0 = nullptr,
                                unsigned long long* e_conv1 = nullptr) {
    const Tables& T = B->tabs;
    if (!cnn) {
        k_jacobi<<<T.vec.nblocks, MD_TB, 0, s>>>(T.vec.seg, B->off, B->d, vin, zout, B->st, 0);
        MD_CHECK_LAUNCH();
        stamp(e_conv0, s);
        stamp(e_conv1, s);
        return MD_OK;
    }
    // instances whose network application broke down continue with Jacobi
    k_jacobi<<<T.vec.nblocks, MD_TB, 0, s>>>(T.vec.seg, B->off, B->d, vin, zout, B->st, 1);
    MD_CHECK_LAUNCH();
    if (B->inner_m > 0) return launch_precond_inner(B, cnn, vin, zout, s, e_conv0, e_conv1);
    if (B->smooth_nu > 0) return launch_precond_smoothed(B, cnn, vin, zout, tmp, s, e_conv0, e_conv1);
    const bool lower = B->prec_order == 1;
    if (lower) {
        k_lower_setup<<<(B->ninst + 31) / 32, 32, 0, s>>>(B->st, B->ninst);
    } else {
        MD_TRY(launch_upper_1d(T, B->d, B->off, B->ninst, B->max_n1, vin, zout, B->st, B->part, s));
    }
    MD_CHECK_LAUNCH();
    if (B->unet) {
        // the U-net over every instance of the batch (one grid size)
        k_unet_in<<<T.n3.nblocks, MD_TB, 0, s>>>(T.n3.seg, B->d, B->off, vin, B->st, lower ? 0 : 1, B->ux);
        MD_CHECK_LAUNCH();
        stamp(e_conv0, s);
        MD_TRY(md_unet_forward(B->unet, B->un, B->ninst, B->ux, B->uy, (md_stream)s));
        stamp(e_conv1, s);
        k_unet_out<<<T.n3.nblocks, MD_TB, 0, s>>>(T.n3.seg, B->d, B->off, vin, B->st, B->uy, zout);
        MD_CHECK_LAUNCH();
    } else {
        MD_TRY(cnn_pack_prec(B->cw, B->d, vin, B->off, B->st, zout, s, !lower));
        OutIO io{zout, B->off, vin, B->off, B->st, B->d};
        MD_TRY(cnn_forward_layers(cnn, B->cw, io, CONV_PREC, s, e_conv0, e_conv1));
    }
    if (lower) {
        MD_TRY(launch_lower_1d(B, vin, zout, s));
    }
    return MD_OK;
}

// Iteration slot j of a restart cycle.
static md_status launch_slot(md_batch* B, int j, cudaStream_t s) {
    const Tables& T = B->tabs;
    const long long tot = B->total;
    const int gb = (B->ninst + 31) / 32;
    const float* Vj = B->V + (long long)j * tot;
    float* Zj = B->Z + (long long)j * tot;
    float* W = B->V + (long long)(j + 1) * tot;
    stamp(stamp_at(B, ST_PRE0), s);
    // W (the next basis vector) is the preconditioner's scratch until the apply below fills it
    MD_TRY(launch_precond(B, B->solver == MD_SOLVER_FGMRES_CNN ? B->cnn : nullptr, Vj, Zj, W, s,
                          stamp_at(B, ST_CONV0), stamp_at(B, ST_CONV1)));
    stamp(stamp_at(B, ST_APPLY0), s);
    MD_TRY(launch_apply(T, B->d, B->ninst, MD_FP32, Zj, B->off, W, s, B->st, 1));
    stamp(stamp_at(B, ST_APPLY1), s);
    launch_gs(B, j, s);
    k_givens<<<gb, 32, 0, s>>>(B->st, B->ninst, j, B->k);
    MD_CHECK_LAUNCH();
    stamp(stamp_at(B, ST_ARN1), s);
    return MD_OK;
}

// Restart: x += Z y (least squares of the cycle), r = b - A x in FP64.
static md_status launch_restart(md_batch* B, cudaStream_t s) {
    const Tables& T = B->tabs;
    const long long tot = B->total;
    const int gb = (B->ninst + 31) / 32;
    stamp(stamp_at(B, ST_REST0), s);
    k_lsq<<<gb, 32, 0, s>>>(B->st, B->ninst);
    k_xupd<<<T.vec.nblocks, MD_TB, 0, s>>>(T.vec.seg, B->off, B->Z, tot, B->x, B->st);
    MD_CHECK_LAUNCH();
    MD_TRY(launch_apply(T, B->d, B->ninst, MD_FP64, B->x, B->off, B->y64, s, B->st, 2));
    k_resid<<<T.vec.nblocks, MD_TB, 0, s>>>(T.vec.seg, T.vec.range, B->off, B->d, B->b, B->y64, B->V, B->st, B->part,
                                             B->ndone, B->res, B->k);
    MD_CHECK_LAUNCH();
    stamp(stamp_at(B, ST_REST1), s);
    return MD_OK;
}

#define CG_CHUNK 25
static md_status launch_cycle_cg(md_batch* B, cudaStream_t s) {
    const Tables& T = B->tabs;
    for (int it = 0; it < CG_CHUNK; ++it) {
        MD_TRY(launch_apply(T, B->d, B->ninst, MD_FP64, B->p64, B->off, B->y64, s, B->st, 1));
        k_cg_alpha<<<T.vec.nblocks, MD_TB, 0, s>>>(T.vec.seg, T.vec.range, B->off, B->p64, B->y64, B->st, B->part);
        k_cg_xr<<<T.vec.nblocks, MD_TB, 0, s>>>(T.vec.seg, T.vec.range, B->off, B->d, B->x, B->r64, B->p64, B->y64,
                                                 B->st, B->part, B->ndone, B->res);
        k_cg_p<<<T.vec.nblocks, MD_TB, 0, s>>>(T.vec.seg, B->off, B->d, B->r64, B->p64, B->st);
        MD_CHECK_LAUNCH();
    }
    MD_TRY(launch_apply(T, B->d, B->ninst, MD_FP64, B->x, B->off, B->y64, s, B->st, 2));
    k_cg_final<<<T.vec.nblocks, MD_TB, 0, s>>>(T.vec.seg, T.vec.range, B->off, B->b, B->y64, B->st, B->part, B->ndone,
                                                B->res);
    MD_CHECK_LAUNCH();
    return MD_OK;
}

// ---- the solve as one graph -------------------------------------------------
// Kernel nodes of a captured graph (the nodes of its conditional bodies are
// counted by the device when those bodies run).
static long long kernel_nodes(cudaGraph_t g) {
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
    long long k = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
    return k;
}

// Append a conditional node (IF or WHILE on handle h) to the graph being
// captured on stream cs, after everything captured so far; *body receives
// its body graph, to be filled by a capture of its own.
static md_status add_conditional(cudaStream_t cs, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                                 cudaGraph_t* body) {
    cudaStreamCaptureStatus status;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edges = nullptr;
    size_t nd = 0;
    MD_CUDA(cudaStreamGetCaptureInfo(cs, &status, nullptr, &g, &deps, &edges, &nd));
    if (status != cudaStreamCaptureStatusActive) { md_set_error("solve graph: capture not active"); return MD_ERR_CUDA; }
    cudaGraphNodeParams prm = {};
    prm.type = cudaGraphNodeTypeConditional;
    prm.conditional.handle = h;
    prm.conditional.type = type;
    prm.conditional.size = 1;
    cudaGraphNode_t node;
    MD_CUDA(cudaGraphAddNode(&node, g, deps, edges, nd, &prm));
    *body = prm.conditional.phGraph_out[0];
    MD_CUDA(cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return MD_OK;
}

// The handle of a conditional node in the graph being captured on cs, reset
// to 0 at every launch of the graph (a kernel sets it before the node).
static md_status capture_handle(cudaStream_t cs, cudaGraphConditionalHandle* h) {
    cudaStreamCaptureStatus status;
    cudaGraph_t g = nullptr;
    MD_CUDA(cudaStreamGetCaptureInfo(cs, &status, nullptr, &g, nullptr, nullptr, nullptr));
    MD_CUDA(cudaGraphConditionalHandleCreate(h, g, 0, cudaGraphCondAssignDefault));
    return MD_OK;
}

// Fill `body` by capturing what `launch` issues on stream cs.
template <class F>
static md_status capture_into(cudaStream_t cs, cudaGraph_t body, F&& launch) {
    MD_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    md_status st = launch(cs);
    cudaGraph_t out = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &out);
    if (st != MD_OK) return st;
    MD_CUDA(e);
    return MD_OK;
}

// The solve graph.  Set-up: state from the control block, ||b||, r = b - A x
// (FP64), the first cycle's basis (CG: its first direction); then
//   WHILE (an instance is unfinished and cycles < limit) {
//     FGMRES: slot condition; for j < k: IF (an instance iterates) { slot j;
//             slot condition }; restart (x += Z y, FP64 residual)
//     CG:     a chunk of CG_CHUNK iterations and the true residual of the
//             instances that stopped
//     loop condition
//   }
// so a solve is one graph launch and the host waits once, at the end.
// Set-up part of a solve: state from the control block, ||b||, r = b - A x
// (FP64), the first cycle's basis (CG: its first direction).
static md_status launch_init(md_batch* B, cudaStream_t s) {
    const Tables& T = B->tabs;
    const int gb = (B->ninst + 31) / 32;
    k_init_state<<<gb, 32, 0, s>>>(B->st, B->ninst, B->ctl, B->ndone);
    k_norm_b<<<T.vec.nblocks, MD_TB, 0, s>>>(T.vec.seg, T.vec.range, B->off, B->b, B->st, B->part);
    MD_CHECK_LAUNCH();
    MD_TRY(launch_apply(T, B->d, B->ninst, MD_FP64, B->x, B->off, B->y64, s, B->st, 2));
    if (B->solver == MD_SOLVER_CG_JACOBI) {
        k_cg_init<<<T.vec.nblocks, MD_TB, 0, s>>>(T.vec.seg, T.vec.range, B->off, B->d, B->b, B->y64, B->r64, B->p64,
                                                   B->st, B->part, B->ndone, B->res);
    } else {
        k_resid<<<T.vec.nblocks, MD_TB, 0, s>>>(T.vec.seg, T.vec.range, B->off, B->d, B->b, B->y64, B->V, B->st,
                                                 B->part, B->ndone, B->res, B->k);
    }
    MD_CHECK_LAUNCH();
    return MD_OK;
}

// One cycle with every iteration slot launched (their kernels return at once
// for instances that left the cycle): the loop body when slots cannot be
// gated by IF nodes, and the host-driven loop's cycle.
static md_status launch_cycle_all_slots(md_batch* B, cudaStream_t s) {
    if (B->solver == MD_SOLVER_CG_JACOBI) return launch_cycle_cg(B, s);
    const int prof = B->profiling ? 1 : 0;
    for (int j = 0; j < B->k; ++j) {
        MD_TRY(launch_slot(B, j, s));
        k_slot_count<<<1, 1, 0, s>>>(B->ctl, prof);
        MD_CHECK_LAUNCH();
    }
    return launch_restart(B, s);
}

// The solve graph: the set-up part, then
//   WHILE (an instance is unfinished and cycles < limit) {
//     FGMRES: every iteration slot (its kernels return at once for instances
//             that left the cycle), then the restart (x += Z y, FP64 residual)
//     CG:     a chunk of CG_CHUNK iterations and the true residual of the
//             instances that stopped
//     loop condition
//   }
// so a solve is one graph launch and the host waits once, at the end.  (Slots
// under conditional IF nodes nested in the WHILE body would skip the empty
// slots of a cycle entirely; the runtime of this toolkit and driver refuses an
// IF node inside a WHILE body, whether captured or added node by node.)
static md_status capture_solve(md_batch* B, cudaStream_t s) {
    const int prof = B->profiling ? 1 : 0;
    MD_TRY(launch_init(B, s));
    cudaGraphConditionalHandle hw;
    MD_TRY(capture_handle(s, &hw));
    k_loop_cond<<<1, 1, 0, s>>>(B->ctl, B->ndone, B->ninst, hw, 0ULL, 0, 0);
    MD_CHECK_LAUNCH();
    cudaGraph_t loop = nullptr;
    MD_TRY(add_conditional(s, hw, cudaGraphCondTypeWhile, &loop));
    return capture_into(B->cap_body, loop, [&](cudaStream_t sb) -> md_status {
        MD_TRY(launch_cycle_all_slots(B, sb));
        cudaStreamCaptureStatus status;
        cudaGraph_t g = nullptr;
        MD_CUDA(cudaStreamGetCaptureInfo(sb, &status, nullptr, &g, nullptr, nullptr, nullptr));
        const unsigned long long nk = (unsigned long long)kernel_nodes(g) + 1;
        k_loop_cond<<<1, 1, 0, sb>>>(B->ctl, B->ndone, B->ninst, hw, nk, 1, prof);
        MD_CHECK_LAUNCH();
        return MD_OK;
    });
}

static void destroy_graphs(md_batch* B) {
    if (B->solve_graph) { cudaGraphExecDestroy(B->solve_graph); B->solve_graph = nullptr; }
    if (B->init_graph) { cudaGraphExecDestroy(B->init_graph); B->init_graph = nullptr; }
    if (B->cycle_graph) { cudaGraphExecDestroy(B->cycle_graph); B->cycle_graph = nullptr; }
}

// Capture what `launch` issues on stream cs into an executable graph.
template <class F>
static md_status capture_exec(cudaStream_t cs, F&& launch, cudaGraphExec_t* out, long long* kernels) {
    cudaGraph_t g = nullptr;
    MD_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    md_status st = launch(cs);
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (st != MD_OK) { if (e == cudaSuccess && g) cudaGraphDestroy(g); return st; }
    MD_CUDA(e);
    if (kernels) *kernels = kernel_nodes(g);
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    MD_CUDA(e);
    return MD_OK;
}

// The host-driven loop (md_batch_set_host_loop): a set-up graph and a
// one-cycle graph, without conditional nodes, launched by the host, which
// reads the count of finished instances after every cycle.  Same kernels as
// the device-driven solve; for tools that cannot look inside conditional
// graph nodes (kernel profilers).
static md_status build_host_loop(md_batch* B) {
    MD_TRY(capture_exec(B->cap, [&](cudaStream_t s) { return launch_init(B, s); }, &B->init_graph, &B->init_kernels));
    MD_TRY(capture_exec(B->cap, [&](cudaStream_t s) -> md_status {
        MD_TRY(launch_cycle_all_slots(B, s));
        k_cycle_count<<<1, 1, 0, s>>>(B->ctl, B->profiling ? 1 : 0);
        MD_CHECK_LAUNCH();
        return MD_OK;
    }, &B->cycle_graph, &B->cycle_kernels));
    B->if_mode = 3;
    return MD_OK;
}

static md_status build_graph(md_batch* B) {
    const int engine = B->cnn ? B->cnn->engine : 0;
    const unsigned long long uid = B->cnn ? B->cnn->uid : 0;
    const bool have = B->host_loop ? B->cycle_graph != nullptr : B->solve_graph != nullptr;
    if (have && B->graph_cnn_uid == uid && B->graph_unet == B->unet && B->graph_prof == B->profiling && B->graph_engine == engine &&
        B->graph_prec_order == B->prec_order && B->graph_smooth_nu == B->smooth_nu &&
        B->graph_smooth_omega == B->smooth_omega && B->graph_inner_m == B->inner_m)
        return MD_OK;
    destroy_graphs(B);
    if (B->host_loop) {
        MD_TRY(build_host_loop(B));
        B->graph_cnn_uid = uid;
        B->graph_unet = B->unet;
        B->graph_prec_order = B->prec_order;
        B->graph_smooth_nu = B->smooth_nu;
        B->graph_smooth_omega = B->smooth_omega;
        B->graph_inner_m = B->inner_m;
        B->graph_prof = B->profiling;
        B->graph_engine = engine;
        return MD_OK;
    }
    cudaGraph_t g = nullptr;
    MD_CUDA(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal));
    md_status st = capture_solve(B, B->cap);
    cudaError_t e = cudaStreamEndCapture(B->cap, &g);
    if (st != MD_OK) {
        if (e == cudaSuccess && g) cudaGraphDestroy(g);
        return st;
    }
    MD_CUDA(e);
    B->if_mode = 2;
    B->init_kernels = kernel_nodes(g);
    e = cudaGraphInstantiate(&B->solve_graph, g, 0);
    cudaGraphDestroy(g);
    MD_CUDA(e);
    B->graph_cnn_uid = uid;
    B->graph_unet = B->unet;
    B->graph_prec_order = B->prec_order;
    B->graph_smooth_nu = B->smooth_nu;
    B->graph_smooth_omega = B->smooth_omega;
    B->graph_inner_m = B->inner_m;
    B->graph_prof = B->profiling;
    B->graph_engine = engine;
    return MD_OK;
}

// ---- autotuning at batch creation --------------------------------------------
// Batches of at least MD_TUNE_MIN_UNKNOWNS unknowns time their choices on the
// GPU once, when they are created, and keep the fastest: the elements per
// block of the Krylov vector kernels (Gram-Schmidt steps at basis lengths 6,
// 14, 22 and 30, those below the restart length, over the whole batch, all
// instances active), and the tiles per plane step of
// the tensor-core convolutions (a network forward pass over every grid).
#define MD_TUNE_MIN_UNKNOWNS 1000000

__global__ void k_tune_state(KState* st, int ninst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ninst) return;
    st[i].active = 1;
    st[i].reorth = 0;
    for (int r = 0; r <= MD_KMAX; ++r) { st[i].sig[r] = 1.0; st[i].coef[r] = 0.0; }
    st[i].wn2_before = 0.0;
}

static md_status tune_vec_chunk(md_batch* B, const std::vector<const InstDesc*>& ptrs) {
    const int cands[] = {4096, 8192, 16384, 32768};
    // one step of each compiled basis bound (8, 16, 24, 32) below the restart length
    const int js[4] = {std::min(5, B->k - 1), 13, 21, 29};
    cudaStream_t s = B->cap;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    MD_CUDA(cudaEventCreate(&e0));
    MD_CUDA(cudaEventCreate(&e1));
    Tables keep = B->tabs;
    double best = 1e300;
    Tables best_t = keep;
    int best_c = MD_VEC_CHUNK_FGMRES;
    md_status st = MD_OK;
    B->tuning.n_vec = 0;
    for (int c : cands) {
        Tables T;
        st = build_tables(ptrs, &T, &B->allocs, c);
        if (st != MD_OK) break;
        B->tabs = T;
        k_tune_state<<<(B->ninst + 31) / 32, 32, 0, s>>>(B->st, B->ninst);
        launch_gs(B, js[0], s);
        cudaEventRecord(e0, s);
        for (int r = 0; r < 3; ++r) {
            for (int q = 0; q < 4; ++q) {
                if (js[q] >= B->k) continue;
                k_tune_state<<<(B->ninst + 31) / 32, 32, 0, s>>>(B->st, B->ninst);
                launch_gs(B, js[q], s);
            }
        }
        cudaEventRecord(e1, s);
        cudaError_t e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) { st = md_cuda_status(e, "vector chunk tuning", __FILE__, __LINE__); break; }
        const double us = 1e3 * ms / 3;
        B->tuning.vec_candidates[B->tuning.n_vec] = c;
        B->tuning.vec_us[B->tuning.n_vec] = us;
        B->tuning.n_vec += 1;
        // candidates in increasing size: a larger chunk is taken only when it is
        // more than 5% faster, since the timing has every instance active while
        // a solve runs later iterations on fewer, where smaller blocks balance
        // the remaining work better
        if (us < 0.95 * best) { best = us; best_t = T; best_c = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    B->tabs = st == MD_OK ? best_t : keep;
    B->tuning.vec_chunk = st == MD_OK ? best_c : MD_VEC_CHUNK_FGMRES;
    // the state is set from scratch by every solve
    MD_CUDA(cudaMemsetAsync(B->st, 0, sizeof(KState) * B->ninst, s));
    MD_CUDA(cudaStreamSynchronize(s));
    return st;
}

extern "C" md_status md_batch_tuning(const md_batch* B, md_tuning_t* out) {
    if (!B || !out) { md_set_error("md_batch_tuning: NULL argument"); return MD_ERR_ARG; }
    *out = B->tuning;
    return MD_OK;
}

extern "C" md_status md_batch_create(int n_ops, const md_op* const* ops, const md_cnn* cnn, md_solver solver,
                                     int restart, md_batch** out) {
    if (!out || n_ops < 1 || !ops) { md_set_error("md_batch_create: bad argument"); return MD_ERR_ARG; }
    *out = nullptr;
    if (solver != MD_SOLVER_CG_JACOBI && (restart < 1 || restart > MD_KMAX)) {
        md_set_error("md_batch_create: restart %d outside [1, %d]", restart, MD_KMAX); return MD_ERR_ARG;
    }
    if (solver == MD_SOLVER_FGMRES_CNN && !cnn) { md_set_error("md_batch_create: network required"); return MD_ERR_ARG; }
    md_batch* B = new md_batch();
    B->ninst = n_ops;
    B->solver = solver;
    B->k = solver == MD_SOLVER_CG_JACOBI ? 1 : restart;
    B->cnn = cnn;
    std::vector<const InstDesc*> ptrs;
    std::vector<int> Ns;
    long long tot = 0;
    for (int i = 0; i < n_ops; ++i) {
        if (!ops[i]) { delete B; md_set_error("md_batch_create: op %d is NULL", i); return MD_ERR_ARG; }
        for (int j2 = 0; j2 < i; ++j2)
            if (ops[j2] == ops[i]) { delete B; md_set_error("md_batch_create: op %d repeated", i); return MD_ERR_ARG; }
        B->ops.push_back(ops[i]);
        B->hdesc.push_back(ops[i]->h);
        B->hoff.push_back(tot);
        tot += ops[i]->h.n;
        B->max_n1 = std::max(B->max_n1, ops[i]->h.n1);
        B->max_nq = std::max(B->max_nq, ops[i]->h.nq);
        Ns.push_back(ops[i]->h.N);
    }
    B->hoff.push_back(tot);
    B->total = tot;
    for (auto& d : B->hdesc) ptrs.push_back(&d);
    md_status st = MD_OK;
    auto chk = [&](md_status s2) { if (st == MD_OK) st = s2; };
    chk(dev_upload(&B->allocs, &B->d, B->hdesc.data(), B->hdesc.size()));
    chk(build_tables(ptrs, &B->tabs, &B->allocs, solver == MD_SOLVER_CG_JACOBI ? MD_VEC_CHUNK_CG : MD_VEC_CHUNK_FGMRES));
    chk(dev_upload(&B->allocs, &B->off, B->hoff.data(), B->hoff.size()));
    chk(dev_alloc(&B->allocs, &B->x, (size_t)tot));
    chk(dev_alloc(&B->allocs, &B->b, (size_t)tot));
    chk(dev_alloc(&B->allocs, &B->y64, (size_t)tot));
    if (solver == MD_SOLVER_CG_JACOBI) {
        chk(dev_alloc(&B->allocs, &B->r64, (size_t)tot));
        chk(dev_alloc(&B->allocs, &B->p64, (size_t)tot));
    } else {
        chk(dev_alloc(&B->allocs, &B->V, (size_t)(B->k + 1) * tot));
        chk(dev_alloc(&B->allocs, &B->Z, (size_t)B->k * tot));
    }
    chk(dev_alloc(&B->allocs, &B->st, (size_t)n_ops));
    // partial sums of one block of a reduction kernel (its table: whole vectors, grid
    // nodes or touched nodes)
    {
        // the smallest vector chunk the autotuner tries (2048) gives the most blocks
        long long vb = 0;
        for (int i = 0; i < n_ops; ++i) vb += (ops[i]->h.n + 2047) / 2048;
        chk(dev_alloc(&B->allocs, &B->part,
                      (size_t)std::max<long long>({vb, B->tabs.vec.nblocks, B->tabs.n3.nblocks, B->tabs.touch.nblocks, 1}) *
                          MD_MAXR));
    }
    chk(dev_alloc(&B->allocs, &B->ndone, 1));
    chk(dev_alloc(&B->allocs, &B->ctl, 1));
    if (st == MD_OK && cudaMallocHost(&B->h_ctl, sizeof(SolveCtl)) != cudaSuccess) chk(MD_ERR_OOM);
    chk(dev_alloc(&B->allocs, &B->res.iters, (size_t)n_ops));
    chk(dev_alloc(&B->allocs, &B->res.net_iters, (size_t)n_ops));
    chk(dev_alloc(&B->allocs, &B->res.relres, (size_t)n_ops));
    chk(dev_alloc(&B->allocs, &B->res.time, (size_t)n_ops));
    if (st == MD_OK && solver == MD_SOLVER_FGMRES_CNN) {
        chk(cnn_work_create(Ns, &B->cw));
        const size_t smem = tree_smem_bytes(B->max_n1);
        if (smem > 227 * 1024) {
            md_set_error("md_batch_create: a 1D mesh of %d nodes exceeds the shared memory of the tree solve", B->max_n1);
            chk(MD_ERR_ARG);
        }
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(k_tree_1d, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_lower_1d, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) chk(md_cuda_status(e, "tree smem", __FILE__, __LINE__));
        }
    }
    if (st == MD_OK) {
        cudaError_t e = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->cap_body, cudaStreamNonBlocking);
        if (e != cudaSuccess) chk(md_cuda_status(e, "cudaStreamCreate", __FILE__, __LINE__));
    }
    if (st == MD_OK) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) chk(md_cuda_status(e, "md_batch_create", __FILE__, __LINE__));
    }
    B->tuning.vec_chunk = solver == MD_SOLVER_CG_JACOBI ? MD_VEC_CHUNK_CG : MD_VEC_CHUNK_FGMRES;
    B->tuning.conv_tps = B->cw ? B->cw->tps : 0;
    if (st == MD_OK && solver != MD_SOLVER_CG_JACOBI && tot >= MD_TUNE_MIN_UNKNOWNS) {
        B->tuning.tuned = 1;
        chk(tune_vec_chunk(B, ptrs));
        if (st == MD_OK && B->cw) {
            chk(cnn_autotune_tps(cnn, B->cw, B->Z, B->off, B->tuning.conv_us));
            B->tuning.conv_tps = B->cw->tps;
        }
    }
    if (st != MD_OK) { md_batch_destroy(B); return st; }
    *out = B;
    return MD_OK;
}

extern "C" void md_batch_destroy(md_batch* B) {
    if (!B) return;
    destroy_graphs(B);
    if (B->h_ctl) cudaFreeHost(B->h_ctl);
    if (B->cap) cudaStreamDestroy(B->cap);
    if (B->cap_body) cudaStreamDestroy(B->cap_body);
    cnn_work_destroy(B->cw);
    dev_free_all(&B->allocs);
    delete B;
}

extern "C" md_status md_batch_offsets(const md_batch* B, long long* offsets) {
    if (!B || !offsets) { md_set_error("md_batch_offsets: NULL argument"); return MD_ERR_ARG; }
    memcpy(offsets, B->hoff.data(), sizeof(long long) * B->hoff.size());
    return MD_OK;
}

static md_status batch_run(md_batch* B, double tol, int maxit, cudaStream_t s) {
    MD_TRY(build_graph(B));
    const int per_cycle = B->solver == MD_SOLVER_CG_JACOBI ? CG_CHUNK : B->k;
    SolveCtl& c = *B->h_ctl;
    memset(&c, 0, sizeof(SolveCtl));
    c.tol = tol;
    c.maxit = maxit;
    c.max_cycles = maxit / per_cycle + 3;
    MD_CUDA(cudaMemcpyAsync(B->ctl, &c, sizeof(SolveCtl), cudaMemcpyHostToDevice, s));
    int ndone = 0;
    if (B->host_loop) {
        MD_CUDA(cudaGraphLaunch(B->init_graph, s));
        B->stats.graph_launches += 1;
        long long cycles = 0;
        for (; cycles < c.max_cycles; ++cycles) {
            MD_CUDA(cudaMemcpyAsync(&ndone, B->ndone, sizeof(int), cudaMemcpyDeviceToHost, s));
            MD_CUDA(cudaStreamSynchronize(s));
            if (ndone >= B->ninst) break;
            MD_CUDA(cudaGraphLaunch(B->cycle_graph, s));
            B->stats.graph_launches += 1;
        }
        MD_CUDA(cudaMemcpyAsync(&c, B->ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, s));
        MD_CUDA(cudaMemcpyAsync(&ndone, B->ndone, sizeof(int), cudaMemcpyDeviceToHost, s));
        MD_CUDA(cudaStreamSynchronize(s));
        B->stats.kernel_launches += B->init_kernels + cycles * B->cycle_kernels;
    } else {
        MD_CUDA(cudaGraphLaunch(B->solve_graph, s));
        MD_CUDA(cudaMemcpyAsync(&c, B->ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, s));
        MD_CUDA(cudaMemcpyAsync(&ndone, B->ndone, sizeof(int), cudaMemcpyDeviceToHost, s));
        MD_CUDA(cudaStreamSynchronize(s));
        B->stats.kernel_launches += B->init_kernels + (long long)c.kernels;
        B->stats.graph_launches += 1;
    }
    B->stats.cycles += c.cycles;
    if (B->profiling && B->solver != MD_SOLVER_CG_JACOBI) {
        B->stats.prec_ms += c.t_prec * 1e-6;
        B->stats.conv_hidden_ms += c.t_conv * 1e-6;
        B->stats.apply_ms += c.t_apply * 1e-6;
        B->stats.arnoldi_ms += c.t_arn * 1e-6;
        B->stats.restart_ms += c.t_restart * 1e-6;
        if (B->solver == MD_SOLVER_FGMRES_CNN) B->stats.conv_hidden_launches += 4 * (long long)c.slots;
    }
    if (B->cw) {
        int err = 0;
        MD_CUDA(cudaMemcpy(&err, B->cw->err, sizeof(int), cudaMemcpyDeviceToHost));
        if (err) { md_set_error("a network convolution timed out waiting on its pipeline"); return MD_ERR_TIMEOUT; }
    }
    if (ndone < B->ninst) { md_set_error("batch solve did not terminate"); return MD_ERR_TIMEOUT; }
    return MD_OK;
}

extern "C" md_status md_batch_solve(md_batch* B, const double* b_all, double* x_all, double tol, int maxit,
                                    int* iters, double* relres, md_stream stream) {
    if (!B || !b_all || !x_all || !(tol > 0) || maxit < 1) { md_set_error("md_batch_solve: bad argument"); return MD_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    MD_CUDA(cudaMemcpyAsync(B->b, b_all, sizeof(double) * B->total, cudaMemcpyDeviceToDevice, s));
    MD_CUDA(cudaMemcpyAsync(B->x, x_all, sizeof(double) * B->total, cudaMemcpyDeviceToDevice, s));
    MD_TRY(batch_run(B, tol, maxit, s));
    MD_CUDA(cudaMemcpyAsync(x_all, B->x, sizeof(double) * B->total, cudaMemcpyDeviceToDevice, s));
    std::vector<int> it(B->ninst), nit(B->ninst);
    std::vector<double> rr(B->ninst);
    B->last_times.resize(B->ninst);
    MD_CUDA(cudaMemcpyAsync(it.data(), B->res.iters, sizeof(int) * B->ninst, cudaMemcpyDeviceToHost, s));
    MD_CUDA(cudaMemcpyAsync(nit.data(), B->res.net_iters, sizeof(int) * B->ninst, cudaMemcpyDeviceToHost, s));
    MD_CUDA(cudaMemcpyAsync(rr.data(), B->res.relres, sizeof(double) * B->ninst, cudaMemcpyDeviceToHost, s));
    MD_CUDA(cudaMemcpyAsync(B->last_times.data(), B->res.time, sizeof(double) * B->ninst, cudaMemcpyDeviceToHost, s));
    MD_CUDA(cudaStreamSynchronize(s));
    bool all = true;
    for (int i = 0; i < B->ninst; ++i) {
        if (iters) iters[i] = it[i];
        if (relres) relres[i] = rr[i];
        if (!(rr[i] <= tol)) all = false;
        B->stats.iterations += it[i];
        if (B->solver == MD_SOLVER_FGMRES_CNN) {
            B->stats.precond_nodes += (long long)nit[i] * B->hdesc[i].n3;
            B->stats.fallback_instances += nit[i] < it[i] ? 1 : 0;
        }
    }
    return all ? MD_OK : MD_NOT_CONVERGED;
}

extern "C" md_status md_batch_set_host_loop(md_batch* B, int enable) {
    if (!B) { md_set_error("md_batch_set_host_loop: NULL batch"); return MD_ERR_ARG; }
    B->host_loop = enable != 0;
    return MD_OK;
}

extern "C" md_status md_batch_set_prec_order(md_batch* B, int lower) {
    if (!B || (lower != 0 && lower != 1)) { md_set_error("md_batch_set_prec_order: bad argument"); return MD_ERR_ARG; }
    B->prec_order = lower;
    return MD_OK;
}

extern "C" md_status md_batch_set_unet(md_batch* B, md_unet* u) {
    if (!B) { md_set_error("md_batch_set_unet: NULL batch"); return MD_ERR_ARG; }
    if (!u) { B->unet = nullptr; return MD_OK; }
    if (B->solver != MD_SOLVER_FGMRES_CNN) { md_set_error("md_batch_set_unet: a network-preconditioned FGMRES batch only"); return MD_ERR_ARG; }
    if (B->inner_m > 0 || B->smooth_nu > 0) {
        md_set_error("md_batch_set_unet: not combined with inner steps or smoothing"); return MD_ERR_ARG;
    }
    const int N = B->hdesc[0].N;
    for (const InstDesc& d : B->hdesc)
        if (d.N != N) { md_set_error("md_batch_set_unet: the instances must share the grid size"); return MD_ERR_ARG; }
    if (N + 1 < 4) { md_set_error("md_batch_set_unet: grids of at least 4^3 nodes"); return MD_ERR_ARG; }
    const long long n3 = (long long)(N + 1) * (N + 1) * (N + 1);
    if (!B->ux) {
        MD_TRY(dev_alloc(&B->allocs, &B->ux, (size_t)(2 * n3 * B->ninst)));
        MD_TRY(dev_alloc(&B->allocs, &B->uy, (size_t)(n3 * B->ninst)));
    }
    B->un = N + 1;
    // a first pass outside any capture sizes the U-net's workspace for this batch
    MD_TRY(md_unet_forward(u, B->un, B->ninst, B->ux, B->uy, nullptr));
    MD_CUDA(cudaDeviceSynchronize());
    B->unet = u;
    return MD_OK;
}

extern "C" md_status md_batch_set_profiling(md_batch* B, int enable) {
    if (!B) { md_set_error("md_batch_set_profiling: NULL batch"); return MD_ERR_ARG; }
    B->profiling = enable != 0;
    return MD_OK;
}

extern "C" md_status md_batch_stats(const md_batch* B, md_batch_stats_t* out) {
    if (!B || !out) { md_set_error("md_batch_stats: NULL argument"); return MD_ERR_ARG; }
    *out = B->stats;
    out->slot_gating = B->if_mode;
    return MD_OK;
}

extern "C" md_status md_batch_reset_stats(md_batch* B) {
    if (!B) { md_set_error("md_batch_reset_stats: NULL batch"); return MD_ERR_ARG; }
    B->stats = md_batch_stats_t{};
    return MD_OK;
}

extern "C" md_status md_batch_times(const md_batch* B, double* seconds) {
    if (!B || !seconds) { md_set_error("md_batch_times: NULL argument"); return MD_ERR_ARG; }
    for (int i = 0; i < B->ninst && i < (int)B->last_times.size(); ++i) seconds[i] = B->last_times[i];
    return MD_OK;
}

static md_status op_batch(const md_op* op_c, md_solver solver, int restart, const md_cnn* cnn, md_batch** out) {
    md_op* op = const_cast<md_op*>(op_c);
    const int slot = (int)solver;
    md_batch*& B = op->solver_cache[slot];
    if (B && (op->solver_cache_restart[slot] != restart)) { md_batch_destroy(B); B = nullptr; }
    if (!B) {
        const md_op* ops[1] = {op};
        MD_TRY(md_batch_create(1, ops, cnn, solver, restart, &B));
        op->solver_cache_restart[slot] = restart;
    }
    B->cnn = cnn;
    *out = B;
    return MD_OK;
}

extern "C" md_status md_solve(const md_op* op, const md_cnn* cnn, const double* b, double* x, double tol, int restart,
                              int maxit, int* iters, double* relres, md_stream s) {
    if (!op || !b || !x) { md_set_error("md_solve: NULL argument"); return MD_ERR_ARG; }
    md_batch* B = nullptr;
    MD_TRY(op_batch(op, cnn ? MD_SOLVER_FGMRES_CNN : MD_SOLVER_CG_JACOBI, cnn ? restart : 1, cnn, &B));
    return md_batch_solve(B, b, x, tol, maxit, iters, relres, s);
}

extern "C" md_status md_solve_batched(int n, const md_op* const* ops, const md_cnn* cnn, const double* const* b,
                                      double* const* x, double tol, int restart, int maxit, int* iters,
                                      double* relres, md_stream stream) {
    if (n < 1 || !ops || !b || !x) { md_set_error("md_solve_batched: bad argument"); return MD_ERR_ARG; }
    md_batch* B = nullptr;
    MD_TRY(md_batch_create(n, ops, cnn, cnn ? MD_SOLVER_FGMRES_CNN : MD_SOLVER_CG_JACOBI, cnn ? restart : 1, &B));
    cudaStream_t s = (cudaStream_t)stream;
    md_status st = MD_OK;
    for (int i = 0; i < n && st == MD_OK; ++i) {
        cudaError_t e = cudaMemcpyAsync(B->b + B->hoff[i], b[i], sizeof(double) * ops[i]->h.n, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(B->x + B->hoff[i], x[i], sizeof(double) * ops[i]->h.n, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) st = md_cuda_status(e, "md_solve_batched copy", __FILE__, __LINE__);
    }
    if (st == MD_OK) st = batch_run(B, tol, maxit, s);
    if (st == MD_OK) {
        for (int i = 0; i < n && st == MD_OK; ++i) {
            cudaError_t e = cudaMemcpyAsync(x[i], B->x + B->hoff[i], sizeof(double) * ops[i]->h.n, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) st = md_cuda_status(e, "md_solve_batched copy", __FILE__, __LINE__);
        }
        std::vector<int> it(n);
        std::vector<double> rr(n);
        cudaMemcpyAsync(it.data(), B->res.iters, sizeof(int) * n, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(rr.data(), B->res.relres, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess && st == MD_OK) st = md_cuda_status(e, "md_solve_batched", __FILE__, __LINE__);
        bool all = true;
        for (int i = 0; i < n; ++i) {
            if (iters) iters[i] = it[i];
            if (relres) relres[i] = rr[i];
            if (!(rr[i] <= tol)) all = false;
        }
        if (st == MD_OK && !all) st = MD_NOT_CONVERGED;
    }
    md_batch_destroy(B);
    return st;
}

// Preconditioner input pieces for ninst instances given from outside a solve
// (training): ||v0||^2, then the 1D solve into z's 1D part, the lift and s.
md_status launch_prec_input(const Tables& T, const InstDesc* d, const long long* off, const float* v, float* z,
                            KState* st, int ninst, int max_n1, double* part, cudaStream_t s) {
    k_norm3<<<T.n3.nblocks, MD_TB, 0, s>>>(T.n3.seg, T.n3.range, off, v, st, part);
    MD_CHECK_LAUNCH();
    const size_t smem = tree_smem_bytes(max_n1);
    if (smem > 227 * 1024) { md_set_error("training: 1D mesh of %d nodes too large for the tree solve", max_n1); return MD_ERR_ARG; }
    if (smem > 48 * 1024) MD_CUDA(cudaFuncSetAttribute(k_tree_1d, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return launch_upper_1d(T, d, off, ninst, max_n1, v, z, st, part, s);
}

// Standalone preconditioner application (one instance).
// a standalone application runs the network whatever an earlier solve with the
// operator's cached batch left behind
__global__ void k_prec_setup(KState* st) {
    st[0].active = 1;
    st[0].fallback = 0;
}
__global__ void k_lift_setup(KState* st) {
    st[0].active = 1;
    st[0].fallback = 0;
    st[0].v3n2 = 0.0;
}

extern "C" md_status md_lift(const md_op* op, const float* r, float* z1, float* l, md_stream stream) {
    if (!op || !r || !l) { md_set_error("md_lift: NULL argument"); return MD_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    md_batch* B = nullptr;
    MD_TRY(op_batch(op, MD_SOLVER_FGMRES_JACOBI, 1, nullptr, &B));
    const size_t smem = tree_smem_bytes(B->max_n1);
    if (smem > 227 * 1024) { md_set_error("md_lift: 1D mesh of %d nodes too large for the tree solve", B->max_n1); return MD_ERR_ARG; }
    if (smem > 48 * 1024) MD_CUDA(cudaFuncSetAttribute(k_tree_1d, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_lift_setup<<<1, 1, 0, s>>>(B->st);
    // z1 = B11^{-1} r1 into the 1D part of the batch's first Z vector (scratch);
    // l = beta Pi^T W Psi z1 into the operator's lift buffer (zero off the
    // nodes the averaging reaches)
    MD_TRY(launch_upper_1d(B->tabs, B->d, B->off, 1, B->max_n1, r, B->Z, B->st, B->part, s));
    const InstDesc& d = B->hdesc[0];
    MD_CUDA(cudaMemcpyAsync(l, d.lift32, sizeof(float) * d.n3, cudaMemcpyDeviceToDevice, s));
    if (z1) MD_CUDA(cudaMemcpyAsync(z1, B->Z + d.n3, sizeof(float) * d.n1, cudaMemcpyDeviceToDevice, s));
    return MD_OK;
}

extern "C" md_status md_precondition_lower(const md_op* op, const md_cnn* cnn, const float* r, float* z,
                                           md_stream stream) {
    if (!op || !cnn || !r || !z) { md_set_error("md_precondition_lower: NULL argument"); return MD_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    md_batch* B = nullptr;
    MD_TRY(op_batch(op, MD_SOLVER_FGMRES_CNN, 1, cnn, &B));
    const int keep = B->prec_order;
    B->prec_order = 1;
    k_prec_setup<<<1, 1, 0, s>>>(B->st);
    const Tables& T = B->tabs;
    k_norm3<<<T.n3.nblocks, MD_TB, 0, s>>>(T.n3.seg, T.n3.range, B->off, r, B->st, B->part);
    MD_CHECK_LAUNCH();
    const md_status st = launch_precond(B, cnn, r, z, B->V + B->total, s);
    B->prec_order = keep;
    return st;
}

// smoothing limits: sweeps per side, damping range of a convergent damped
// Jacobi iteration on an SPD matrix with unit-scaled diagonal
#define MD_SMOOTH_MAX 8

static md_status check_smoothing(int nu, double omega, const char* who) {
    if (nu < 0 || nu > MD_SMOOTH_MAX || !(omega > 0.0 && omega < 2.0)) {
        md_set_error("%s: smoothing needs 0 <= nu <= %d and 0 < omega < 2 (got %d, %g)", who, MD_SMOOTH_MAX, nu,
                     omega);
        return MD_ERR_ARG;
    }
    return MD_OK;
}

extern "C" md_status md_batch_set_smoothing(md_batch* B, int nu, double omega) {
    if (!B) { md_set_error("md_batch_set_smoothing: NULL batch"); return MD_ERR_ARG; }
    MD_TRY(check_smoothing(nu, omega, "md_batch_set_smoothing"));
    if (nu > 0 && B->inner_m > 0) {
        md_set_error("md_batch_set_smoothing: not combined with inner FGMRES steps");
        return MD_ERR_ARG;
    }
    if (nu > 0 && B->unet) { md_set_error("md_batch_set_smoothing: not combined with the U-net"); return MD_ERR_ARG; }
    B->smooth_nu = nu;
    B->smooth_omega = (float)omega;
    return MD_OK;
}

extern "C" md_status md_precondition_smoothed(const md_op* op, const md_cnn* cnn, int lower, int nu, double omega,
                                              const float* r, float* z, md_stream stream) {
    if (!op || !cnn || !r || !z || (lower != 0 && lower != 1)) {
        md_set_error("md_precondition_smoothed: bad argument");
        return MD_ERR_ARG;
    }
    MD_TRY(check_smoothing(nu, omega, "md_precondition_smoothed"));
    cudaStream_t s = (cudaStream_t)stream;
    md_batch* B = nullptr;
    MD_TRY(op_batch(op, MD_SOLVER_FGMRES_CNN, 1, cnn, &B));
    const int keep_order = B->prec_order, keep_nu = B->smooth_nu;
    const float keep_omega = B->smooth_omega;
    const int keep_m = B->inner_m;
    B->prec_order = lower;
    B->smooth_nu = nu;
    B->smooth_omega = (float)omega;
    B->inner_m = 0;
    // active, not fallen back; the input norm pieces are recomputed
    k_lift_setup<<<1, 1, 0, s>>>(B->st);
    const Tables& T = B->tabs;
    k_norm3<<<T.n3.nblocks, MD_TB, 0, s>>>(T.n3.seg, T.n3.range, B->off, r, B->st, B->part);
    md_status st = MD_OK;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = md_cuda_status(e, "md_precondition_smoothed", __FILE__, __LINE__);
    if (st == MD_OK) st = launch_precond(B, cnn, r, z, B->V + B->total, s);
    B->prec_order = keep_order;
    B->smooth_nu = keep_nu;
    B->smooth_omega = keep_omega;
    B->inner_m = keep_m;
    return st;
}

extern "C" md_status md_precondition(const md_op* op, const md_cnn* cnn, const float* r, float* z, md_stream stream) {
    if (!op || !r || !z) { md_set_error("md_precondition: NULL argument"); return MD_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    md_batch* B = nullptr;
    MD_TRY(op_batch(op, cnn ? MD_SOLVER_FGMRES_CNN : MD_SOLVER_FGMRES_JACOBI, 1, cnn, &B));
    k_prec_setup<<<1, 1, 0, s>>>(B->st);
    if (cnn) {
        const Tables& T = B->tabs;
        k_norm3<<<T.n3.nblocks, MD_TB, 0, s>>>(T.n3.seg, T.n3.range, B->off, r, B->st, B->part);
        MD_CHECK_LAUNCH();
    }
    return launch_precond(B, cnn, r, z, B->V + B->total, s);
}

// Inner FGMRES buffers of a network-preconditioned batch, allocated once at
// the largest step count (their addresses are baked into captured graphs).
static md_status ensure_inner(md_batch* B) {
    if (B->solver != MD_SOLVER_FGMRES_CNN || !B->cw) {
        md_set_error("inner FGMRES steps need a network-preconditioned batch");
        return MD_ERR_ARG;
    }
    // each buffer on its own, so that a failed allocation is retried by the next call
    if (!B->iV) MD_TRY(dev_alloc(&B->allocs, &B->iV, (size_t)(MD_INNER_MAX + 1) * B->total));
    if (!B->iZ) MD_TRY(dev_alloc(&B->allocs, &B->iZ, (size_t)MD_INNER_MAX * B->total));
    return MD_OK;
}

static md_status check_inner(int m, const char* who) {
    if (m < 0 || m > MD_INNER_MAX) {
        md_set_error("%s: inner steps must be in [0, %d] (got %d)", who, MD_INNER_MAX, m);
        return MD_ERR_ARG;
    }
    return MD_OK;
}

extern "C" md_status md_batch_set_inner_iters(md_batch* B, int m) {
    if (!B) { md_set_error("md_batch_set_inner_iters: NULL batch"); return MD_ERR_ARG; }
    MD_TRY(check_inner(m, "md_batch_set_inner_iters"));
    if (m > 0 && B->smooth_nu > 0) {
        md_set_error("md_batch_set_inner_iters: not combined with smoothing");
        return MD_ERR_ARG;
    }
    if (m > 0 && B->unet) { md_set_error("md_batch_set_inner_iters: not combined with the U-net"); return MD_ERR_ARG; }
    if (m > 0) MD_TRY(ensure_inner(B));
    B->inner_m = m;
    return MD_OK;
}

extern "C" md_status md_precondition_inner(const md_op* op, const md_cnn* cnn, int lower, int m, const float* r,
                                           float* z, md_stream stream) {
    if (!op || !cnn || !r || !z || (lower != 0 && lower != 1)) {
        md_set_error("md_precondition_inner: bad argument");
        return MD_ERR_ARG;
    }
    MD_TRY(check_inner(m, "md_precondition_inner"));
    cudaStream_t s = (cudaStream_t)stream;
    md_batch* B = nullptr;
    MD_TRY(op_batch(op, MD_SOLVER_FGMRES_CNN, 1, cnn, &B));
    MD_TRY(ensure_inner(B));
    const int keep_order = B->prec_order, keep_m = B->inner_m, keep_nu = B->smooth_nu;
    B->prec_order = lower;
    B->inner_m = m;
    B->smooth_nu = 0;
    k_lift_setup<<<1, 1, 0, s>>>(B->st);
    const Tables& T = B->tabs;
    k_norm3<<<T.n3.nblocks, MD_TB, 0, s>>>(T.n3.seg, T.n3.range, B->off, r, B->st, B->part);
    md_status st = MD_OK;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = md_cuda_status(e, "md_precondition_inner", __FILE__, __LINE__);
    if (st == MD_OK) st = launch_precond(B, cnn, r, z, B->V + B->total, s);
    B->prec_order = keep_order;
    B->inner_m = keep_m;
    B->smooth_nu = keep_nu;
    return st;
}
