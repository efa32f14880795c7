// Matrix-free apply of the coupled operator A = K + beta M (eq. (mainsys)):
//
//   t_q  = (Pi u0)(q) - (Psi u1)(q)                      quadrature points
//   y0   = K00 u0 + beta Pi^T W t                         grid nodes
//   y1   = kappa K1 u1 - beta Psi^T W t                   1D nodes
//
// since M [u0; u1] = [Pi^T W (Pi u0 - Psi u1); -Psi^T W (Pi u0 - Psi u1)].
// Launch A runs the 27-point Q1 stencil (kind 0) and the averaging gather
// (kind 1) side by side; launch B adds the Pi^T scatter on the grid nodes the
// averaging reaches (kind 2) and computes the 1D rows (kind 3).  All sums are
// in a fixed order, so results are deterministic.
#include <algorithm>
#include <cmath>

#include "md_common.cuh"

// y0 over [begin, end) of the grid: Dirichlet nodes copy u, interior nodes
// take the stencil with boundary neighbours treated as zero (eliminated
// columns).  Offset class c = |dx|+|dy|+|dz| selects the coefficient.
template <typename T>
__device__ inline T stencil_node(const InstDesc& d, const T* __restrict__ u, int n, bool& boundary) {
    const int N = d.N, M = N + 1;
    const int i = n % M, r = n / M, j = r % M, k = r / M;
    boundary = (i == 0 || i == N || j == 0 || j == N || k == 0 || k == N);
    if (boundary) return u[n];
    const bool xm = i >= 2, xp = i <= N - 2;
    const bool ym = j >= 2, yp = j <= N - 2;
    const bool zm = k >= 2, zp = k <= N - 2;
    T s[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz) {
        const bool mz = dz < 0 ? zm : (dz > 0 ? zp : true);
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const bool my = dy < 0 ? ym : (dy > 0 ? yp : true);
            if (!(mz && my)) continue;
            const int base = n + dy * M + dz * M * M;
            const int cls = (dy != 0) + (dz != 0);
            T b = u[base];
            T ac = (xm ? u[base - 1] : T(0)) + (xp ? u[base + 1] : T(0));
            s[cls] += b;
            s[cls + 1] += ac;
        }
    }
    return Pr<T>::st(d, 0) * s[0] + Pr<T>::st(d, 1) * s[1] + Pr<T>::st(d, 2) * s[2] + Pr<T>::st(d, 3) * s[3];
}

template <typename T>
__device__ inline T gather_q(const InstDesc& d, const T* __restrict__ u0, const T* __restrict__ u1, int q) {
    const T* pv = Pr<T>::pi(d);
    T acc = T(0);
    for (int jj = d.pi_ptr[q]; jj < d.pi_ptr[q + 1]; ++jj) acc += pv[jj] * u0[d.pi_col[jj]];
    return acc - (Pr<T>::psa(d)[q] * u1[d.qa[q]] + Pr<T>::psb(d)[q] * u1[d.qb[q]]);
}

__device__ inline bool gate_skip(const KState* st, int gate, int inst) {
    if (!st || gate == 0) return false;
    return gate == 1 ? !st[inst].active : st[inst].t_done != 0ULL;
}

template <typename T>
__global__ void __launch_bounds__(MD_TB) k_apply_a(const InstDesc* __restrict__ D, const Seg* __restrict__ seg,
                                                   const long long* __restrict__ off, const T* __restrict__ u,
                                                   T* __restrict__ y, const KState* __restrict__ st, int gate) {
    const Seg sg = seg[blockIdx.x];
    if (gate_skip(st, gate, sg.inst)) return;
    const InstDesc& d = D[sg.inst];
    const T* ui = u + off[sg.inst];
    T* yi = y + off[sg.inst];
    if (sg.kind == 0) {
        for (int n = sg.begin + threadIdx.x; n < sg.end; n += blockDim.x) {
            bool bd;
            yi[n] = stencil_node<T>(d, ui, n, bd);
        }
    } else {
        T* t = Pr<T>::t(d);
        for (int q = sg.begin + threadIdx.x; q < sg.end; q += blockDim.x) t[q] = gather_q<T>(d, ui, ui + d.n3, q);
    }
}

template <typename T>
__global__ void __launch_bounds__(MD_TB) k_apply_b(const InstDesc* __restrict__ D, const Seg* __restrict__ seg,
                                                   const long long* __restrict__ off, const T* __restrict__ u,
                                                   T* __restrict__ y, const KState* __restrict__ st, int gate) {
    const Seg sg = seg[blockIdx.x];
    if (gate_skip(st, gate, sg.inst)) return;
    const InstDesc& d = D[sg.inst];
    const T* ui = u + off[sg.inst];
    T* yi = y + off[sg.inst];
    const T* t = Pr<T>::t(d);
    const T beta = (T)d.beta;
    if (sg.kind == 2) {
        const T* tv = Pr<T>::tn(d);
        for (int idx = sg.begin + threadIdx.x; idx < sg.end; idx += blockDim.x) {
            T acc = T(0);
            for (int jj = d.tn_ptr[idx]; jj < d.tn_ptr[idx + 1]; ++jj) acc += tv[jj] * t[d.tn_q[jj]];
            yi[d.tn_node[idx]] += beta * acc;
        }
    } else {
        const T* u1 = ui + d.n3;
        T* y1 = yi + d.n3;
        const T* kv = Pr<T>::k1(d);
        const T* pv = Pr<T>::pw(d);
        for (int i = sg.begin + threadIdx.x; i < sg.end; i += blockDim.x) {
            T a1 = T(0), a2 = T(0);
            for (int jj = d.k1_ptr[i]; jj < d.k1_ptr[i + 1]; ++jj) a1 += kv[jj] * u1[d.k1_col[jj]];
            for (int jj = d.pw_ptr[i]; jj < d.pw_ptr[i + 1]; ++jj) a2 += pv[jj] * t[d.pw_q[jj]];
            y1[i] = a1 - beta * a2;
        }
    }
}

md_status launch_apply(const Tables& T, const InstDesc* d, int ninst, md_prec prec, const void* u,
                       const long long* off, void* y, cudaStream_t s, const KState* st, int gate) {
    (void)ninst;
    if (prec == MD_FP32) {
        k_apply_a<float><<<T.apply_a.nblocks, MD_TB, 0, s>>>(d, T.apply_a.seg, off, (const float*)u, (float*)y, st, gate);
        k_apply_b<float><<<T.apply_b.nblocks, MD_TB, 0, s>>>(d, T.apply_b.seg, off, (const float*)u, (float*)y, st, gate);
    } else {
        k_apply_a<double><<<T.apply_a.nblocks, MD_TB, 0, s>>>(d, T.apply_a.seg, off, (const double*)u, (double*)y, st, gate);
        k_apply_b<double><<<T.apply_b.nblocks, MD_TB, 0, s>>>(d, T.apply_b.seg, off, (const double*)u, (double*)y, st, gate);
    }
    MD_CHECK_LAUNCH();
    return MD_OK;
}

// ---- load vector: b0 = M_Omega f (0 on Dirichlet nodes), b1 = g int psi_i
__global__ void k_rhs(const InstDesc* __restrict__ D, const double* __restrict__ f, double g, double* __restrict__ b) {
    const InstDesc& d = *D;
    const long long total = d.n;
    const int N = d.N, M = N + 1;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total; idx += (long long)gridDim.x * blockDim.x) {
        if (idx >= d.n3) { b[idx] = g * d.load1[idx - d.n3]; continue; }
        const int n = (int)idx;
        const int i = n % M, r = n / M, j = r % M, k = r / M;
        if (!f || i == 0 || i == N || j == 0 || j == N || k == 0 || k == N) { b[n] = 0.0; continue; }
        double s[4] = {0.0, 0.0, 0.0, 0.0};
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx)
                    s[(dx != 0) + (dy != 0) + (dz != 0)] += f[n + dx + dy * M + dz * M * M];
        b[n] = d.ms64[0] * s[0] + d.ms64[1] * s[1] + d.ms64[2] * s[2] + d.ms64[3] * s[3];
    }
}

md_status launch_rhs(const md_op* op, const double* f, double g, double* b, cudaStream_t s) {
    int blocks = (int)std::min<long long>((op->h.n + MD_TB - 1) / MD_TB, 152 * 16);
    k_rhs<<<blocks, MD_TB, 0, s>>>(op->d, f, g, b);
    MD_CHECK_LAUNCH();
    return MD_OK;
}

// ---- distance field d_h: min over the graph's straight segments, FP64
__global__ void k_dist(const InstDesc* __restrict__ D) {
    const InstDesc& d = *D;
    const int N = d.N, M = N + 1;
    float* out = const_cast<float*>(d.dist);
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < d.n3; n += gridDim.x * blockDim.x) {
        const int i = n % M, r = n / M, j = r % M, k = r / M;
        const double px = (double)i / N, py = (double)j / N, pz = (double)k / N;
        double best = 1e300;
        for (int e = 0; e < d.nsegs; ++e) {
            const double* sg = d.segs + 6 * e;
            const double ax = sg[0], ay = sg[1], az = sg[2];
            const double dx = sg[3] - ax, dy = sg[4] - ay, dz = sg[5] - az;
            const double dd = dx * dx + dy * dy + dz * dz;
            double t = ((px - ax) * dx + (py - ay) * dy + (pz - az) * dz) / dd;
            t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
            const double ex = px - (ax + t * dx), ey = py - (ay + t * dy), ez = pz - (az + t * dz);
            const double q = ex * ex + ey * ey + ez * ez;
            best = q < best ? q : best;
        }
        out[n] = (float)sqrt(best);
    }
}

md_status launch_dist(md_op* op, cudaStream_t s) {
    int blocks = std::min((op->h.n3 + MD_TB - 1) / MD_TB, 152 * 8);
    k_dist<<<blocks, MD_TB, 0, s>>>(op->d);
    MD_CHECK_LAUNCH();
    return MD_OK;
}

// ---- 1 / diag(A): grid interior c0 (+ beta (Pi^T W Pi)_nn at touched nodes),
// 1 on Dirichlet nodes, diag(B11) on 1D nodes.  Built on the host once.
// 1 / diag(A), and the Jacobi smoother's scaling of the 3D rows: rho_i / c_ii
// with rho_i = min(1, 2 c_ii / S_i), S_i = sum_j |K00_ij| + beta sum_j (Pi^T W Pi)_ij
// a bound of the absolute row sum of C (Gershgorin): 1 / c_ii on the stencil
// rows, smaller where the coupling is heavy, so that damped sweeps with
// omega < 1 contract on every mode; 1 on Dirichlet rows.
md_status launch_dinv_fill(md_op* op, const std::vector<double>& touch_m, const std::vector<double>& touch_rs,
                           const std::vector<double>& d1, cudaStream_t s) {
    (void)s;
    const InstDesc& D = op->h;
    const int N = D.N, M = N + 1;
    std::vector<double> dv((size_t)D.n), kabs((size_t)D.n3, 0.0);
    std::vector<float> fv((size_t)D.n);
    // |stencil| row sum over the interior neighbours: per axis, n_a of the two
    // neighbour offsets stay interior; the neighbours of offset class m (m
    // nonzero offsets) number the t^m coefficient of prod_a (1 + n_a t)
    const double a0 = std::fabs(D.st64[0]), a1 = std::fabs(D.st64[1]), a2 = std::fabs(D.st64[2]),
                 a3 = std::fabs(D.st64[3]);
    auto nside = [&](int c) { return (double)((c - 1 >= 1) + (c + 1 <= N - 1)); };
    for (int k = 0; k < M; ++k)
        for (int j = 0; j < M; ++j)
            for (int i = 0; i < M; ++i) {
                const bool bd = i == 0 || i == N || j == 0 || j == N || k == 0 || k == N;
                const int n = i + M * (j + M * k);
                dv[n] = bd ? 1.0 : 1.0 / D.st64[0];
                if (!bd) {
                    const double x = nside(i), y = nside(j), z = nside(k);
                    kabs[n] = a0 + (x + y + z) * a1 + (x * y + x * z + y * z) * a2 + x * y * z * a3;
                }
            }
    std::vector<int> tn((size_t)D.ntouch);
    if (D.ntouch) MD_CUDA(cudaMemcpy(tn.data(), D.tn_node, sizeof(int) * D.ntouch, cudaMemcpyDeviceToHost));
    std::vector<double> srow((size_t)D.n3, 0.0);  // beta (Pi^T W Pi) row sums
    for (int i = 0; i < D.ntouch; ++i) {
        dv[tn[i]] = 1.0 / (D.st64[0] + D.beta * touch_m[i]);
        srow[tn[i]] = D.beta * touch_rs[i];
    }
    std::vector<float> sv((size_t)D.n3);
    for (int n = 0; n < D.n3; ++n) {
        if (kabs[n] == 0.0) { sv[n] = 1.f; continue; }   // Dirichlet row
        const double c = 1.0 / dv[n];
        const double rho = std::min(1.0, 2.0 * c / (kabs[n] + srow[n]));
        sv[n] = (float)(rho / c);
    }
    for (int i = 0; i < D.n1; ++i) dv[D.n3 + i] = 1.0 / d1[i];
    for (size_t i = 0; i < dv.size(); ++i) fv[i] = (float)dv[i];
    MD_CUDA(cudaMemcpy((void*)D.dinv64, dv.data(), sizeof(double) * dv.size(), cudaMemcpyHostToDevice));
    MD_CUDA(cudaMemcpy((void*)D.dinv32, fv.data(), sizeof(float) * fv.size(), cudaMemcpyHostToDevice));
    MD_CUDA(cudaMemcpy((void*)D.sminv32, sv.data(), sizeof(float) * sv.size(), cudaMemcpyHostToDevice));
    return MD_OK;
}

// ---- public entry points -------------------------------------------------
extern "C" md_status md_apply(const md_op* op, md_prec prec, const void* u, void* y, md_stream s) {
    if (!op || !u || !y) { md_set_error("md_apply: NULL argument"); return MD_ERR_ARG; }
    if (prec != MD_FP32 && prec != MD_FP64) { md_set_error("md_apply: bad precision"); return MD_ERR_ARG; }
    if (u == y) { md_set_error("md_apply: u and y alias"); return MD_ERR_ARG; }
    return launch_apply(op->tabs, op->d, 1, prec, u, op->off0, y, (cudaStream_t)s);
}

extern "C" md_status md_rhs(const md_op* op, const double* f, double g, double* b, md_stream s) {
    if (!op || !b) { md_set_error("md_rhs: NULL argument"); return MD_ERR_ARG; }
    return launch_rhs(op, f, g, b, (cudaStream_t)s);
}
