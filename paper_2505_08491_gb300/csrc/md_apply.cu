// Matrix-free apply of the coupled operator A = K + beta M (eq. (mainsys)):
//
//   t_q  = (Pi u0)(q) - (Psi u1)(q)                      quadrature points
//   y0   = K00 u0 + beta Pi^T W t                         grid nodes
//   y1   = kappa K1 u1 - beta Psi^T W t                   1D nodes
//
// since M [u0; u1] = [Pi^T W (Pi u0 - Psi u1); -Psi^T W (Pi u0 - Psi u1)].
// Launch A runs the averaging gather t (kind 1); launch B runs the 27-point
// Q1 stencil tile by tile with the Pi^T W t rows of each tile's nodes added
// before the tile is stored (kind 4), and the 1D rows (kind 3).  All sums are
// in a fixed order, so results are deterministic.
#include <algorithm>
#include <cmath>

#include "md_common.cuh"

template <typename T>
__device__ inline T gather_q(const InstDesc& d, const T* __restrict__ u0, const T* __restrict__ u1, int q) {
    const T acc = csr_row<T, T>(d.pi_col, Pr<T>::pi(d), d.pi_ptr[q], d.pi_ptr[q + 1], u0);
    return acc - (Pr<T>::psa(d)[q] * u1[d.qa[q]] + Pr<T>::psb(d)[q] * u1[d.qb[q]]);
}

__device__ inline bool gate_skip(const KState* st, int gate, int inst) {
    if (!st || gate == 0) return false;
    return gate == 1 ? !st[inst].active : st[inst].t_done != 0ULL;
}

// Row (i, j, k) of a Q1 operator on the cube with natural conditions on its
// faces: the element-by-element sum gives neighbour (i, j, k) + d the
// coefficient c[|dx|+|dy|+|dz|] of the interior stencil times 1/2 for every
// axis a with d_a = 0 on which the node lies on a face (half of the elements
// around that axis are missing).  u: grid vector; neighbours outside the
// grid do not exist.
template <typename T>
__device__ inline T q1_row_natural(const T* __restrict__ u, int i, int j, int k, int N, const T* c) {
    const int M = N + 1;
    const T fx = (i == 0 || i == N) ? T(0.5) : T(1), fy = (j == 0 || j == N) ? T(0.5) : T(1),
            fz = (k == 0 || k == N) ? T(0.5) : T(1);
    T acc = T(0);
    for (int dz = -1; dz <= 1; ++dz) {
        if (k + dz < 0 || k + dz > N) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            if (j + dy < 0 || j + dy > N) continue;
            for (int dx = -1; dx <= 1; ++dx) {
                if (i + dx < 0 || i + dx > N) continue;
                T w = c[(dx != 0) + (dy != 0) + (dz != 0)];
                if (dx == 0) w *= fx;
                if (dy == 0) w *= fy;
                if (dz == 0) w *= fz;
                acc += w * u[(i + dx) + M * ((j + dy) + M * (k + dz))];
            }
        }
    }
    return acc;
}

// a / (N+1) for 0 <= a < 2^20 (InstDesc::mdiv)
__device__ __forceinline__ int div_m(unsigned int a, unsigned int mdiv) { return (int)__umulhi(a, mdiv); }

// Launch A: t_q = (Pi u0)(q) - (Psi u1)(q) at the quadrature points (kind 1).
template <typename T>
__global__ void __launch_bounds__(MD_TB) k_apply_a(const InstDesc* __restrict__ D, const Seg* __restrict__ seg,
                                                   const long long* __restrict__ off, const T* __restrict__ u,
                                                   const KState* __restrict__ st, int gate) {
    const Seg sg = seg[blockIdx.x];
    if (gate_skip(st, gate, sg.inst)) return;
    const InstDesc& d = D[sg.inst];
    const T* ui = u + off[sg.inst];
    T* t = Pr<T>::t(d);
    for (int q = sg.begin + threadIdx.x; q < sg.end; q += blockDim.x) t[q] = gather_q<T>(d, ui, ui + d.n3, q);
}

// Launch B, kind 4: one stencil tile -- planes [z0, z0 + nz), rows [y0, y0 + ny),
// all N+1 columns -- of y0 = K00 u0 + beta Pi^T W t.
//  1. The tile and a one-node halo in y and z are copied into shared memory,
//     Dirichlet nodes as zero (their columns are eliminated): each plane's
//     rows are one contiguous range of the grid, read with consecutive
//     threads on consecutive nodes.
//  2. Each thread owns one column (x, y) of the tile and walks z.  With
//     plane sums at (x, y) of plane p -- P0 = u, P1 = the 4 in-plane face
//     neighbours, P2 = the 4 in-plane corner neighbours -- the 27-point Q1
//     stencil by offset class is
//       centre P0(z); face P1(z) + P0(z-1) + P0(z+1);
//       edge P2(z) + P1(z-1) + P1(z+1); corner P2(z-1) + P2(z+1),
//     so every plane's sums serve three output planes.  Dirichlet nodes
//     copy u.  Results go to a shared output tile.
//  3. The rows of Pi^T W of the tile's touched nodes (grouped by tile at
//     assembly) add beta sum_q (Pi^T W)_{n,q} t_q to their nodes.
//  4. The output tile is stored plane by plane, each plane one contiguous
//     range.  So y0 is written once, without a read-modify-write.
// Kind 3: the 1D rows y1 = kappa K1 u1 - beta Psi^T W t.
template <typename T>
__device__ inline void stencil_tile(const InstDesc& d, int tile, const T* __restrict__ ui, T* __restrict__ yi,
                                    T* s_in) {
    const int N = d.N, M = N + 1, TY = d.ty;
    const unsigned int mdiv = d.mdiv;
    const bool natural = d.natural != 0;
    const int zt = tile / d.nyt, yt = tile - zt * d.nyt;
    const int z0 = zt * d.tz, y0 = yt * TY;
    const int nz = min(d.tz, M - z0), ny = min(TY, M - y0);
    const int rows_in = ny + 2, slab_in = rows_in * M;  // one halo-padded plane of the tile
    T* s_out = s_in + (size_t)(nz + 2) * slab_in;
    // 1. input tile: planes z0-1 .. z0+nz, rows y0-1 .. y0+ny (out-of-grid rows
    // zero).  Element e of the tile is plane e / slab_in, row r, column x of it;
    // each thread issues APPLY_LU loads before storing any (the loads then
    // overlap instead of each store waiting on its own load).
    {
        constexpr int APPLY_LU = 8;
        const int total_in = (nz + 2) * slab_in;
        const unsigned int sdiv = 0xFFFFFFFFu / (unsigned int)slab_in + 1u;  // ceil(2^32 / slab_in)
        for (int e0 = threadIdx.x; e0 < total_in; e0 += APPLY_LU * blockDim.x) {
            T v[APPLY_LU];
#pragma unroll
            for (int k = 0; k < APPLY_LU; ++k) {
                const int e = e0 + k * blockDim.x;
                v[k] = T(0);
                if (e < total_in) {
                    const int pz = (int)__umulhi((unsigned int)e, sdiv), er = e - pz * slab_in;
                    const int r = div_m((unsigned int)er, mdiv), x = er - r * M;
                    const int z = z0 - 1 + pz, y = y0 - 1 + r;
                    // Dirichlet nodes are eliminated columns (zero); with natural
                    // conditions only nodes outside the grid are
                    const bool keep = natural ? (z >= 0 && z <= N && y >= 0 && y <= N)
                                              : (z >= 1 && z <= N - 1 && y >= 1 && y <= N - 1 && x >= 1 && x <= N - 1);
                    if (keep) v[k] = ui[((long long)z * M + y) * M + x];
                }
            }
#pragma unroll
            for (int k = 0; k < APPLY_LU; ++k) {
                const int e = e0 + k * blockDim.x;
                if (e < total_in) s_in[e] = v[k];
            }
        }
    }
    __syncthreads();
    // 2. stencil, one column per thread
    const T c0 = Pr<T>::st(d, 0), c1 = Pr<T>::st(d, 1), c2 = Pr<T>::st(d, 2), c3 = Pr<T>::st(d, 3);
    for (int c = threadIdx.x; c < ny * M; c += blockDim.x) {
        const int r = div_m((unsigned int)c, mdiv), x = c - r * M, y = y0 + r;
        T* so = s_out + c;
        // a node on a cube face: with natural conditions its row of the
        // element-by-element sum (the neighbour of offset d weighs the class
        // coefficient times 1/2 per axis a with d_a = 0 on which the node lies
        // on a face; the tile's out-of-grid rows and planes are zero), a
        // Dirichlet row (u itself) otherwise
        auto face_node = [&](int zz) -> T {
            const int z = z0 + zz;
            if (!natural) return ui[((long long)z * M + y) * M + x];
            const T fx = (x == 0 || x == N) ? T(0.5) : T(1), fy = (y == 0 || y == N) ? T(0.5) : T(1),
                    fz = (z == 0 || z == N) ? T(0.5) : T(1);
            T acc = T(0);
            for (int dz = -1; dz <= 1; ++dz) {
                const T* pl = s_in + (size_t)(zz + 1 + dz) * slab_in + (size_t)(r + 1) * M;
                for (int dy = -1; dy <= 1; ++dy) {
                    const T* row = pl + dy * M;
                    for (int dx = -1; dx <= 1; ++dx) {
                        if (x + dx < 0 || x + dx > N) continue;
                        T w = Pr<T>::st(d, (dx != 0) + (dy != 0) + (dz != 0));
                        if (dx == 0) w *= fx;
                        if (dy == 0) w *= fy;
                        if (dz == 0) w *= fz;
                        acc += w * row[x + dx];
                    }
                }
            }
            return acc;
        };
        const bool col_bd = x == 0 || x == N || y == 0 || y == N;
        if (col_bd) {
            for (int zz = 0; zz < nz; ++zz) so[(size_t)zz * ny * M] = face_node(zz);
            continue;
        }
        // plane sums of input plane pz at this column
        const T* base = s_in + (size_t)(r + 1) * M + x;
        auto sums = [&](int pz, T& p0, T& p1, T& p2) {
            const T* b = base + (size_t)pz * slab_in;
            const T l = b[-1], rr = b[1], up = b[M], dn = b[-M];
            const T ul = b[M - 1], ur = b[M + 1], dl = b[-M - 1], dr = b[-M + 1];
            p0 = b[0];
            p1 = (l + rr) + (up + dn);
            p2 = (ul + ur) + (dl + dr);
        };
        T a0, a1, a2, b0, b1, b2, f0, f1, f2;
        sums(0, a0, a1, a2);
        sums(1, b0, b1, b2);
        for (int zz = 0; zz < nz; ++zz) {
            sums(zz + 2, f0, f1, f2);
            const int z = z0 + zz;
            T v;
            if (z == 0 || z == N) {
                v = face_node(zz);
            } else {
                const T face = b1 + (a0 + f0);
                const T edge = b2 + (a1 + f1);
                const T corner = a2 + f2;
                v = c0 * b0 + c1 * face + c2 * edge + c3 * corner;
            }
            so[(size_t)zz * ny * M] = v;
            a0 = b0; a1 = b1; a2 = b2;
            b0 = f0; b1 = f1; b2 = f2;
        }
    }
    __syncthreads();
    // 3. coupling rows of the tile's touched nodes
    const T* tv = Pr<T>::tn(d);
    const T* tq = Pr<T>::t(d);
    const T beta = (T)d.beta;
    for (int idx = d.tile_tptr[tile] + threadIdx.x; idx < d.tile_tptr[tile + 1]; idx += blockDim.x) {
        const T acc = csr_row<T, T>(d.tn_q, tv, d.tn_ptr[idx], d.tn_ptr[idx + 1], tq);
        const int n = d.tn_node[idx];
        const int zy = n / M, x = n - zy * M, z = zy / M, y = zy - z * M;
        s_out[((size_t)(z - z0) * ny + (y - y0)) * M + x] += beta * acc;
    }
    __syncthreads();
    // 4. store, plane by plane
    for (int zz = 0; zz < nz; ++zz) {
        T* gp = yi + ((long long)(z0 + zz) * M + y0) * M;
        const T* sp = s_out + (size_t)zz * ny * M;
        for (int e = threadIdx.x; e < ny * M; e += blockDim.x) gp[e] = sp[e];
    }
}

template <typename T>
__global__ void __launch_bounds__(MD_TB, 5) k_apply_b(const InstDesc* __restrict__ D, const Seg* __restrict__ seg,
                                                   const long long* __restrict__ off, const T* __restrict__ u,
                                                   T* __restrict__ y, const KState* __restrict__ st, int gate) {
    extern __shared__ __align__(16) unsigned char apply_smem[];
    const Seg sg = seg[blockIdx.x];
    if (gate_skip(st, gate, sg.inst)) return;
    const InstDesc& d = D[sg.inst];
    const T* ui = u + off[sg.inst];
    T* yi = y + off[sg.inst];
    if (sg.kind == 4) {
        stencil_tile<T>(d, sg.begin, ui, yi, reinterpret_cast<T*>(apply_smem));
        return;
    }
    const T* t = Pr<T>::t(d);
    const T beta = (T)d.beta;
    const T* u1 = ui + d.n3;
    T* y1 = yi + d.n3;
    const T* kv = Pr<T>::k1(d);
    const T* pv = Pr<T>::pw(d);
    for (int i = sg.begin + threadIdx.x; i < sg.end; i += blockDim.x) {
        const T a1 = csr_row<T, T>(d.k1_col, kv, d.k1_ptr[i], d.k1_ptr[i + 1], u1);
        const T a2 = csr_row<T, T>(d.pw_q, pv, d.pw_ptr[i], d.pw_ptr[i + 1], t);
        y1[i] = a1 - beta * a2;
    }
}

// Dynamic shared memory of the stencil tiles, set when a launch table is built
// (with its device current, outside any stream capture).
md_status apply_prepare(int smem32, int smem64) {
    if (smem32 > 48 * 1024) MD_CUDA(cudaFuncSetAttribute(k_apply_b<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem32));
    if (smem64 > 48 * 1024) MD_CUDA(cudaFuncSetAttribute(k_apply_b<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem64));
    return MD_OK;
}

md_status launch_apply(const Tables& T, const InstDesc* d, int ninst, md_prec prec, const void* u,
                       const long long* off, void* y, cudaStream_t s, const KState* st, int gate) {
    (void)ninst;
    if (prec == MD_FP32) {
        k_apply_a<float><<<T.apply_a.nblocks, MD_TB, 0, s>>>(d, T.apply_a.seg, off, (const float*)u, st, gate);
        k_apply_b<float><<<T.apply_b.nblocks, MD_TB, T.apply_b.smem32, s>>>(d, T.apply_b.seg, off, (const float*)u,
                                                                          (float*)y, st, gate);
    } else {
        k_apply_a<double><<<T.apply_a.nblocks, MD_TB, 0, s>>>(d, T.apply_a.seg, off, (const double*)u, st, gate);
        k_apply_b<double><<<T.apply_b.nblocks, MD_TB, T.apply_b.smem64, s>>>(d, T.apply_b.seg, off, (const double*)u,
                                                                           (double*)y, st, gate);
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
        if (idx >= d.n3) {
            const int i1 = (int)(idx - d.n3);
            b[idx] = g * d.load1[i1] + (d.rhs1 ? d.rhs1[i1] : 0.0);
            continue;
        }
        const int n = (int)idx;
        const int i = n % M, r = n / M, j = r % M, k = r / M;
        const double lift = d.rhs0 ? d.rhs0[n] : 0.0;
        if (d.natural) {
            b[n] = (f ? q1_row_natural<double>(f, i, j, k, N, d.ms64) : 0.0) + lift;
            continue;
        }
        if (!f || i == 0 || i == N || j == 0 || j == N || k == 0 || k == N) {
            b[n] = (i == 0 || i == N || j == 0 || j == N || k == 0 || k == N) ? 0.0 : lift;
            continue;
        }
        double s[4] = {0.0, 0.0, 0.0, 0.0};
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx)
                    s[(dx != 0) + (dy != 0) + (dz != 0)] += f[n + dx + dy * M + dz * M * M];
        b[n] = d.ms64[0] * s[0] + d.ms64[1] * s[1] + d.ms64[2] * s[2] + d.ms64[3] * s[3] + lift;
    }
}

md_status launch_rhs(const md_op* op, const double* f, double g, double* b, cudaStream_t s) {
    int blocks = (int)std::min<long long>((op->h.n + MD_TB - 1) / MD_TB, 152 * 16);
    k_rhs<<<blocks, MD_TB, 0, s>>>(op->d, f, g, b);
    MD_CHECK_LAUNCH();
    return MD_OK;
}

// ---- distance field d_h: min over the graph's straight segments, FP64
// Squared distance from a grid point to segment e in FP64 (NaN for a segment
// of zero length, which the minimum then ignores).
__device__ __forceinline__ double seg_q64(const double* sg, double px, double py, double pz) {
    const double ax = sg[0], ay = sg[1], az = sg[2];
    const double dx = sg[3] - ax, dy = sg[4] - ay, dz = sg[5] - az;
    const double dd = dx * dx + dy * dy + dz * dz;
    double t = ((px - ax) * dx + (py - ay) * dy + (pz - az) * dz) / dd;
    t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
    const double ex = px - (ax + t * dx), ey = py - (ay + t * dy), ez = pz - (az + t * dz);
    return ex * ex + ey * ey + ez * ez;
}

// Segments staged in shared memory for the FP32 search: start point, direction,
// 1 / squared length; a zero-length segment is staged far away (never nearest).
#define DIST_CHUNK 256
__device__ __forceinline__ void stage_seg(float* s7, const double* sg) {
    const double dx = sg[3] - sg[0], dy = sg[4] - sg[1], dz = sg[5] - sg[2];
    const double dd = dx * dx + dy * dy + dz * dz;
    const bool ok = dd > 0.0;
    s7[0] = ok ? (float)sg[0] : 1e18f;
    s7[1] = (float)sg[1];
    s7[2] = (float)sg[2];
    s7[3] = ok ? (float)dx : 0.f;
    s7[4] = ok ? (float)dy : 0.f;
    s7[5] = ok ? (float)dz : 0.f;
    s7[6] = ok ? (float)(1.0 / dd) : 0.f;
}
__device__ __forceinline__ float seg_q32(const float* s7, float fx, float fy, float fz) {
    const float ux = fx - s7[0], uy = fy - s7[1], uz = fz - s7[2];
    float t = (ux * s7[3] + uy * s7[4] + uz * s7[5]) * s7[6];
    t = fminf(fmaxf(t, 0.f), 1.f);
    const float ex = ux - t * s7[3], ey = uy - t * s7[4], ez = uz - t * s7[5];
    return ex * ex + ey * ey + ez * ez;
}

// The minimum over all segments is searched in FP32, then taken in FP64 over
// the segments whose FP32 value lies within 1e-5 of the FP32 minimum: with
// coordinates in [0, 1] an FP32 squared distance is within ~2e-6 of its FP64
// value, so the FP64 minimiser is always among them and d_h is the FP64
// minimum over every segment (FP64 runs at a small fraction of the FP32 rate
// on this GPU; the FP64 pass now touches one to a few segments per node).
__global__ void __launch_bounds__(MD_TB) k_dist(const InstDesc* __restrict__ D) {
    __shared__ float sseg[DIST_CHUNK * 7];
    const InstDesc& d = *D;
    const int N = d.N, M = N + 1, S = d.nsegs;
    float* out = const_cast<float*>(d.dist);
    const float invN = 1.0f / (float)N;
    // block-uniform trips: every thread takes part in the staging
    for (long long base = (long long)blockIdx.x * blockDim.x; base < d.n3; base += (long long)gridDim.x * blockDim.x) {
        const int n = (int)base + threadIdx.x;
        const bool valid = n < d.n3;
        int i = 0, j = 0, k = 0;
        if (valid) {
            i = n % M;
            const int r = n / M;
            j = r % M;
            k = r / M;
        }
        const float fx = i * invN, fy = j * invN, fz = k * invN;
        const double px = (double)i / N, py = (double)j / N, pz = (double)k / N;
        float best32 = 3.0e38f;
        for (int c0 = 0; c0 < S; c0 += DIST_CHUNK) {
            const int cn = min(DIST_CHUNK, S - c0);
            __syncthreads();
            for (int e = threadIdx.x; e < cn; e += blockDim.x) stage_seg(sseg + 7 * e, d.segs + 6 * (c0 + e));
            __syncthreads();
            for (int e = 0; e < cn; ++e) best32 = fminf(best32, seg_q32(sseg + 7 * e, fx, fy, fz));
        }
        const float lim = best32 + 1e-5f;
        double best = 1e300;
        for (int c0 = 0; c0 < S; c0 += DIST_CHUNK) {
            const int cn = min(DIST_CHUNK, S - c0);
            if (S > DIST_CHUNK) {  // one chunk stays staged from the search
                __syncthreads();
                for (int e = threadIdx.x; e < cn; e += blockDim.x) stage_seg(sseg + 7 * e, d.segs + 6 * (c0 + e));
                __syncthreads();
            }
            for (int e = 0; e < cn; ++e)
                if (seg_q32(sseg + 7 * e, fx, fy, fz) <= lim) {
                    const double q = seg_q64(d.segs + 6 * (c0 + e), px, py, pz);
                    best = q < best ? q : best;
                }
        }
        if (valid) out[n] = (float)sqrt(best);
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
    // natural conditions: every node is a row; the stencil centre of a node on
    // f faces is scaled by 1/2^f, and each neighbour's coefficient by 1/2 per
    // boundary axis it does not move along (q1_row_natural)
    auto fac = [&](int c) { return (c == 0 || c == N) ? 0.5 : 1.0; };
    std::vector<double> cdiag((size_t)D.n3, 0.0);  // diagonal of K00 (0: Dirichlet row)
    for (int k = 0; k < M; ++k)
        for (int j = 0; j < M; ++j)
            for (int i = 0; i < M; ++i) {
                const int n = i + M * (j + M * k);
                if (D.natural) {
                    const double f[3] = {fac(i), fac(j), fac(k)};
                    const int c[3] = {i, j, k};
                    cdiag[n] = D.st64[0] * f[0] * f[1] * f[2];
                    double sabs = 0.0;
                    for (int dz = -1; dz <= 1; ++dz)
                        for (int dy = -1; dy <= 1; ++dy)
                            for (int dx = -1; dx <= 1; ++dx) {
                                const int dd[3] = {dx, dy, dz};
                                bool in = true;
                                double w = std::fabs(D.st64[(dx != 0) + (dy != 0) + (dz != 0)]);
                                for (int a = 0; a < 3; ++a) {
                                    if (c[a] + dd[a] < 0 || c[a] + dd[a] > N) in = false;
                                    if (dd[a] == 0) w *= f[a];
                                }
                                if (in) sabs += w;
                            }
                    kabs[n] = sabs;
                    continue;
                }
                const bool bd = i == 0 || i == N || j == 0 || j == N || k == 0 || k == N;
                if (!bd) {
                    cdiag[n] = D.st64[0];
                    const double x = nside(i), y = nside(j), z = nside(k);
                    kabs[n] = a0 + (x + y + z) * a1 + (x * y + x * z + y * z) * a2 + x * y * z * a3;
                }
            }
    std::vector<int> tn((size_t)D.ntouch);
    if (D.ntouch) MD_CUDA(cudaMemcpy(tn.data(), D.tn_node, sizeof(int) * D.ntouch, cudaMemcpyDeviceToHost));
    std::vector<double> srow((size_t)D.n3, 0.0);  // beta (Pi^T W Pi) row sums
    for (int i = 0; i < D.ntouch; ++i) {
        cdiag[tn[i]] += D.beta * touch_m[i];
        srow[tn[i]] = D.beta * touch_rs[i];
    }
    for (int n = 0; n < D.n3; ++n) dv[n] = cdiag[n] != 0.0 ? 1.0 / cdiag[n] : 1.0;
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
