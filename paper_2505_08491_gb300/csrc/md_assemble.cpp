// md_assemble: geometry and sparse structure of one 3D-1D instance
// (eq. (mainsys), Section 2.1), built on the host in FP64 and uploaded.
//
// Readings of points the paper leaves open, shared with the oracle by
// specification only (no code is shared):
//   - homogeneous Dirichlet rows/columns on the cube boundary, or the natural
//     condition of eq. (problem) (md_params.natural_boundary), with the 1D
//     Dirichlet nodes of dLambda_D eliminated symmetrically;
//   - beta multiplies the coupling form with unit line weight;
//   - 1D diffusion kappa = k_lambda * pi R^2;
//   - 2 Gauss points per 1D element; 8 circle points at theta_k = 2 pi k / 8
//     with exact cosines/sines; frame n1 = unit(t x e_a) with e_a the axis of
//     smallest |t_a| (lowest index on ties), n2 = t x n1;
//   - circle point in cell clamp(floor(x N), 0, N-1), trilinear weights,
//     boundary-node weights dropped.
#include <algorithm>
#include <functional>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>

#include "md_internal.h"

namespace {

struct Vec3 { double x, y, z; };
inline Vec3 sub(Vec3 a, Vec3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline Vec3 add(Vec3 a, Vec3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline Vec3 scale(double s, Vec3 a) { return {s * a.x, s * a.y, s * a.z}; }
inline double norm(Vec3 a) { return std::sqrt(a.x * a.x + a.y * a.y + a.z * a.z); }
inline Vec3 cross(Vec3 a, Vec3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

struct Entry { int col; double val; };

}  // namespace

// Operator arrays staged on the host and uploaded with one device allocation,
// one copy and one clear (each array 256-byte aligned) instead of an
// allocation and a copy per array.  commit() writes the device pointers to
// their slots.
struct UploadArena {
    std::vector<unsigned char> stage;  // arrays with host data, then the zero-filled ones
    size_t zero_bytes = 0;
    std::vector<std::function<void(unsigned char*)>> bind;
    static size_t align(size_t b) { return (b + 255) & ~(size_t)255; }
    template <class T>
    void up(const T** slot, const std::vector<T>& v) {
        const size_t off = align(stage.size()), bytes = v.size() * sizeof(T);
        stage.resize(off + (bytes ? bytes : 1));
        if (bytes) memcpy(stage.data() + off, v.data(), bytes);
        bind.push_back([slot, off](unsigned char* b) { *slot = reinterpret_cast<const T*>(b + off); });
    }
    void up32(const float** slot, const std::vector<double>& v) {
        const std::vector<float> f(v.begin(), v.end());
        up(slot, f);
    }
    template <class T>
    void zeros(T** slot, size_t count) {  // placed after every staged array
        const size_t off = align(zero_bytes);
        zero_bytes = off + (count ? count : 1) * sizeof(T);
        bind.push_back([this, slot, off](unsigned char* b) { *slot = reinterpret_cast<T*>(b + align(stage.size()) + off); });
    }
    md_status commit(std::vector<void*>* allocs) {
        const size_t zoff = align(stage.size());
        unsigned char* base = nullptr;
        MD_TRY(dev_upload(allocs, &base, (const unsigned char*)nullptr, zoff + zero_bytes));
        MD_CUDA(cudaMemcpy(base, stage.data(), stage.size(), cudaMemcpyHostToDevice));
        MD_CUDA(cudaMemset(base + zoff, 0, zero_bytes));
        for (auto& f : bind) f(base);
        return MD_OK;
    }
};

extern "C" md_status md_assemble(int N, const md_graph* g, double radius, double beta,
                                 const md_params* prm, md_op** out) {
    if (!out) { md_set_error("md_assemble: out is NULL"); return MD_ERR_ARG; }
    *out = nullptr;
    if (N < 2 || N > 1024) { md_set_error("md_assemble: N=%d outside [2, 1024]", N); return MD_ERR_ARG; }
    if (!g || !g->xyz || !g->edges || g->n_nodes < 2 || g->n_edges < 1 || g->elems_per_edge < 1) {
        md_set_error("md_assemble: invalid graph"); return MD_ERR_ARG;
    }
    if (!(radius > 0.0) || !(beta >= 0.0)) { md_set_error("md_assemble: radius must be > 0 and beta >= 0"); return MD_ERR_ARG; }
    const double k_omega = prm ? prm->k_omega : 1.0;
    const double sigma_omega = prm ? prm->sigma_omega : 0.0;
    const double k_lambda = prm ? prm->k_lambda : 1.0;
    const bool natural = prm && prm->natural_boundary;
    const double u_d = prm ? prm->u_d : 1.0;
    const int V = g->n_nodes, E = g->n_edges, m = g->elems_per_edge;
    if (prm && prm->n_dirichlet_1d > 0) {
        if (!prm->dirichlet_1d) { md_set_error("md_assemble: dirichlet_1d is NULL"); return MD_ERR_ARG; }
        for (int i = 0; i < prm->n_dirichlet_1d; ++i)
            if (prm->dirichlet_1d[i] < 0 || prm->dirichlet_1d[i] >= V) {
                md_set_error("md_assemble: 1D Dirichlet node %d is not a graph node", prm->dirichlet_1d[i]);
                return MD_ERR_ARG;
            }
    }
    if (prm && (prm->n_dirichlet_1d < 0 || !std::isfinite(prm->u_d))) { md_set_error("md_assemble: bad 1D Dirichlet data"); return MD_ERR_ARG; }
    if (natural && !(sigma_omega > 0.0) && !(prm->n_dirichlet_1d > 0 && beta > 0.0)) {
        md_set_error("md_assemble: natural conditions on the cube need sigma_omega > 0 or a coupled 1D Dirichlet node");
        return MD_ERR_ARG;
    }
    for (int e = 0; e < E; ++e) {
        int a = g->edges[2 * e], b = g->edges[2 * e + 1];
        if (a < 0 || a >= V || b < 0 || b >= V || a == b) { md_set_error("md_assemble: bad edge %d", e); return MD_ERR_ARG; }
    }
    for (int i = 0; i < 3 * V; ++i) {
        double c = g->xyz[i];
        if (!(c > 0.0 && c < 1.0)) { md_set_error("md_assemble: node coordinate %d outside (0,1)", i); return MD_ERR_ARG; }
    }

    const int M = N + 1;
    const long long n3ll = (long long)M * M * M;
    if (n3ll > (1LL << 30)) { md_set_error("md_assemble: grid too large"); return MD_ERR_ARG; }
    const int n3 = (int)n3ll;
    const double h = 1.0 / N;

    // ---- 1D mesh: graph nodes first, then interior points of each edge
    const int n1 = V + E * (m - 1);
    std::vector<Vec3> X1(n1);
    for (int i = 0; i < V; ++i) X1[i] = {g->xyz[3 * i], g->xyz[3 * i + 1], g->xyz[3 * i + 2]};
    std::vector<int> elA, elB;
    elA.reserve((size_t)E * m); elB.reserve((size_t)E * m);
    for (int e = 0; e < E; ++e) {
        int p = g->edges[2 * e], q = g->edges[2 * e + 1];
        Vec3 pa = X1[p], pb = X1[q];
        Vec3 d = sub(pb, pa);
        std::vector<int> chain;
        chain.push_back(p);
        for (int i = 1; i < m; ++i) {
            int id = V + e * (m - 1) + (i - 1);
            X1[id] = add(pa, scale((double)i / (double)m, d));
            chain.push_back(id);
        }
        chain.push_back(q);
        for (int i = 0; i < m; ++i) { elA.push_back(chain[i]); elB.push_back(chain[i + 1]); }
    }
    const int ne = (int)elA.size();
    const int nq = 2 * ne;

    // ---- forest check and elimination order (children before parents)
    std::vector<std::vector<int>> adj(n1);
    for (int e = 0; e < ne; ++e) { adj[elA[e]].push_back(elB[e]); adj[elB[e]].push_back(elA[e]); }
    std::vector<int> parent(n1, -2), bfs;
    bfs.reserve(n1);
    for (int r = 0; r < n1; ++r) {
        if (parent[r] != -2) continue;
        parent[r] = -1;
        size_t head = bfs.size();
        bfs.push_back(r);
        while (head < bfs.size()) {
            int u = bfs[head++];
            for (int v : adj[u]) {
                if (v == parent[u]) continue;
                if (parent[v] != -2) { md_set_error("md_assemble: the graph has a cycle"); return MD_ERR_ARG; }
                parent[v] = u;
                bfs.push_back(v);
            }
        }
    }
    // a repeated edge between the same two nodes is a cycle too
    {
        std::vector<std::pair<int, int>> ed;
        for (int e = 0; e < E; ++e) {
            int a = g->edges[2 * e], b = g->edges[2 * e + 1];
            ed.push_back({std::min(a, b), std::max(a, b)});
        }
        std::sort(ed.begin(), ed.end());
        if (std::adjacent_find(ed.begin(), ed.end()) != ed.end()) { md_set_error("md_assemble: repeated edge"); return MD_ERR_ARG; }
    }
    std::vector<int> order(bfs.rbegin(), bfs.rend());

    // ---- quadrature points, circle points, averaging rows
    const double gxi[2] = {(1.0 - 1.0 / std::sqrt(3.0)) / 2.0, (1.0 + 1.0 / std::sqrt(3.0)) / 2.0};
    const double S = std::sqrt(0.5);
    const double ccos[8] = {1.0, S, 0.0, -S, -1.0, -S, 0.0, S};
    const double csin[8] = {0.0, S, 1.0, S, 0.0, -S, -1.0, -S};
    // Dirichlet grid nodes (none with natural conditions on the cube faces)
    auto is_bd = [&](int i, int j, int k) {
        return !natural && (i == 0 || i == N || j == 0 || j == N || k == 0 || k == N);
    };

    std::vector<int> qa(nq), qb(nq);
    std::vector<double> psa(nq), psb(nq), wq(nq), elen(ne);
    std::vector<int> pi_ptr(nq + 1, 0);
    std::vector<int> pi_col;
    std::vector<double> pi_val;
    std::vector<Entry> row;
    for (int el = 0; el < ne; ++el) {
        Vec3 a = X1[elA[el]], b = X1[elB[el]];
        Vec3 d = sub(b, a);
        double L = norm(d);
        if (!(L > 0.0)) { md_set_error("md_assemble: zero-length element"); return MD_ERR_ARG; }
        elen[el] = L;
        Vec3 t = {d.x / L, d.y / L, d.z / L};
        double at[3] = {std::fabs(t.x), std::fabs(t.y), std::fabs(t.z)};
        int ax = 0;
        if (at[1] < at[ax]) ax = 1;
        if (at[2] < at[ax]) ax = 2;
        Vec3 ea = {ax == 0 ? 1.0 : 0.0, ax == 1 ? 1.0 : 0.0, ax == 2 ? 1.0 : 0.0};
        Vec3 v = cross(t, ea);
        double nv = norm(v);
        Vec3 n1v = {v.x / nv, v.y / nv, v.z / nv};
        Vec3 n2v = cross(t, n1v);
        for (int gp = 0; gp < 2; ++gp) {
            int q = 2 * el + gp;
            double xi = gxi[gp];
            Vec3 c = add(a, scale(xi, d));
            qa[q] = elA[el]; qb[q] = elB[el];
            psa[q] = 1.0 - xi; psb[q] = xi;
            wq[q] = L / 2.0;
            row.clear();
            for (int k = 0; k < 8; ++k) {
                Vec3 tmp = add(scale(ccos[k], n1v), scale(csin[k], n2v));
                Vec3 x = add(c, scale(radius, tmp));
                if (!(x.x >= 0.0 && x.x <= 1.0 && x.y >= 0.0 && x.y <= 1.0 && x.z >= 0.0 && x.z <= 1.0)) {
                    md_set_error("md_assemble: a cross-section circle leaves the cube (element %d)", el);
                    return MD_ERR_ARG;
                }
                double xs[3] = {x.x * (double)N, x.y * (double)N, x.z * (double)N};
                int cell[3];
                double fr[3];
                for (int dd = 0; dd < 3; ++dd) {
                    int ci = (int)std::floor(xs[dd]);
                    if (ci < 0) ci = 0;
                    if (ci > N - 1) ci = N - 1;
                    cell[dd] = ci;
                    fr[dd] = xs[dd] - (double)ci;
                }
                for (int corner = 0; corner < 8; ++corner) {
                    int ca = corner & 1, cb = (corner >> 1) & 1, cc = (corner >> 2) & 1;
                    double wx = ca ? fr[0] : 1.0 - fr[0];
                    double wy = cb ? fr[1] : 1.0 - fr[1];
                    double wz = cc ? fr[2] : 1.0 - fr[2];
                    int ii = cell[0] + ca, jj = cell[1] + cb, kk = cell[2] + cc;
                    if (is_bd(ii, jj, kk)) continue;
                    row.push_back({ii + M * (jj + M * kk), (wx * wy * wz) / 8.0});
                }
            }
            std::sort(row.begin(), row.end(), [](const Entry& p, const Entry& r) { return p.col < r.col; });
            for (size_t i = 0; i < row.size();) {
                size_t j = i;
                double s = 0.0;
                while (j < row.size() && row[j].col == row[i].col) { s += row[j].val; ++j; }
                pi_col.push_back(row[i].col);
                pi_val.push_back(s);
                i = j;
            }
            pi_ptr[q + 1] = (int)pi_col.size();
        }
    }

    // ---- Pi^T W over touched nodes: entries (q, Pi[q,n] w_q) by node, q ascending
    // within a node; nodes grouped by the apply's stencil tile, in node order
    // within a tile
    int ty = 1, tz = 1;
    apply_tile_shape(N, &ty, &tz);
    const int nyt = (N + 1 + ty - 1) / ty, nzt = (N + 1 + tz - 1) / tz;
    auto tile_of = [&](int node) {
        const int M = N + 1, z = node / (M * M), y = (node / M) % M;
        return (z / tz) * nyt + y / ty;
    };
    struct TE { int node, q; double v; };
    std::vector<TE> te(pi_col.size());
    if (n3 <= (1 << 22)) {
        // counting transpose of the q-major rows of Pi (entries arrive in q
        // order, so each node's stay in q order), then the touched nodes
        // visited tile by tile: tiles are (z, y) blocks, and node order within
        // a tile is (z, y, x) order
        std::vector<int> start((size_t)n3 + 1, 0);
        for (int c : pi_col) start[(size_t)c + 1] += 1;
        for (int i = 0; i < n3; ++i) start[(size_t)i + 1] += start[i];
        std::vector<TE> byn(pi_col.size());
        {
            std::vector<int> fill(start.begin(), start.end() - 1);
            for (int q = 0; q < nq; ++q)
                for (int j = pi_ptr[q]; j < pi_ptr[q + 1]; ++j) byn[fill[pi_col[j]]++] = {pi_col[j], q, pi_val[j] * wq[q]};
        }
        size_t k = 0;
        for (int zb = 0; zb < nzt; ++zb)
            for (int yb = 0; yb < nyt; ++yb)
                for (int z = zb * tz; z < std::min(M, (zb + 1) * tz); ++z)
                    for (int y = yb * ty; y < std::min(M, (yb + 1) * ty); ++y)
                        for (int x = 0; x < M; ++x) {
                            const int node = x + M * (y + M * z);
                            for (int e = start[node]; e < start[node + 1]; ++e) te[k++] = byn[e];
                        }
    } else {
        // very large grids: the same order by a sort on precomputed keys
        struct TK { int tile, node, q; double v; };
        std::vector<TK> tk;
        tk.reserve(pi_col.size());
        for (int q = 0; q < nq; ++q)
            for (int j = pi_ptr[q]; j < pi_ptr[q + 1]; ++j) tk.push_back({tile_of(pi_col[j]), pi_col[j], q, pi_val[j] * wq[q]});
        std::sort(tk.begin(), tk.end(), [](const TK& p, const TK& r) {
            if (p.tile != r.tile) return p.tile < r.tile;
            return p.node != r.node ? p.node < r.node : p.q < r.q;
        });
        for (size_t i = 0; i < tk.size(); ++i) te[i] = {tk[i].node, tk[i].q, tk[i].v};
    }
    // row sums of Pi (less than 1 where boundary weights were dropped)
    std::vector<double> pi_rowsum(nq, 0.0);
    for (int q = 0; q < nq; ++q)
        for (int j = pi_ptr[q]; j < pi_ptr[q + 1]; ++j) pi_rowsum[q] += pi_val[j];
    std::vector<int> tn_node, tn_ptr(1, 0), tn_q;
    // touch_m: diag of Pi^T W Pi at the node; touch_rs: its row sum (all entries
    // are >= 0), sum_q Pi[q,n] w_q sum_j Pi[q,j]
    std::vector<double> tn_v, touch_m, touch_rs;
    for (size_t i = 0; i < te.size();) {
        size_t j = i;
        double dm = 0.0, rs = 0.0;
        while (j < te.size() && te[j].node == te[i].node) {
            tn_q.push_back(te[j].q);
            tn_v.push_back(te[j].v);
            // Pi[q,n]^2 w_q = (Pi[q,n] w_q) * Pi[q,n]
            dm += te[j].v * (te[j].v / wq[te[j].q]);
            rs += te[j].v * pi_rowsum[te[j].q];
            ++j;
        }
        tn_node.push_back(te[i].node);
        tn_ptr.push_back((int)tn_q.size());
        touch_m.push_back(dm);
        touch_rs.push_back(rs);
        i = j;
    }
    const int ntouch = (int)tn_node.size();
    std::vector<int> tile_tptr((size_t)nyt * nzt + 1, 0);
    for (int i = 0; i < ntouch; ++i) tile_tptr[tile_of(tn_node[i]) + 1] += 1;
    for (size_t b = 1; b < tile_tptr.size(); ++b) tile_tptr[b] += tile_tptr[b - 1];

    // ---- 1D operators
    const double kappa = k_lambda * M_PI * radius * radius;
    // kappa K1 rows and Psi^T W rows per 1D node
    std::vector<std::map<int, double>> k1rows(n1);
    std::vector<std::vector<std::pair<int, double>>> pwrows(n1);
    std::vector<std::map<int, double>> brows(n1);  // B11
    std::vector<double> load1(n1, 0.0);
    for (int el = 0; el < ne; ++el) {
        int a = elA[el], b = elB[el];
        double L = elen[el];
        double kk = kappa / L;
        k1rows[a][a] += kk; k1rows[a][b] -= kk;
        k1rows[b][b] += kk; k1rows[b][a] -= kk;
        brows[a][a] += kk; brows[a][b] -= kk;
        brows[b][b] += kk; brows[b][a] -= kk;
        load1[a] += L / 2.0;
        load1[b] += L / 2.0;
        for (int gp = 0; gp < 2; ++gp) {
            int q = 2 * el + gp;
            pwrows[a].push_back({q, psa[q] * wq[q]});
            pwrows[b].push_back({q, psb[q] * wq[q]});
            brows[a][a] += beta * wq[q] * psa[q] * psa[q];
            brows[a][b] += beta * wq[q] * psa[q] * psb[q];
            brows[b][a] += beta * wq[q] * psb[q] * psa[q];
            brows[b][b] += beta * wq[q] * psb[q] * psb[q];
        }
    }
    // 1D Dirichlet nodes (dLambda_D): eliminated symmetrically.  Their known
    // value moves to the right-hand side through the columns of the full
    // operator: b0 += beta Pi^T W Psi_D u_d (the coupling columns), b1 -=
    // B11[:, D] u_d; then their rows and columns of B11 become the identity
    // (b1 = u_d there), their coupling columns vanish (Psi's values at those
    // nodes zero in the averaging difference), and their load is replaced.
    std::vector<char> isd(n1, 0);
    if (prm)
        for (int i = 0; i < prm->n_dirichlet_1d; ++i) isd[prm->dirichlet_1d[i]] = 1;
    const bool any_d = std::find(isd.begin(), isd.end(), 1) != isd.end();
    std::vector<double> rhs0, rhs1;
    if (any_d) {
        rhs0.assign((size_t)n3, 0.0);
        rhs1.assign((size_t)n1, 0.0);
        for (int q = 0; q < nq; ++q) {
            const double tD = (isd[qa[q]] ? psa[q] * u_d : 0.0) + (isd[qb[q]] ? psb[q] * u_d : 0.0);
            if (tD == 0.0) continue;
            for (int jj = pi_ptr[q]; jj < pi_ptr[q + 1]; ++jj) rhs0[pi_col[jj]] += beta * pi_val[jj] * wq[q] * tD;
        }
        for (int i = 0; i < n1; ++i) {
            if (isd[i]) { rhs1[i] = u_d; continue; }
            for (auto& kv : brows[i])
                if (isd[kv.first]) rhs1[i] -= kv.second * u_d;
        }
        for (int i = 0; i < n1; ++i) {
            if (isd[i]) {
                brows[i].clear();
                brows[i][i] = 1.0;
                k1rows[i].clear();
                k1rows[i][i] = 1.0;  // y1 = u1 on the row (no Psi^T W entries below)
                pwrows[i].clear();
                load1[i] = 0.0;
                continue;
            }
            for (auto it = brows[i].begin(); it != brows[i].end();) it = isd[it->first] ? brows[i].erase(it) : std::next(it);
            for (auto it = k1rows[i].begin(); it != k1rows[i].end();) it = isd[it->first] ? k1rows[i].erase(it) : std::next(it);
        }
        for (int q = 0; q < nq; ++q) {
            if (isd[qa[q]]) psa[q] = 0.0;
            if (isd[qb[q]]) psb[q] = 0.0;
        }
    }
    std::vector<int> k1_ptr(1, 0), k1_col, pw_ptr(1, 0), pw_q;
    std::vector<double> k1_v, pw_v, d1(n1);
    for (int i = 0; i < n1; ++i) {
        for (auto& kv : k1rows[i]) { k1_col.push_back(kv.first); k1_v.push_back(kv.second); }
        k1_ptr.push_back((int)k1_col.size());
        std::sort(pwrows[i].begin(), pwrows[i].end());
        for (auto& kv : pwrows[i]) { pw_q.push_back(kv.first); pw_v.push_back(kv.second); }
        pw_ptr.push_back((int)pw_q.size());
        d1[i] = brows[i][i];
    }
    // tree LDL^T of B11
    std::vector<double> dd(n1), tl(n1, 0.0), tdinv(n1);
    for (int i = 0; i < n1; ++i) dd[i] = brows[i][i];
    for (int idx = 0; idx < n1; ++idx) {
        int i = order[idx];
        if (!(dd[i] > 0.0)) { md_set_error("md_assemble: B11 is not positive definite (beta = 0?)"); return MD_ERR_ARG; }
        int p = parent[i];
        if (p >= 0) {
            double bpi = brows[p][i];
            tl[i] = bpi / dd[i];
            dd[p] -= tl[i] * bpi;
        }
    }
    for (int i = 0; i < n1; ++i) tdinv[i] = 1.0 / dd[i];
    std::vector<int> tr_order = order, tr_parent(n1);
    for (int i = 0; i < n1; ++i) tr_parent[i] = parent[i];
    // level schedule: height (leaves 0) from the children-first order, depth
    // (roots 0) from the reverse order; children lists in elimination order
    std::vector<int> hgt(n1, 0), dep(n1, 0), ch_ptr(n1 + 1, 0), ch_idx;
    for (int idx = 0; idx < n1; ++idx) {
        const int i = order[idx], p = parent[i];
        if (p >= 0) { hgt[p] = std::max(hgt[p], hgt[i] + 1); ch_ptr[p + 1] += 1; }
    }
    for (int idx = n1 - 1; idx >= 0; --idx) {
        const int i = order[idx], p = parent[i];
        dep[i] = p >= 0 ? dep[p] + 1 : 0;
    }
    for (int i = 0; i < n1; ++i) ch_ptr[i + 1] += ch_ptr[i];
    ch_idx.assign((size_t)ch_ptr[n1], 0);
    {
        std::vector<int> fill(ch_ptr.begin(), ch_ptr.end() - 1);
        for (int idx = 0; idx < n1; ++idx) {
            const int i = order[idx], p = parent[i];
            if (p >= 0) ch_idx[fill[p]++] = i;
        }
    }
    auto levels = [&](const std::vector<int>& key, std::vector<int>& ptr, std::vector<int>& nodes) {
        const int nl = n1 ? *std::max_element(key.begin(), key.end()) + 1 : 0;
        ptr.assign((size_t)nl + 1, 0);
        for (int i = 0; i < n1; ++i) ptr[key[i] + 1] += 1;
        for (int l = 0; l < nl; ++l) ptr[l + 1] += ptr[l];
        nodes.assign((size_t)n1, 0);
        std::vector<int> fill(ptr.begin(), ptr.end() - 1);
        for (int idx = 0; idx < n1; ++idx) nodes[fill[key[order[idx]]]++] = order[idx];
        return nl;
    };
    std::vector<int> lvu_ptr, lv_up, lvd_ptr, lv_dn;
    const int nlvu = levels(hgt, lvu_ptr, lv_up), nlvd = levels(dep, lvd_ptr, lv_dn);

    // ---- stencils and diagonal
    // Q1 stencil by offset class |dx|+|dy|+|dz| (h-scaled): stiffness {8/3, 0, -1/6, -1/12} h,
    // mass (h/6)^3 {64, 16, 4, 1}
    const double Kst[4] = {8.0 / 3.0 * h, 0.0, -1.0 / 6.0 * h, -1.0 / 12.0 * h};
    const double h3 = h * h * h;
    const double Mst[4] = {64.0 * h3 / 216.0, 16.0 * h3 / 216.0, 4.0 * h3 / 216.0, 1.0 * h3 / 216.0};
    md_op* op = new md_op();
    InstDesc& D = op->h;
    memset(&D, 0, sizeof(D));
    D.N = N; D.n3 = n3; D.n1 = n1; D.nq = nq; D.ntouch = ntouch; D.nsegs = E;
    D.natural = natural ? 1 : 0;
    D.n = (long long)n3 + n1;
    D.h = h; D.beta = beta;
    D.ty = ty; D.tz = tz; D.nyt = nyt; D.ntiles = nyt * nzt;
    D.mdiv = (unsigned int)((((unsigned long long)1 << 32) + (unsigned long long)N) / (unsigned long long)(N + 1));
    for (int c = 0; c < 4; ++c) {
        D.st64[c] = k_omega * Kst[c] + sigma_omega * Mst[c];
        D.st32[c] = (float)D.st64[c];
        D.ms64[c] = Mst[c];
    }
    // alpha = ||diag(C_II)|| / sqrt(n_I) over the unknown grid nodes (all of
    // them with natural conditions, where the diagonal of a node on a face,
    // edge or corner has the stencil centre times 1/2 per boundary axis)
    {
        const double c0 = D.st64[0];
        auto fac = [&](int i) { return (i == 0 || i == N) ? 0.5 : 1.0; };
        std::vector<double> dg;
        long long nI = 0;
        double ss = 0.0;
        if (natural) {
            dg.assign((size_t)n3, 0.0);
            for (int k = 0; k < M; ++k)
                for (int j = 0; j < M; ++j)
                    for (int i = 0; i < M; ++i) dg[i + M * (j + M * k)] = c0 * fac(i) * fac(j) * fac(k);
            for (int i = 0; i < ntouch; ++i) dg[tn_node[i]] += beta * touch_m[i];
            for (double v : dg) ss += v * v;
            nI = n3;
        } else {
            nI = (long long)(N - 1) * (N - 1) * (N - 1);
            ss = (double)nI * c0 * c0;
            for (int i = 0; i < ntouch; ++i) {
                double dc = c0 + beta * touch_m[i];
                ss += dc * dc - c0 * c0;
            }
        }
        D.alpha = nI > 0 ? std::sqrt(ss / (double)nI) : 1.0;
    }

    auto fail = [&](md_status s) { dev_free_all(&op->allocs); delete op; return s; };
#define UP(x) do { md_status s_ = (x); if (s_ != MD_OK) return fail(s_); } while (0)
    UploadArena ar;
    ar.up(&D.pi_ptr, pi_ptr); ar.up(&D.pi_col, pi_col); ar.up(&D.pi_v64, pi_val); ar.up32(&D.pi_v32, pi_val);
    ar.up(&D.qa, qa); ar.up(&D.qb, qb);
    ar.up(&D.psa64, psa); ar.up(&D.psb64, psb); ar.up32(&D.psa32, psa); ar.up32(&D.psb32, psb);
    ar.up(&D.tn_node, tn_node); ar.up(&D.tn_ptr, tn_ptr); ar.up(&D.tn_q, tn_q); ar.up(&D.tile_tptr, tile_tptr);
    ar.up(&D.tn_v64, tn_v); ar.up32(&D.tn_v32, tn_v);
    ar.up(&D.k1_ptr, k1_ptr); ar.up(&D.k1_col, k1_col); ar.up(&D.k1_v64, k1_v); ar.up32(&D.k1_v32, k1_v);
    ar.up(&D.pw_ptr, pw_ptr); ar.up(&D.pw_q, pw_q); ar.up(&D.pw_v64, pw_v); ar.up32(&D.pw_v32, pw_v);
    ar.up(&D.load1, load1);
    if (any_d) { ar.up(&D.rhs0, rhs0); ar.up(&D.rhs1, rhs1); }
    {
        D.nlvu = nlvu; D.nlvd = nlvd;
        ar.up(&D.tr_order, tr_order); ar.up(&D.tr_parent, tr_parent);
        ar.up(&D.lvu_ptr, lvu_ptr); ar.up(&D.lv_up, lv_up); ar.up(&D.ch_ptr, ch_ptr); ar.up(&D.ch_idx, ch_idx);
        ar.up(&D.lvd_ptr, lvd_ptr); ar.up(&D.lv_dn, lv_dn);
        ar.up(&D.tr_l64, tl); ar.up(&D.tr_dinv64, tdinv); ar.up32(&D.tr_l32, tl); ar.up32(&D.tr_dinv32, tdinv);
    }
    {
        std::vector<double> segs((size_t)E * 6);
        for (int e = 0; e < E; ++e) {
            int a = g->edges[2 * e], b = g->edges[2 * e + 1];
            for (int c = 0; c < 3; ++c) { segs[6 * e + c] = g->xyz[3 * a + c]; segs[6 * e + 3 + c] = g->xyz[3 * b + c]; }
        }
        ar.up(&D.segs, segs);
    }
    ar.zeros(&D.dist, (size_t)n3);
    ar.zeros(&D.dinv64, (size_t)D.n);
    ar.zeros(&D.dinv32, (size_t)D.n);
    ar.zeros(&D.sminv32, (size_t)n3);
    ar.zeros(&D.t64, (size_t)nq);
    ar.zeros(&D.t32, (size_t)nq);
    ar.zeros(&D.lift32, (size_t)n3);
    ar.zeros(&D.ltouch32, (size_t)ntouch);
    UP(ar.commit(&op->allocs));
    UP(dev_upload(&op->allocs, &op->d, &D, 1));
    {
        std::vector<const InstDesc*> one{&op->h};
        UP(build_tables(one, &op->tabs, &op->allocs));
        long long z = 0;
        UP(dev_upload(&op->allocs, &op->off0, &z, 1));
    }
    UP(launch_dist(op, 0));
    UP(launch_dinv_fill(op, touch_m, touch_rs, d1, 0));
    {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return fail(md_cuda_status(e, "md_assemble sync", __FILE__, __LINE__));
    }
#undef UP
    op->n_touch_nodes = ntouch;
    *out = op;
    return MD_OK;
}

extern "C" void md_op_destroy(md_op* op) {
    if (!op) return;
    for (int i = 0; i < 3; ++i)
        if (op->solver_cache[i]) md_batch_destroy(op->solver_cache[i]);
    dev_free_all(&op->allocs);
    delete op;
}

extern "C" md_status md_op_get_info(const md_op* op, md_op_info_t* info) {
    if (!op || !info) { md_set_error("md_op_get_info: NULL argument"); return MD_ERR_ARG; }
    info->N = op->h.N; info->n3 = op->h.n3; info->n1 = op->h.n1; info->nq = op->h.nq;
    info->n_touch = op->h.ntouch; info->n = op->h.n; info->alpha = op->h.alpha; info->beta = op->h.beta;
    return MD_OK;
}

extern "C" md_status md_op_distance(const md_op* op, float* d, md_stream s) {
    if (!op || !d) { md_set_error("md_op_distance: NULL argument"); return MD_ERR_ARG; }
    MD_CUDA(cudaMemcpyAsync(d, op->h.dist, sizeof(float) * op->h.n3, cudaMemcpyDeviceToDevice, (cudaStream_t)s));
    return MD_OK;
}
