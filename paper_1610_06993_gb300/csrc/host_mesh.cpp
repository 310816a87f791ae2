// Host-side mesh preprocessing: see host_mesh.h.
#include "host_mesh.h"

#include <algorithm>
#include <cstdint>
#include <unordered_map>
#include <utility>

#include "subdomain.h"

namespace cgp {

namespace {

// Unique edges in order of first visit (triangles in order, local edges a-b, b-c, c-a).
// edge_of[t*3+e] = edge index; edges[2*i], edges[2*i+1] = (min, max) endpoints; count = uses.
void first_visit_edges(int n, const std::vector<int>& tri, std::vector<int>& edges,
                       std::vector<int>& edge_of, std::vector<int>& count) {
    const int t = (int)(tri.size() / 3);
    std::unordered_map<uint64_t, int> id;
    id.reserve((size_t)t * 2);
    edges.clear();
    count.clear();
    edge_of.assign((size_t)t * 3, -1);
    for (int e = 0; e < t; ++e) {
        for (int k = 0; k < 3; ++k) {
            int a = tri[e * 3 + k], b = tri[e * 3 + (k + 1) % 3];
            int lo = std::min(a, b), hi = std::max(a, b);
            uint64_t key = (uint64_t)lo * (uint64_t)n + (uint64_t)hi;
            auto it = id.find(key);
            int idx;
            if (it == id.end()) {
                idx = (int)(edges.size() / 2);
                id.emplace(key, idx);
                edges.push_back(lo);
                edges.push_back(hi);
                count.push_back(0);
            } else {
                idx = it->second;
            }
            edge_of[e * 3 + k] = idx;
            count[idx] += 1;
        }
    }
}

void build_csr(int n, const std::vector<int>& edges, HostCsr& c) {
    c.n = n;
    const int ne = (int)(edges.size() / 2);
    std::vector<int> deg(n, 1);
    for (int i = 0; i < ne; ++i) {
        deg[edges[2 * i]]++;
        deg[edges[2 * i + 1]]++;
    }
    c.rp.assign(n + 1, 0);
    for (int i = 0; i < n; ++i) c.rp[i + 1] = c.rp[i] + deg[i];
    c.nnz = c.rp[n];
    c.ci.assign(c.nnz, 0);
    std::vector<int> fill(c.rp.begin(), c.rp.end() - 1);
    for (int i = 0; i < n; ++i) c.ci[fill[i]++] = i;
    for (int i = 0; i < ne; ++i) {
        int a = edges[2 * i], b = edges[2 * i + 1];
        c.ci[fill[a]++] = b;
        c.ci[fill[b]++] = a;
    }
    c.diag.assign(n, 0);
    for (int i = 0; i < n; ++i) {
        std::sort(c.ci.begin() + c.rp[i], c.ci.begin() + c.rp[i + 1]);
        c.diag[i] = (int)(std::lower_bound(c.ci.begin() + c.rp[i], c.ci.begin() + c.rp[i + 1], i) - c.ci.begin());
    }
}

int build_elems(const HostLevel& lv, const HostCsr& c, HostElems& el) {
    const int t = lv.t;
    el.slot.assign((size_t)t * 9, 0);
    for (int e = 0; e < t; ++e) {
        for (int a = 0; a < 3; ++a) {
            int r = lv.tri[e * 3 + a];
            for (int b = 0; b < 3; ++b) {
                int col = lv.tri[e * 3 + b];
                auto beg = c.ci.begin() + c.rp[r], end = c.ci.begin() + c.rp[r + 1];
                auto it = std::lower_bound(beg, end, col);
                if (it == end || *it != col) return CGP_ERR_MESH;
                el.slot[(size_t)e * 9 + a * 3 + b] = (int)(it - c.ci.begin());
            }
        }
    }
    // Greedy colouring: no two elements of one colour share a node, so an element loop over one
    // colour writes every CSR row from at most one thread.
    std::vector<uint64_t> used(lv.n, 0);
    std::vector<int> col(t);
    int ncol = 0;
    for (int e = 0; e < t; ++e) {
        const int* v = &lv.tri[e * 3];
        uint64_t forb = used[v[0]] | used[v[1]] | used[v[2]];
        if (~forb == 0) return CGP_ERR_MESH;   // more than 64 colours: degenerate mesh
        int k = __builtin_ctzll(~forb);
        col[e] = k;
        ncol = std::max(ncol, k + 1);
        for (int a = 0; a < 3; ++a) used[v[a]] |= (1ull << k);
    }
    el.colptr.assign(ncol + 1, 0);
    for (int e = 0; e < t; ++e) el.colptr[col[e] + 1]++;
    for (int k = 0; k < ncol; ++k) el.colptr[k + 1] += el.colptr[k];
    std::vector<int> fill(el.colptr.begin(), el.colptr.end() - 1);
    el.perm.assign(t, 0);
    for (int e = 0; e < t; ++e) el.perm[fill[col[e]]++] = e;
    return CGP_OK;
}

void boundary_flags(int n, const std::vector<int>& edges, const std::vector<int>& count,
                    std::vector<unsigned char>& onb) {
    onb.assign(n, 0);
    for (size_t i = 0; i < count.size(); ++i) {
        if (count[i] == 1) {
            onb[edges[2 * i]] = 1;
            onb[edges[2 * i + 1]] = 1;
        }
    }
}

}  // namespace

void build_sell(const HostCsr& c, int C, int sigma, HostSell& out) {
    out = HostSell();
    out.C = C;
    const int n = c.n;
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    for (int w0 = 0; w0 < n; w0 += sigma) {
        const int w1 = std::min(n, w0 + sigma);
        std::stable_sort(order.begin() + w0, order.begin() + w1, [&](int a, int b) {
            return (c.rp[a + 1] - c.rp[a]) > (c.rp[b + 1] - c.rp[b]);
        });
    }
    out.nslices = (n + C - 1) / C;
    out.ptr.assign(out.nslices + 1, 0);
    out.width.assign(out.nslices, 0);
    out.perm.assign((size_t)out.nslices * C, -1);
    for (int s = 0; s < out.nslices; ++s) {
        int w = 0;
        for (int l = 0; l < C; ++l) {
            const int q = s * C + l;
            if (q < n) {
                out.perm[q] = order[q];
                w = std::max(w, c.rp[order[q] + 1] - c.rp[order[q]]);
            }
        }
        out.width[s] = w;
        out.ptr[s + 1] = out.ptr[s] + w * C;
    }
    out.col.assign(out.ptr[out.nslices], 0);
    out.src.assign(out.ptr[out.nslices], -1);
    for (int s = 0; s < out.nslices; ++s) {
        for (int l = 0; l < C; ++l) {
            const int r = out.perm[s * C + l];
            for (int k = 0; k < out.width[s]; ++k) {
                const size_t p = (size_t)out.ptr[s] + (size_t)k * C + l;
                if (r >= 0 && k < c.rp[r + 1] - c.rp[r]) {
                    out.col[p] = c.ci[c.rp[r] + k];
                    out.src[p] = c.rp[r] + k;
                } else {
                    out.col[p] = r >= 0 ? r : 0;
                    out.src[p] = -1;
                }
            }
        }
    }
}

int build_host_mesh(const cgp_mesh_desc* d, int levels, HostMesh& out, bool renumber_fine) {
    if (!d || !d->xy_host || !d->tri_host || d->n_nodes <= 2 || d->n_tris <= 0) return CGP_ERR_ARG;
    if (levels < 0 || levels > 4) return CGP_ERR_ARG;
    HostLevel c;
    c.n = d->n_nodes;
    c.t = d->n_tris;
    c.xy.assign(d->xy_host, d->xy_host + 2 * (size_t)c.n);
    c.tri.assign(d->tri_host, d->tri_host + 3 * (size_t)c.t);
    // validation: indices in range, strictly positive (counter-clockwise) area
    for (int e = 0; e < c.t; ++e) {
        int v[3];
        for (int k = 0; k < 3; ++k) {
            v[k] = c.tri[e * 3 + k];
            if (v[k] < 0 || v[k] >= c.n) return CGP_ERR_MESH;
        }
        const double* p0 = &c.xy[2 * v[0]];
        const double* p1 = &c.xy[2 * v[1]];
        const double* p2 = &c.xy[2 * v[2]];
        double a2 = (p1[0] - p0[0]) * (p2[1] - p0[1]) - (p2[0] - p0[0]) * (p1[1] - p0[1]);
        if (!(a2 > 0.0)) return CGP_ERR_MESH;
    }
    out = HostMesh();
    out.lv.push_back(std::move(c));
    std::vector<int> edges, edge_of, count;
    out.su.resize(out.lv[0].n);
    for (int i = 0; i < out.lv[0].n; ++i) out.su[i] = i;

    for (int k = 0; k <= levels; ++k) {
        HostLevel& L = out.lv[k];
        first_visit_edges(L.n, L.tri, edges, edge_of, count);
        for (int cnt : count)
            if (cnt > 2) return CGP_ERR_MESH;   // non-manifold edge
        if (k == 0) boundary_flags(L.n, edges, count, out.onb_c);
        if (k == levels) {
            boundary_flags(L.n, edges, count, out.onb_f);
            break;
        }
        // one conforming 1:4 split: parents keep their numbers, midpoints are appended in order
        // of first visit; s^p pairs (alpha, alpha) for parents and the edge ends for midpoints.
        const int ne = (int)(edges.size() / 2);
        HostLevel F;
        F.n = L.n + ne;
        F.t = 4 * L.t;
        F.xy.resize(2 * (size_t)F.n);
        std::copy(L.xy.begin(), L.xy.end(), F.xy.begin());
        std::vector<int> sp(2 * (size_t)F.n);
        for (int i = 0; i < L.n; ++i) sp[2 * i] = sp[2 * i + 1] = i;
        for (int i = 0; i < ne; ++i) {
            int a = edges[2 * i], b = edges[2 * i + 1];
            F.xy[2 * (L.n + i)] = 0.5 * (L.xy[2 * a] + L.xy[2 * b]);
            F.xy[2 * (L.n + i) + 1] = 0.5 * (L.xy[2 * a + 1] + L.xy[2 * b + 1]);
            sp[2 * (L.n + i)] = a;
            sp[2 * (L.n + i) + 1] = b;
        }
        F.tri.resize(3 * (size_t)F.t);
        for (int e = 0; e < L.t; ++e) {
            int a = L.tri[e * 3], b = L.tri[e * 3 + 1], cc = L.tri[e * 3 + 2];
            int mab = L.n + edge_of[e * 3], mbc = L.n + edge_of[e * 3 + 1], mca = L.n + edge_of[e * 3 + 2];
            int kids[12] = {a, mab, mca, mab, b, mbc, mca, mbc, cc, mab, mbc, mca};
            std::copy(kids, kids + 12, F.tri.begin() + (size_t)e * 12);
        }
        out.sp.push_back(std::move(sp));
        // s^u: parents keep their indices, so the coarse node's fine index is unchanged
        out.lv.push_back(std::move(F));
    }
    // Stored order of the fine nodes: along a Hilbert curve of their coordinates, so that the rows
    // of a warp, and the columns they gather, lie close together (in the refinement order a
    // parent's fine neighbours are midpoints created far apart). The s^p rows of the last level,
    // s^u and the boundary flags follow; the coarser levels keep the refinement order.
    if (renumber_fine && levels >= 1) {
        HostLevel& F = out.lv[levels];
        out.fperm = hilbert_order(F.xy, F.n);
        std::vector<int> inv(F.n);
        for (int i = 0; i < F.n; ++i) inv[out.fperm[i]] = i;
        std::vector<double> xy(2 * (size_t)F.n);
        std::vector<unsigned char> onb(F.n);
        const std::vector<int>& sp0 = out.sp[levels - 1];
        std::vector<int> sp(sp0.size());
        for (int i = 0; i < F.n; ++i) {
            const int p = out.fperm[i];
            xy[2 * i] = F.xy[2 * p];
            xy[2 * i + 1] = F.xy[2 * p + 1];
            onb[i] = out.onb_f[p];
            sp[2 * i] = sp0[2 * p];
            sp[2 * i + 1] = sp0[2 * p + 1];
        }
        for (int& v : F.tri) v = inv[v];
        for (int& x : out.su) x = inv[x];
        F.xy.swap(xy);
        out.onb_f.swap(onb);
        out.sp[levels - 1].swap(sp);
        // triangles follow their nodes (the assembly's element loops then read and write nearby
        // rows): stable sort by the smallest stored node index
        std::vector<int> tkey(F.t);
        for (int t = 0; t < F.t; ++t)
            tkey[t] = std::min({F.tri[3 * t], F.tri[3 * t + 1], F.tri[3 * t + 2]});
        out.tperm.resize(F.t);
        for (int t = 0; t < F.t; ++t) out.tperm[t] = t;
        std::stable_sort(out.tperm.begin(), out.tperm.end(), [&](int a, int b) { return tkey[a] < tkey[b]; });
        std::vector<int> tri(F.tri.size());
        for (int t = 0; t < F.t; ++t)
            for (int a = 0; a < 3; ++a) tri[3 * (size_t)t + a] = F.tri[3 * (size_t)out.tperm[t] + a];
        F.tri.swap(tri);
    }
    // CSR patterns and element data of the coarse and fine meshes
    {
        HostLevel& Lc = out.lv[0];
        first_visit_edges(Lc.n, Lc.tri, edges, edge_of, count);
        build_csr(Lc.n, edges, out.coarse);
        int s = build_elems(Lc, out.coarse, out.ec);
        if (s != CGP_OK) return s;
    }
    {
        HostLevel& Lf = out.lv[levels];
        first_visit_edges(Lf.n, Lf.tri, edges, edge_of, count);
        build_csr(Lf.n, edges, out.fine);
        int s = build_elems(Lf, out.fine, out.ef);
        if (s != CGP_OK) return s;
    }
    return CGP_OK;
}

}  // namespace cgp
