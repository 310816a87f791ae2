// Flow diagnostics of the paper's benchmark flows (Sect. 3.2: reattachment length of the
// backward-facing step; Sect. 3.3: drag and lift of the cylinder, split into pressure and viscous
// parts). Standard definitions (the paper prints none for the forces):
//   force on a body  F = sum over its boundary edges of int sigma n_b, sigma = -p I + mu (grad u +
//                    grad u^T), n_b the unit normal from the body into the fluid; p is P1 along the
//                    edge (trapezoid rule, exact), grad u the constant P1 gradient of the fluid
//                    triangle that owns the edge; p = P p_c, the coarse pressure prolonged (Eq. 29);
//   wall shear       tau = mu t . (grad u) n_f per wall edge (t the unit tangent towards larger x,
//                    n_f the unit normal into the fluid); the reattachment point is the first x
//                    past a start abscissa where tau turns from negative to non-negative, linear
//                    between edge midpoints.
#include <algorithm>
#include <cmath>
#include <vector>

#include "ctx.h"

namespace cgp {

namespace {

// Unit normal from the body into the fluid for a boundary edge a -> b that is CCW in its owning
// fluid triangle (the fluid lies to the left, so the body to the right).
__device__ __forceinline__ void edge_frame(const double* __restrict__ xy, int a, int b, double& len, double& nx,
                                           double& ny, double& tx, double& ty) {
    const double dx = xy[2 * b] - xy[2 * a], dy = xy[2 * b + 1] - xy[2 * a + 1];
    len = sqrt(dx * dx + dy * dy);
    tx = dx / len;
    ty = dy / len;
    nx = -ty;   // left of a -> b: into the fluid
    ny = tx;
}

// Constant P1 velocity gradient of fine triangle t: G[c][d] = d u_c / d x_d.
__device__ __forceinline__ void tri_grad(const int* __restrict__ tri, const double* __restrict__ geo,
                                         const double* __restrict__ u, int t, double G[2][2]) {
    const double* g = geo + 8 * (size_t)t;
    G[0][0] = G[0][1] = G[1][0] = G[1][1] = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double ux, uy;
        load2(u, tri[3 * t + k], ux, uy);
        G[0][0] += ux * g[1 + k];
        G[0][1] += ux * g[4 + k];
        G[1][0] += uy * g[1 + k];
        G[1][1] += uy * g[4 + k];
    }
}

// Pressure and viscous force on the body: one block, edges strided over its threads, a fixed-order
// block reduction (deterministic). out[0..1] pressure force, out[2..3] viscous force.
__global__ void __launch_bounds__(256) k_body_force(int ne, const int4* __restrict__ e, const double* __restrict__ xy,
                                                    const int* __restrict__ tri, const double* __restrict__ geo,
                                                    const double* __restrict__ u, const double* __restrict__ p,
                                                    double mu, double* __restrict__ out) {
    __shared__ double s_red[32 * 4];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < ne; i += blockDim.x) {
        const int4 q = e[i];
        double len, nx, ny, tx, ty;
        edge_frame(xy, q.x, q.y, len, nx, ny, tx, ty);
        const double pm = 0.5 * (p[q.x] + p[q.y]) * len;
        acc[0] -= pm * nx;
        acc[1] -= pm * ny;
        double G[2][2];
        tri_grad(tri, geo, u, q.z, G);
        const double sxx = 2.0 * G[0][0], sxy = G[0][1] + G[1][0], syy = 2.0 * G[1][1];
        acc[2] += mu * len * (sxx * nx + sxy * ny);
        acc[3] += mu * len * (sxy * nx + syy * ny);
    }
    block_sum<4>(acc, s_red);
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) out[k] = acc[k];
}

// Wall shear per wall edge (edges sorted by midpoint x on the host).
__global__ void k_wall_shear(int ne, const int4* __restrict__ e, const double* __restrict__ xy, const int* __restrict__ tri,
                             const double* __restrict__ geo, const double* __restrict__ u, double mu,
                             double* __restrict__ xs, double* __restrict__ tau) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    const int4 q = e[i];
    double len, nx, ny, tx, ty;
    edge_frame(xy, q.x, q.y, len, nx, ny, tx, ty);
    if (tx < 0.0) {
        tx = -tx;
        ty = -ty;
    }
    double G[2][2];
    tri_grad(tri, geo, u, q.z, G);
    xs[i] = 0.5 * (xy[2 * q.x] + xy[2 * q.y]);
    tau[i] = mu * (tx * (G[0][0] * nx + G[0][1] * ny) + ty * (G[1][0] * nx + G[1][1] * ny));
}

// The first crossing from tau < 0 to tau >= 0 past x_start (a sequential scan of at most a few
// thousand edges by one thread); NaN if there is none.
__global__ void k_reattach(int ne, const double* __restrict__ xs, const double* __restrict__ tau, double x_start,
                           double* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double r = __longlong_as_double(0x7ff8000000000000ll);
    for (int k = 0; k + 1 < ne; ++k) {
        if (xs[k] < x_start) continue;
        if (tau[k] < 0.0 && tau[k + 1] >= 0.0) {
            r = xs[k] - tau[k] * (xs[k + 1] - xs[k]) / (tau[k + 1] - tau[k]);
            break;
        }
    }
    *out = r;
}

}  // namespace

}  // namespace cgp

using namespace cgp;

extern "C" {

int cgp_set_surface(cgp_ctx c, int which, const unsigned char* mask, int* n_edges) {
    if (!c || !mask || which < 0 || which > 1) return CGP_ERR_ARG;
    const HostLevel& F = c->hm.lv[c->levels];
    const std::vector<int>& fp = c->hm.fperm;   // the mask is in the refinement order
    auto pub = [&](int v) { return fp.empty() ? v : fp[v]; };
    // boundary edges (one owning triangle), in the owner's CCW order
    std::vector<long long> key;
    std::vector<int4> loc;
    key.reserve(3 * (size_t)F.t);
    loc.reserve(3 * (size_t)F.t);
    for (int t = 0; t < F.t; ++t)
        for (int k = 0; k < 3; ++k) {
            const int a = F.tri[3 * t + k], b = F.tri[3 * t + (k + 1) % 3];
            key.push_back((long long)std::min(a, b) * F.n + std::max(a, b));
            loc.push_back(make_int4(a, b, t, 0));
        }
    std::vector<int> ord(key.size());
    for (size_t i = 0; i < ord.size(); ++i) ord[i] = (int)i;
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return key[x] < key[y]; });
    std::vector<int4> sel;
    for (size_t i = 0; i < ord.size();) {
        size_t j = i;
        while (j < ord.size() && key[ord[j]] == key[ord[i]]) ++j;
        if (j - i == 1) {
            const int4 q = loc[ord[i]];
            if (mask[pub(q.x)] && mask[pub(q.y)]) sel.push_back(q);
        }
        i = j;
    }
    // body edges in triangle order, wall edges by midpoint x
    if (which == 0) {
        std::stable_sort(sel.begin(), sel.end(), [](const int4& x, const int4& y) { return x.z < y.z; });
    } else {
        auto mid = [&](const int4& q) { return 0.5 * (F.xy[2 * q.x] + F.xy[2 * q.y]); };
        std::stable_sort(sel.begin(), sel.end(), [&](const int4& x, const int4& y) { return mid(x) < mid(y); });
    }
    cgp_ctx_s::Surface& S = c->surf[which];
    if (S.e) cudaFree(S.e);
    if (S.xs) cudaFree(S.xs);
    S = cgp_ctx_s::Surface();
    S.n = (int)sel.size();
    if (n_edges) *n_edges = S.n;
    if (S.n == 0) return CGP_OK;
    if (cudaMalloc(&S.e, sizeof(int4) * sel.size()) != cudaSuccess) return CGP_ERR_NOMEM;
    if (cudaMalloc(&S.xs, 2 * sizeof(double) * sel.size()) != cudaSuccess) return CGP_ERR_NOMEM;
    if (cudaMemcpy(S.e, sel.data(), sizeof(int4) * sel.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return CGP_ERR_CUDA;
    return CGP_OK;
}

int cgp_body_force(cgp_ctx c, const double* u_dev, const double* pc_dev, double* force_dev, void* stream) {
    if (!c || !u_dev || !pc_dev || !force_dev) return CGP_ERR_ARG;
    if (c->surf[0].n == 0) return CGP_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    const double* u = u_dev;
    if (c->fperm) {
        if (c->u_asm == c->u_int) c->u_asm = nullptr;   // the copy no longer holds the assembly's u^n
        if (fine_to_stored(c, u_dev, c->u_int, 2, s) != cudaSuccess) return CGP_ERR_CUDA;
        u = c->u_int;
    }
    if (launch_prolong(c, pc_dev, c->pf, s) != cudaSuccess) return CGP_ERR_CUDA;
    k_body_force<<<1, 256, 0, s>>>(c->surf[0].n, c->surf[0].e, c->xy_f, c->EF.tri, c->EF.geo, u, c->pf,
                                   c->prm.mu, force_dev);
    return cudaGetLastError() == cudaSuccess ? CGP_OK : CGP_ERR_CUDA;
}

int cgp_reattachment(cgp_ctx c, const double* u_dev, double x_start, double* xr_dev, double* x_dev, double* tau_dev,
                     void* stream) {
    if (!c || !u_dev || !xr_dev) return CGP_ERR_ARG;
    const cgp_ctx_s::Surface& S = c->surf[1];
    if (S.n == 0) return CGP_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    double* xs = x_dev ? x_dev : S.xs;
    double* tau = tau_dev ? tau_dev : S.xs + S.n;
    const double* u = u_dev;
    if (c->fperm) {
        if (c->u_asm == c->u_int) c->u_asm = nullptr;   // the copy no longer holds the assembly's u^n
        if (fine_to_stored(c, u_dev, c->u_int, 2, s) != cudaSuccess) return CGP_ERR_CUDA;
        u = c->u_int;
    }
    k_wall_shear<<<(S.n + 255) / 256, 256, 0, s>>>(S.n, S.e, c->xy_f, c->EF.tri, c->EF.geo, u, c->prm.mu, xs, tau);
    k_reattach<<<1, 32, 0, s>>>(S.n, xs, tau, x_start, xr_dev);
    return cudaGetLastError() == cudaSuccess ? CGP_OK : CGP_ERR_CUDA;
}

}  // extern "C"
