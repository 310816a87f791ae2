// Grid-transfer and correction kernels of the CGP step (the paper's Eqs. 20-23, 29-30).
#include <algorithm>
#include <vector>

#include "ctx.h"

namespace cgp {

namespace {

// Eqs. 20-21 with Eq. 30: b_c[eta] = -(rho/dt) sum_j (Dx_c[eta,j] u~_f[xi_j].x + Dy_c[eta,j] u~_f[xi_j].y),
// the injection u~_c[j] = u~_f[xi_j] fused into the gather (cif[k] = xi of column ci[k]).
// Rows held at p = 0 get 0. One warp-group of `lanes` threads per coarse row.
__global__ void k_restrict_rhs(int nc, const int* __restrict__ rp, const int* __restrict__ cif,
                               const double* __restrict__ Dxy, const double* __restrict__ ut,
                               const unsigned char* __restrict__ pm, double scale, double* __restrict__ bc,
                               int lanes) {
    const int gid = (blockIdx.x * blockDim.x + threadIdx.x);
    const int row = gid / lanes, l = gid & (lanes - 1);
    double acc = 0.0;
    if (row < nc) {
        const int k1 = rp[row + 1];
        for (int k = rp[row] + l; k < k1; k += lanes) {
            double dx, dy, ux, uy;
            load2(Dxy, k, dx, dy);
            load2(ut, cif[k], ux, uy);
            acc += dx * ux + dy * uy;
        }
    }
    acc = group_sum(acc, lanes);
    if (row < nc && l == 0) bc[row] = pm[row] ? 0.0 : scale * acc;
}

// Eq. 22 through the table of Eq. 29: p_{k+1}[alpha] = (p_k[beta] + p_k[gamma]) / 2.
__global__ void k_prolong(int n, const int2* __restrict__ sp, const double* __restrict__ src, double* __restrict__ dst) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int2 bg = sp[i];
    dst[i] = 0.5 * (src[bg.x] + src[bg.y]);
}

// g = G p_f, G_ij = int phi_i grad psi_j (both components), `lanes` threads per row.
__global__ void k_gradient(int nf, const int* __restrict__ rp, const int* __restrict__ ci,
                           const double* __restrict__ Gxy, const double* __restrict__ pf, double* __restrict__ g,
                           int lanes) {
    const int gid = (blockIdx.x * blockDim.x + threadIdx.x);
    const int row = gid / lanes, l = gid & (lanes - 1);
    double ax = 0.0, ay = 0.0;
    if (row < nf) {
        const int k1 = rp[row + 1];
        for (int k = rp[row] + l; k < k1; k += lanes) {
            double gx, gy;
            load2(Gxy, k, gx, gy);
            const double p = pf[ci[k]];
            ax += gx * p;
            ay += gy * p;
        }
    }
    ax = group_sum(ax, lanes);
    ay = group_sum(ay, lanes);
    if (row < nf && l == 0) store2(g, row, ax, ay);
}

// Eq. 23 with Eq. 15's dt/rho: u = u~ - (dt/rho) w, then prescribed velocity values at Dirichlet
// nodes (Eq. 3). Optionally copies w out.
// u = u~ - c w with Dirichlet values restored (Eq. 23); the outputs go to position perm[i] of the
// refinement order when perm is given (the caller's arrays), else to i.
__global__ void k_correct(int nf, const double* ut, const double* __restrict__ w, double c,
                          const unsigned char* __restrict__ mask, const double* __restrict__ gd, double* u,
                          double* gp_out, const int* __restrict__ perm) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    double tx, ty, wx, wy, gx, gy;
    load2(ut, i, tx, ty);
    load2(w, i, wx, wy);
    load2(gd, i, gx, gy);
    const unsigned char m = mask[i];
    const int o = perm ? perm[i] : i;
    store2(u, o, (m & CGP_BC_U) ? gx : tx - c * wx, (m & CGP_BC_V) ? gy : ty - c * wy);
    if (gp_out) store2(gp_out, o, wx, wy);
}

// Between the stored fine order and the refinement order: dst[i] = src[perm[i]] (to_stored) or
// dst[perm[i]] = src[i], for `comps` interleaved values per node (1 or 2).
__global__ void k_permute(int n, int comps, const int* __restrict__ perm, const double* __restrict__ src,
                          double* __restrict__ dst, int to_stored) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int p = perm[i];
    const int from = to_stored ? p : i, to = to_stored ? i : p;
    if (comps == 2) {
        double x, y;
        load2(src, from, x, y);
        store2(dst, to, x, y);
    } else {
        dst[to] = src[from];
    }
}

__global__ void k_copy_pairs(const double2* __restrict__ src, double2* __restrict__ dst, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[i];
}

// Fine divergence d_i = sum_j Dx_f[i,j] u~_x[j] + Dy_f[i,j] u~_y[j] (D_f = G_f on the fine mesh,
// where velocity and pressure share the P1 space), one thread per row.
__global__ void k_divergence(int nf, const int* __restrict__ rp, const int* __restrict__ ci,
                             const double* __restrict__ Gxy, const double* __restrict__ ut, double* __restrict__ d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    double acc = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
        double gx, gy, ux, uy;
        load2(Gxy, k, gx, gy);
        load2(ut, ci[k], ux, uy);
        acc += gx * ux + gy * uy;
    }
    d[i] = acc;
}

// One level of P^T (the transpose of Eq. 29's prolongation): r_k[i] = r_{k+1}[self[i]] (the
// parent-coincident row alpha with beta = gamma = i, weight 1) + 1/2 sum over the finer nodes
// alpha whose pair (beta, gamma) contains i with beta != gamma of r_{k+1}[alpha], in the fixed
// order of the inverse child list. With `pm` (the last level) the result is scaled and zeroed at
// pressure-held rows: b_c = scale P^T d.
__global__ void k_restrict_transpose(int n, const int* __restrict__ ptr, const int* __restrict__ idx,
                                     const int* __restrict__ self, const double* __restrict__ src,
                                     double* __restrict__ dst, const unsigned char* __restrict__ pm, double scale) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double h = 0.0;
    for (int m = ptr[i]; m < ptr[i + 1]; ++m) h += src[idx[m]];
    const double r = src[self[i]] + 0.5 * h;
    dst[i] = pm ? (pm[i] ? 0.0 : scale * r) : r;
}

// Fine divergence scaled straight into b_c (no refinement: P = I).
__global__ void k_scale_mask(int n, const double* __restrict__ src, const unsigned char* __restrict__ pm,
                             double scale, double* __restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = pm[i] ? 0.0 : scale * src[i];
}

// Incremental forms: p += phi, and with the rotational term also - mu chi where
// chi = -(dt/rho) b_c / m_i (m the lumped coarse mass), i.e. p += phi + c b_c / m_i, c = mu dt / rho.
__global__ void k_pressure_update(int n, const double* __restrict__ bc, const double* __restrict__ phi,
                                  const double* __restrict__ m, double c, double* __restrict__ p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = p[i] + phi[i];
    if (m) v += c * bc[i] / m[i];
    p[i] = v;
}

// Row sums of a CSR matrix (the lumped mass from the assembled coarse mass matrix).
__global__ void k_row_sums(int n, const int* __restrict__ rp, const double* __restrict__ val, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) s += val[k];
    out[i] = s;
}

}  // namespace

cudaError_t launch_restrict_rhs(cgp_ctx_s* c, const double* ut, double* bc, cudaStream_t s) {
    const double scale = -(c->prm.rho / c->prm.dt);
    if (c->prm.restrict_mode == 1) {
        // b_c = -(rho/dt) P^T D_f u~_f: fine divergence, then P^T from the finest level down
        k_divergence<<<(c->nf + 255) / 256, 256, 0, s>>>(c->nf, c->F.rp, c->F.ci, c->Gxy, ut, c->gal_div);
        if (c->levels == 0) {
            k_scale_mask<<<(c->nc + 255) / 256, 256, 0, s>>>(c->nc, c->gal_div, c->p_mask, scale, bc);
            return cudaGetLastError();
        }
        const double* src = c->gal_div;
        for (int k = c->levels - 1; k >= 0; --k) {
            const int n = c->lv_n[k];
            const bool last = k == 0;
            double* dst = last ? bc : c->pl[k - 1];   // pl[k - 1] holds N_k values
            k_restrict_transpose<<<(n + 255) / 256, 256, 0, s>>>(n, c->gal_ptr[k], c->gal_idx[k], c->gal_self[k], src,
                                                                dst, last ? c->p_mask : nullptr, scale);
            src = dst;
        }
        return cudaGetLastError();
    }
    const int lanes = c->sh_c.lanes, threads = 256;
    const long long tot = (long long)c->nc * lanes;
    k_restrict_rhs<<<(int)((tot + threads - 1) / threads), threads, 0, s>>>(
        c->nc, c->C.rp, c->cif_su, c->Dc_xy, ut, c->p_mask, scale, bc, lanes);
    return cudaGetLastError();
}

cudaError_t launch_prolong(cgp_ctx_s* c, const double* pc, double* pf, cudaStream_t s) {
    const double* src = pc;
    for (int k = 0; k < c->levels; ++k) {
        const int n = c->lv_n[k + 1];
        double* dst = (k + 1 == c->levels) ? pf : c->pl[k];
        k_prolong<<<(n + 255) / 256, 256, 0, s>>>(n, c->sp[k], src, dst);
        src = dst;
    }
    if (c->levels == 0) {
        cudaError_t e = cudaMemcpyAsync(pf, pc, sizeof(double) * (size_t)c->nf, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

cudaError_t launch_gradient(cgp_ctx_s* c, const double* pf, double* grad, cudaStream_t s) {
    const int lanes = c->sh_f.lanes, threads = 256;
    const long long tot = (long long)c->nf * lanes;
    k_gradient<<<(int)((tot + threads - 1) / threads), threads, 0, s>>>(c->nf, c->F.rp, c->F.ci, c->Gxy, pf, grad, lanes);
    return cudaGetLastError();
}

cudaError_t launch_correct(cgp_ctx_s* c, const double* ut, const double* w, double* u, double* gp_out,
                           cudaStream_t s, bool to_public) {
    k_correct<<<(c->nf + 255) / 256, 256, 0, s>>>(c->nf, ut, w, c->prm.dt / c->prm.rho, c->vel_mask, c->g, u, gp_out,
                                                  to_public ? c->fperm : nullptr);
    return cudaGetLastError();
}

cudaError_t fine_to_stored(cgp_ctx_s* c, const double* pub, double* st, int comps, cudaStream_t s) {
    if (!c->fperm) {
        if (pub == st) return cudaSuccess;
        return cudaMemcpyAsync(st, pub, sizeof(double) * comps * (size_t)c->nf, cudaMemcpyDeviceToDevice, s);
    }
    k_permute<<<(c->nf + 255) / 256, 256, 0, s>>>(c->nf, comps, c->fperm, pub, st, 1);
    return cudaGetLastError();
}

cudaError_t fine_to_public(cgp_ctx_s* c, const double* st, double* pub, int comps, cudaStream_t s) {
    if (!c->fperm) {
        if (pub == st) return cudaSuccess;
        return cudaMemcpyAsync(pub, st, sizeof(double) * comps * (size_t)c->nf, cudaMemcpyDeviceToDevice, s);
    }
    k_permute<<<(c->nf + 255) / 256, 256, 0, s>>>(c->nf, comps, c->fperm, st, pub, 0);
    return cudaGetLastError();
}

namespace {

struct PredictArgs {
    const double* in;   // the latest value v^n
    double* out;        // the prediction (may be `in`)
    double* prev;       // v^(n-1), replaced by v^n
    double* prev2;      // v^(n-2), replaced by v^(n-1)
    double* prev3;      // v^(n-3), replaced by v^(n-2)
    int* flag;          // number of recorded values, 0 .. 3
    int n, order;       // order 1: linear, 2: quadratic, 3: cubic extrapolation
};

// Extrapolation in time of a solver's initial guess from the values the previous calls recorded,
// the polynomial through the last min(order, recorded) + 1 values taken one step on:
// 4 v^n - 6 v^(n-1) + 4 v^(n-2) - v^(n-3), 3 v^n - 3 v^(n-1) + v^(n-2), 2 v^n - v^(n-1) or v^n;
// then the history shifts by v^n. blockIdx.y selects the vector of a batch. The flag is only read
// here; k_predict_flag, launched after this kernel, counts it up.
__global__ void k_predict(const PredictArgs* __restrict__ tab, PredictArgs single) {
    const PredictArgs a = tab ? tab[blockIdx.y] : single;
    const int have = *a.flag;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const int k = min(have, a.order);
    const double vn = a.in[i], v1 = a.prev[i], v2 = a.prev2[i];
    double o = vn;
    if (k >= 3) o = 4.0 * (vn + v2) - 6.0 * v1 - a.prev3[i];
    else if (k == 2) o = fma(3.0, vn - v1, v2);
    else if (k == 1) o = 2.0 * vn - v1;
    a.out[i] = o;
    a.prev3[i] = v2;
    a.prev2[i] = v1;
    a.prev[i] = vn;
}

__global__ void k_predict_flag(const PredictArgs* __restrict__ tab, PredictArgs single) {
    const PredictArgs a = tab ? tab[blockIdx.x] : single;
    if (threadIdx.x == 0) *a.flag = min(*a.flag + 1, 3);
}

}  // namespace

cudaError_t launch_predict_vec(const double* in, double* out, double* prev, double* prev2, double* prev3, int* flag,
                               int n, int order, cudaStream_t s) {
    const PredictArgs a{in, out, prev, prev2, prev3, flag, n, order};
    k_predict<<<dim3((n + 255) / 256, 1), 256, 0, s>>>(nullptr, a);
    k_predict_flag<<<1, 32, 0, s>>>(nullptr, a);
    return cudaGetLastError();
}

cudaError_t launch_predict(cgp_ctx_s* c, double* pc, cudaStream_t s) {
    return launch_predict_vec(pc, pc, c->pc_prev, c->pc_prev2, c->pc_prev3, c->pc_flag, c->nc,
                              std::max(1, c->prm.warm_start), s);
}

// Batched predictors of every instance with warm_start >= 1 (coarse pressure and mass-solve initial
// guess, both in place), one launch at the start of a step, while both vectors still hold their
// values from the previous step.
cudaError_t batch_predict_build(cgp_batch_s* b) {
    b->predict = false;
    int nmax = 0;
    std::vector<PredictArgs> tab;
    for (int i = 0; i < b->n; ++i) {
        cgp_ctx_s* c = b->ctx[i];
        if (c->prm.warm_start < 1) continue;
        const int n2 = 2 * c->nf, order = c->prm.warm_start;
        tab.push_back(PredictArgs{b->pc[i], b->pc[i], c->pc_prev, c->pc_prev2, c->pc_prev3, c->pc_flag, c->nc, order});
        tab.push_back(PredictArgs{c->w, c->w, c->w_prev, c->w_prev2, c->w_prev3, c->w_flag, n2, order});
        nmax = std::max({nmax, c->nc, n2});
    }
    if (tab.empty()) return cudaSuccess;
    void* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(PredictArgs) * tab.size());
    if (e != cudaSuccess) return e;
    b->allocs.push_back(d);
    if ((e = cudaMemcpy(d, tab.data(), sizeof(PredictArgs) * tab.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
        return e;
    b->tab_predict = d;
    b->predict_nmax = nmax;
    b->predict_count = (int)tab.size();
    b->predict = true;
    return cudaSuccess;
}

cudaError_t batch_predict_launch(cgp_batch_s* b, cudaStream_t s) {
    if (!b->predict) return cudaSuccess;
    const PredictArgs* tab = (const PredictArgs*)b->tab_predict;
    k_predict<<<dim3((b->predict_nmax + 255) / 256, b->predict_count), 256, 0, s>>>(tab, PredictArgs{});
    k_predict_flag<<<b->predict_count, 32, 0, s>>>(tab, PredictArgs{});
    return cudaGetLastError();
}

cudaError_t launch_copy_pairs(const double* src, double* dst, int n, cudaStream_t s) {
    k_copy_pairs<<<(n + 255) / 256, 256, 0, s>>>((const double2*)src, (double2*)dst, n);
    return cudaGetLastError();
}

// G_f P p_c into grad_n: the pressure term of the incremental forms' momentum right-hand side.
cudaError_t launch_pressure_term(cgp_ctx_s* c, const double* pc, cudaStream_t s) {
    cudaError_t e = launch_prolong(c, pc, c->pf, s);
    if (e != cudaSuccess) return e;
    return launch_gradient(c, c->pf, c->grad_n, s);
}

cudaError_t launch_pressure_update(cgp_ctx_s* c, const double* bc, const double* phi, double* pc, cudaStream_t s) {
    const bool rot = c->prm.projection == 2;
    k_pressure_update<<<(c->nc + 255) / 256, 256, 0, s>>>(c->nc, bc, phi, rot ? c->mlump_c : nullptr,
                                                          c->prm.mu * c->prm.dt / c->prm.rho, pc);
    return cudaGetLastError();
}

// Lumped coarse mass: the coarse P1 mass matrix assembled into tmp (nnz_c doubles, zeroed here),
// then its row sums.
cudaError_t launch_lumped_mass(cgp_ctx_s* c, double* tmp, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(tmp, 0, sizeof(double) * (size_t)c->C.nnz, s);
    if (e != cudaSuccess) return e;
    if ((e = launch_const_assembly(c->EC, tmp, nullptr, nullptr, s)) != cudaSuccess) return e;
    k_row_sums<<<(c->nc + 255) / 256, 256, 0, s>>>(c->nc, c->C.rp, tmp, c->mlump_c);
    return cudaGetLastError();
}

// Inverse child lists of the s^p tables (host, once per context): for level k, node i of level k
// lists the nodes alpha >= N_k of level k + 1 whose pair (beta, gamma) contains i, in increasing
// alpha (a node with beta = gamma = i only is the parent-coincident row, taken with weight 1).
int galerkin_build(cgp_ctx_s* c) {
    const HostMesh& H = c->hm;
    for (int k = 0; k < c->levels; ++k) {
        const int nk = H.lv[k].n, nk1 = H.lv[k + 1].n;
        const std::vector<int>& sp = H.sp[k];   // [nk1][2]
        // the finer node coinciding with each coarser one (beta = gamma) and the inverse lists of
        // the midpoints (beta != gamma), in the order of the finer level's stored numbering
        std::vector<int> ptr(nk + 1, 0), idx, self(nk, -1);
        for (int a = 0; a < nk1; ++a) {
            if (sp[2 * a] == sp[2 * a + 1]) {
                self[sp[2 * a]] = a;
                continue;
            }
            ptr[sp[2 * a] + 1] += 1;
            ptr[sp[2 * a + 1] + 1] += 1;
        }
        for (int i = 0; i < nk; ++i)
            if (self[i] < 0) return CGP_ERR_MESH;
        for (int i = 0; i < nk; ++i) ptr[i + 1] += ptr[i];
        idx.assign(ptr[nk], 0);
        std::vector<int> pos(ptr.begin(), ptr.end() - 1);
        for (int a = 0; a < nk1; ++a) {
            if (sp[2 * a] == sp[2 * a + 1]) continue;
            idx[pos[sp[2 * a]]++] = a;
            idx[pos[sp[2 * a + 1]]++] = a;
        }
        void *dp = nullptr, *di = nullptr, *ds = nullptr;
        if (cudaMalloc(&dp, sizeof(int) * ptr.size()) != cudaSuccess) return CGP_ERR_NOMEM;
        c->allocs.push_back(dp);
        if (cudaMalloc(&di, sizeof(int) * std::max<size_t>(1, idx.size())) != cudaSuccess) return CGP_ERR_NOMEM;
        c->allocs.push_back(di);
        if (cudaMalloc(&ds, sizeof(int) * self.size()) != cudaSuccess) return CGP_ERR_NOMEM;
        c->allocs.push_back(ds);
        if (cudaMemcpy(dp, ptr.data(), sizeof(int) * ptr.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            (!idx.empty() && cudaMemcpy(di, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice) != cudaSuccess) ||
            cudaMemcpy(ds, self.data(), sizeof(int) * self.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return CGP_ERR_CUDA;
        c->gal_ptr.push_back((int*)dp);
        c->gal_idx.push_back((int*)di);
        c->gal_self.push_back((int*)ds);
    }
    return CGP_OK;
}

namespace {

// Per-instance arguments of the batched gathers between the persistent stages of a batched step
// (one launch per stage for all instances; blockIdx.y selects the instance).
struct GatherArgs {
    int nc, nf, levels;
    int lv_n[CGP_MAX_LEVELS + 1];
    const int* rp_c;
    const int* cif;
    const double* Dxy_c;
    const unsigned char* pm;
    double scale;
    const double* ut;
    double* bc;
    const int2* sp[CGP_MAX_LEVELS];
    double* pl[CGP_MAX_LEVELS];
    const double* pc;
    double* pf;
    const int* rp_f;
    const int* ci_f;
    const double* Gxy;
    double* grad;
    const double* w;
    double cdr;
    const unsigned char* vmask;
    const double* g;
    double* u;
    const int* perm;    // refinement-order position of stored fine node i (nullptr: i)
};

// The same arithmetic as k_restrict_rhs (one lane per row), k_prolong, k_gradient (one lane per
// row) and k_correct, for instance blockIdx.y of the batch table.
__global__ void k_restrict_b(const GatherArgs* __restrict__ tab) {
    const GatherArgs& a = tab[blockIdx.y];
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= a.nc) return;
    double acc = 0.0;
    for (int k = a.rp_c[row]; k < a.rp_c[row + 1]; ++k) {
        double dx, dy, ux, uy;
        load2(a.Dxy_c, k, dx, dy);
        load2(a.ut, a.cif[k], ux, uy);
        acc += dx * ux + dy * uy;
    }
    a.bc[row] = a.pm[row] ? 0.0 : a.scale * acc;
}

__global__ void k_prolong_b(const GatherArgs* __restrict__ tab, int level) {
    const GatherArgs& a = tab[blockIdx.y];
    if (level >= a.levels) return;
    const int n = a.lv_n[level + 1];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* src = level == 0 ? a.pc : a.pl[level - 1];
    double* dst = level + 1 == a.levels ? a.pf : a.pl[level];
    const int2 bg = a.sp[level][i];
    dst[i] = 0.5 * (src[bg.x] + src[bg.y]);
}

__global__ void k_gradient_b(const GatherArgs* __restrict__ tab) {
    const GatherArgs& a = tab[blockIdx.y];
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= a.nf) return;
    double ax = 0.0, ay = 0.0;
    for (int k = a.rp_f[row]; k < a.rp_f[row + 1]; ++k) {
        double gx, gy;
        load2(a.Gxy, k, gx, gy);
        const double p = a.pf[a.ci_f[k]];
        ax += gx * p;
        ay += gy * p;
    }
    store2(a.grad, row, ax, ay);
}

__global__ void k_correct_b(const GatherArgs* __restrict__ tab) {
    const GatherArgs& a = tab[blockIdx.y];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.nf) return;
    double tx, ty, wx, wy, gx, gy;
    load2(a.ut, i, tx, ty);
    load2(a.w, i, wx, wy);
    load2(a.g, i, gx, gy);
    const unsigned char m = a.vmask[i];
    store2(a.u, a.perm ? a.perm[i] : i, (m & CGP_BC_U) ? gx : tx - a.cdr * wx, (m & CGP_BC_V) ? gy : ty - a.cdr * wy);
}

// The velocities of the instances that store their fine nodes in another order, gathered into
// that order (instance blockIdx.y of the table) at the start of a batched step.
struct PermArgs {
    int n;
    const int* perm;
    const double* pub;
    double* st;
};

__global__ void k_permute_b(const PermArgs* __restrict__ tab) {
    const PermArgs& a = tab[blockIdx.y];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    double x, y;
    load2(a.pub, a.perm[i], x, y);
    store2(a.st, i, x, y);
}

}  // namespace

// Table of the batched gathers; false (per-instance launches stay) when an instance uses the
// Galerkin restriction or has no refinement level.
bool batch_gather_build(cgp_batch_s* b) {
    b->gather = false;
    std::vector<GatherArgs> tab(b->n);
    int maxc = 0, maxf = 0, maxl = 0, maxlv = 0;
    for (int i = 0; i < b->n; ++i) {
        cgp_ctx_s* c = b->ctx[i];
        if (c->prm.restrict_mode != 0 || c->levels < 1 || c->levels > CGP_MAX_LEVELS) return false;
        GatherArgs& a = tab[i];
        a = GatherArgs();
        a.nc = c->nc;
        a.nf = c->nf;
        a.levels = c->levels;
        for (int k = 0; k <= c->levels; ++k) a.lv_n[k] = c->lv_n[k];
        a.rp_c = c->C.rp;
        a.cif = c->cif_su;
        a.Dxy_c = c->Dc_xy;
        a.pm = c->p_mask;
        a.scale = -(c->prm.rho / c->prm.dt);
        a.ut = c->ut;
        a.bc = c->bc;
        for (int k = 0; k < c->levels; ++k) {
            a.sp[k] = c->sp[k];
            a.pl[k] = c->pl[k];
        }
        a.pc = b->pc[i];
        a.pf = c->pf;
        a.rp_f = c->F.rp;
        a.ci_f = c->F.ci;
        a.Gxy = c->Gxy;
        a.grad = c->grad;
        a.w = c->w;
        a.cdr = c->prm.dt / c->prm.rho;
        a.vmask = c->vel_mask;
        a.g = c->g;
        a.u = b->u[i];
        a.perm = c->fperm;
        maxc = std::max(maxc, c->nc);
        maxf = std::max(maxf, c->nf);
        maxl = std::max(maxl, c->levels);
        for (int k = 1; k <= c->levels; ++k) maxlv = std::max(maxlv, c->lv_n[k]);
    }
    void* d = nullptr;
    if (cudaMalloc(&d, sizeof(GatherArgs) * tab.size()) != cudaSuccess) return false;
    b->allocs.push_back(d);
    if (cudaMemcpy(d, tab.data(), sizeof(GatherArgs) * tab.size(), cudaMemcpyHostToDevice) != cudaSuccess) return false;
    b->tab_gather = d;
    b->gather_nc = maxc;
    b->gather_nf = maxf;
    b->gather_levels = maxl;
    b->gather_nlv = maxlv;
    b->gather = true;
    return true;
}

cudaError_t batch_restrict_launch(cgp_batch_s* b, cudaStream_t s) {
    k_restrict_b<<<dim3((b->gather_nc + 255) / 256, b->n), 256, 0, s>>>((const GatherArgs*)b->tab_gather);
    return cudaGetLastError();
}

cudaError_t batch_prolong_gradient_launch(cgp_batch_s* b, cudaStream_t s) {
    const GatherArgs* t = (const GatherArgs*)b->tab_gather;
    for (int k = 0; k < b->gather_levels; ++k) k_prolong_b<<<dim3((b->gather_nlv + 255) / 256, b->n), 256, 0, s>>>(t, k);
    k_gradient_b<<<dim3((b->gather_nf + 255) / 256, b->n), 256, 0, s>>>(t);
    return cudaGetLastError();
}

cudaError_t batch_correct_launch(cgp_batch_s* b, cudaStream_t s) {
    k_correct_b<<<dim3((b->gather_nf + 255) / 256, b->n), 256, 0, s>>>((const GatherArgs*)b->tab_gather);
    return cudaGetLastError();
}

cudaError_t batch_perm_build(cgp_batch_s* b) {
    b->perm_count = 0;
    std::vector<PermArgs> tab;
    int nmax = 0;
    for (int i = 0; i < b->n; ++i) {
        cgp_ctx_s* c = b->ctx[i];
        if (!c->fperm) continue;
        tab.push_back(PermArgs{c->nf, c->fperm, b->u[i], c->u_int});
        nmax = std::max(nmax, c->nf);
    }
    if (tab.empty()) return cudaSuccess;
    void* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(PermArgs) * tab.size());
    if (e != cudaSuccess) return e;
    b->allocs.push_back(d);
    if ((e = cudaMemcpy(d, tab.data(), sizeof(PermArgs) * tab.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    b->tab_perm = d;
    b->perm_nmax = nmax;
    b->perm_count = (int)tab.size();
    return cudaSuccess;
}

cudaError_t batch_perm_launch(cgp_batch_s* b, cudaStream_t s) {
    if (b->perm_count == 0) return cudaSuccess;
    k_permute_b<<<dim3((b->perm_nmax + 255) / 256, b->perm_count), 256, 0, s>>>((const PermArgs*)b->tab_perm);
    return cudaGetLastError();
}

namespace {
// out = the extrapolation in time of order k through v0 (newest) .. vk: 2 v0 - v1, 3 v0 - 3 v1 + v2,
// 4 v0 - 6 v1 + 4 v2 - v3 (the predictors of k_predict, without a history)
__global__ void k_extrapolate(size_t n, int order, const double* __restrict__ v0, const double* __restrict__ v1,
                              const double* __restrict__ v2, const double* __restrict__ v3, double* __restrict__ out) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double o = v0[i];
    if (order >= 3) o = 4.0 * (v0[i] + v2[i]) - 6.0 * v1[i] - v3[i];
    else if (order == 2) o = fma(3.0, v0[i] - v1[i], v2[i]);
    else if (order == 1) o = 2.0 * v0[i] - v1[i];
    out[i] = o;
}
}  // namespace

}  // namespace cgp

extern "C" int cgp_extrapolate(long long n, int order, const double* v0, const double* v1, const double* v2,
                               const double* v3, double* out, void* stream) {
    if (n <= 0 || order < 0 || order > 3 || !v0 || !out) return CGP_ERR_ARG;
    if ((order >= 1 && !v1) || (order >= 2 && !v2) || (order >= 3 && !v3)) return CGP_ERR_ARG;
    cgp::k_extrapolate<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>((size_t)n, order, v0, v1, v2, v3,
                                                                                      out);
    return cudaGetLastError() == cudaSuccess ? CGP_OK : CGP_ERR_CUDA;
}
