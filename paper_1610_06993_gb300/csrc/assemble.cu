// P1 finite-element assembly on the device (the paper's Eqs. 16-19).
//
// Element integrals of a triangle T with area |T| and constant shape-function gradients
// grad phi_i = (y_j - y_k, x_k - x_j) / (2|T|), (i, j, k) cyclic:
//   mass        M_ab = |T| (1 + delta_ab) / 12
//   stiffness   K_ab = |T| grad phi_a . grad phi_b
//   div / grad  D_ab = |T| / 3 * grad phi_b            (int phi_a d phi_b, not integrated by parts)
//   convection  N_ab = |T| / 12 * (sum_k u_k + u_a) . grad phi_b     (u in P1)
// Element loops run one colour at a time; elements of one colour share no node, so every CSR
// slot is updated by one thread per colour: no atomics and a fixed summation order.
#include "ctx.h"
#include "assemble_kernels.cuh"

namespace cgp {

namespace {

__global__ void k_geometry(const double* __restrict__ xy, const int* __restrict__ tri, int t,
                           double* __restrict__ geo) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= t) return;
    int v0 = tri[3 * e], v1 = tri[3 * e + 1], v2 = tri[3 * e + 2];
    double x0 = xy[2 * v0], y0 = xy[2 * v0 + 1];
    double x1 = xy[2 * v1], y1 = xy[2 * v1 + 1];
    double x2 = xy[2 * v2], y2 = xy[2 * v2 + 1];
    double area = 0.5 * ((x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0));
    double inv2a = 1.0 / (2.0 * area);
    double* g = geo + 8 * (size_t)e;
    g[0] = area;
    g[1] = (y1 - y2) * inv2a;   // d/dx phi_0 = (y_1 - y_2) / 2|T|
    g[2] = (y2 - y0) * inv2a;
    g[3] = (y0 - y1) * inv2a;
    g[4] = (x2 - x1) * inv2a;   // d/dy phi_0 = (x_2 - x_1) / 2|T|
    g[5] = (x0 - x2) * inv2a;
    g[6] = (x1 - x0) * inv2a;
    g[7] = 0.0;
}

// One colour of the constant matrices: M, K and the interleaved (Dx, Dy) pair.
__global__ void k_const_colour(int k0, int k1, const int* __restrict__ perm, const int* __restrict__ slot,
                               const double* __restrict__ geo, double* M, double* K, double* Dxy) {
    int k = k0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= k1) return;
    int e = perm[k];
    const double* g = geo + 8 * (size_t)e;
    double area = g[0];
    const int* sl = slot + 9 * (size_t)e;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            int s = sl[a * 3 + b];
            if (M) M[s] += area * (a == b ? 2.0 : 1.0) / 12.0;
            if (K) K[s] += area * (g[1 + a] * g[1 + b] + g[4 + a] * g[4 + b]);
            if (Dxy) {
                Dxy[2 * (size_t)s] += area / 3.0 * g[1 + b];
                Dxy[2 * (size_t)s + 1] += area / 3.0 * g[4 + b];
            }
        }
    }
}

// Symmetric elimination of pressure-Dirichlet rows/columns (Eq. 14 and the pin): zero the row and
// column, unit diagonal. Also the Jacobi inverse diagonal and the FP32 copies.
__global__ void k_pressure_bc(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                              const unsigned char* __restrict__ pm, const double* __restrict__ Kraw,
                              double* K, float* K32, double* dinv, float* dinv32) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool mi = pm[i] != 0;
    double diag = 1.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
        int j = ci[k];
        double v;
        if (mi || pm[j]) v = (i == j) ? 1.0 : 0.0;
        else v = Kraw[k];
        if (i == j) diag = v;
        K[k] = v;
        K32[k] = (float)v;
    }
    dinv[i] = 1.0 / diag;
    dinv32[i] = (float)(1.0 / diag);
}

__global__ void k_make_A0(int nnz, double rho, double dtmu, const double* __restrict__ M,
                          const double* __restrict__ K, double* A0) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nnz) A0[k] = rho * M[k] + dtmu * K[k];
}

__global__ void k_inv_diag(int n, const int* __restrict__ diag, const double* __restrict__ val, double* dinv) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dinv[i] = 1.0 / val[diag[i]];
}

__global__ void k_to_f32(int n, const double* __restrict__ src, float* dst) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (float)src[i];
}

}  // namespace

cudaError_t launch_geometry(const double* xy, const int* tri, int t, double* geo, cudaStream_t s) {
    k_geometry<<<(t + 255) / 256, 256, 0, s>>>(xy, tri, t, geo);
    return cudaGetLastError();
}

namespace {
// The element gradients scaled once by dt rho |T| / 12, the factor of every convection entry
// (Eq. 16's N; A carries dt rho N), so the per-step kernels need no division and fewer FP64
// products (this GPU issues FP64 at a small fraction of its FP32 rate).
__global__ void k_conv_scale(const double* __restrict__ geo, int t, double dtrho, double* __restrict__ conv) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= t) return;
    const double* g = geo + 8 * (size_t)e;
    const double c = dtrho * (g[0] / 12.0);
    double* o = conv + 6 * (size_t)e;
#pragma unroll
    for (int k = 0; k < 6; ++k) o[k] = c * g[1 + k];
}
}  // namespace

cudaError_t launch_conv_scale(const double* geo, int t, double dtrho, double* conv, cudaStream_t s) {
    k_conv_scale<<<(t + 255) / 256, 256, 0, s>>>(geo, t, dtrho, conv);
    return cudaGetLastError();
}

cudaError_t launch_const_assembly(const DevElems& E, double* M, double* K, double* Dxy, cudaStream_t s) {
    for (int c = 0; c < E.ncol; ++c) {
        int k0 = E.colptr[c], k1 = E.colptr[c + 1];
        if (k1 <= k0) continue;
        k_const_colour<<<(k1 - k0 + 255) / 256, 256, 0, s>>>(k0, k1, E.perm, E.slot, E.geo, M, K, Dxy);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_apply_pressure_bc(cgp_ctx_s* c, cudaStream_t s) {
    k_pressure_bc<<<(c->nc + 255) / 256, 256, 0, s>>>(c->nc, c->C.rp, c->C.ci, c->p_mask, c->Kc_raw, c->Kc,
                                                       c->Kc32, c->dinvK, c->dinvK32);
    return cudaGetLastError();
}

cudaError_t launch_make_A0(cgp_ctx_s* c, const double* K, cudaStream_t s) {
    const int nnz = c->F.nnz;
    k_make_A0<<<(nnz + 255) / 256, 256, 0, s>>>(nnz, c->prm.rho, c->prm.dt * c->prm.mu, c->M, K, c->A0);
    k_inv_diag<<<(c->nf + 255) / 256, 256, 0, s>>>(c->nf, c->F.diag, c->M, c->dinvM);
    k_to_f32<<<(nnz + 255) / 256, 256, 0, s>>>(nnz, c->M, c->M32);
    k_to_f32<<<(c->nf + 255) / 256, 256, 0, s>>>(c->nf, c->dinvM, c->dinvM32);
    return cudaGetLastError();
}

namespace {

StepAsmArgs asm_args(cgp_ctx_s* c, const double* u, SyncWords* sw) {
    StepAsmArgs a;
    a.nf = c->nf;
    a.nnz = c->F.nnz;
    a.ncol = c->EF.ncol;
    a.colptr = c->EF.colptr_dev;
    a.perm = c->EF.perm;
    a.slot = c->EF.slot;
    a.conv = c->EF.conv;
    a.tri = c->EF.tri;
    a.rp = c->F.rp;
    a.ci = c->F.ci;
    a.diag = c->F.diag;
    a.A0 = c->A0;
    a.M = c->M;
    a.u = u;
    a.mask = c->vel_mask;
    a.g = c->g;
    a.A = c->A;
    a.A32 = c->fp32_A ? c->A32 : nullptr;
    a.dinv = c->dinvA;
    a.dinv32 = c->fp32_A ? c->dinvA32 : nullptr;
    a.b = c->b_mom;
    a.bound = c->prm.momentum_degree >= 2 ? c->mom_bound : nullptr;
    a.rho = c->prm.rho;
    a.sw = sw;
    a.barrier_status = &c->stats->barrier_status;
    return a;
}

}  // namespace

// ---- per-step assembly without colours (single contexts) ------------------------------------
// The convection matrix is a sum of element contributions. Instead of scattering them colour by
// colour behind grid barriers, each element writes its 9 contributions to a buffer and each CSR
// entry then gathers its own (the list of contributions per entry is fixed by the mesh and built
// once, in element order, so the sum is deterministic): three plain launches, no barrier.
namespace {

// ev[9 e + 3 r + q] = dt rho (|T|/12) ((u_sum + u_r) . grad phi_q)  (Eq. 16's N, element e), from
// the pre-scaled gradients: S_q + u_r . (c grad phi_q) with S_q = u_sum . (c grad phi_q)
__global__ void k_conv_elements(int t, const int* __restrict__ tri, const double* __restrict__ conv,
                                const double* __restrict__ u, double* __restrict__ ev,
                                unsigned int* __restrict__ bound) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (bound && e == 0) *bound = 0u;   // k_rows, launched after this kernel, takes the max
    if (e >= t) return;
    const double* g = conv + 6 * (size_t)e;
    double gx[3], gy[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        gx[q] = g[q];
        gy[q] = g[3 + q];
    }
    double ux[3], uy[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) load2(u, tri[3 * e + q], ux[q], uy[q]);
    const double sx = ux[0] + ux[1] + ux[2], sy = uy[0] + uy[1] + uy[2];
    // the gradients of the three P1 basis functions sum to zero, so the third column of the
    // element matrix is minus the sum of the first two (24 FP64 operations per element instead of
    // 28; this GPU issues FP64 at a small fraction of its FP32 rate, and this kernel is bound by it)
    double S[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) S[q] = fma(sy, gy[q], sx * gx[q]);
    double* o = ev + 9 * (size_t)e;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const double o0 = fma(ux[r], gx[0], fma(uy[r], gy[0], S[0]));
        const double o1 = fma(ux[r], gx[1], fma(uy[r], gy[1], S[1]));
        o[r * 3] = o0;
        o[r * 3 + 1] = o1;
        o[r * 3 + 2] = -(o0 + o1);
    }
}

// A[k] = A0[k] + the element contributions of entry k (and its FP32 copy); with `pos`, the same
// value also goes to the entry's slot of the solvers' sliced-ELL copies
__global__ void k_gather_entries(int nnz, const int* __restrict__ ip, const int* __restrict__ idx,
                                 const double* __restrict__ ev, const double* __restrict__ A0, double* __restrict__ A,
                                 float* __restrict__ A32, const int* __restrict__ pos, double* __restrict__ Aell,
                                 float* __restrict__ A32ell) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nnz) return;
    double v = A0[k];
    for (int m = ip[k]; m < ip[k + 1]; ++m) v += ev[idx[m]];
    A[k] = v;
    if (A32) A32[k] = (float)v;
    if (pos) {
        const int p = pos[k];
        Aell[p] = v;
        if (A32ell) A32ell[p] = (float)v;
    }
}

// Jacobi diagonals and the right-hand side b = rho M u^n (Dirichlet rows: prescribed values), with
// `gpn` (incremental forms) b = rho M u^n - dt gpn, gpn = G_f P p_c^n; with `bound`, the largest
// Gershgorin bound 1 + sum_j!=i |A_ij| / |A_ii| of D^-1 A over the rows (from the FP32 copy;
// identity rows for Dirichlet components), as an atomic max of float bits
__global__ void k_rows(int nf, const int* __restrict__ rp, const int* __restrict__ ci, const int* __restrict__ diag,
                       const double* __restrict__ A, const float* __restrict__ A32, const double* __restrict__ M,
                       const double* __restrict__ u, const unsigned char* __restrict__ mask,
                       const double* __restrict__ g, double rho, double* __restrict__ dinv,
                       float* __restrict__ dinv32, double* __restrict__ b, unsigned int* __restrict__ bound,
                       const double* __restrict__ gpn, double dt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float gmax = 1.f;
    if (i < nf) {
        const unsigned char m = mask[i];
        const int kd = diag[i];
        if (dinv) {
            const double di = 1.0 / A[kd];
            const double dx = (m & CGP_BC_U) ? 1.0 : di, dy = (m & CGP_BC_V) ? 1.0 : di;
            store2(dinv, i, dx, dy);
            if (dinv32) store2(dinv32, i, (float)dx, (float)dy);
        } else {
            // FP32 inner iterations only: the FP32 inverse diagonal, without an FP64 division
            const float di = 1.f / (float)A[kd];
            store2(dinv32, i, (m & CGP_BC_U) ? 1.f : di, (m & CGP_BC_V) ? 1.f : di);
        }
        double mx = 0.0, my = 0.0;
        float off = 0.f;
        for (int k = rp[i]; k < rp[i + 1]; ++k) {
            double ujx, ujy;
            load2(u, ci[k], ujx, ujy);
            mx += M[k] * ujx;
            my += M[k] * ujy;
            if (bound && k != kd) off += fabsf(A32[k]);
        }
        double gx, gy, bx = rho * mx, by = rho * my;
        if (gpn) {
            double px, py;
            load2(gpn, i, px, py);
            bx -= dt * px;
            by -= dt * py;
        }
        load2(g, i, gx, gy);
        store2(b, i, (m & CGP_BC_U) ? gx : bx, (m & CGP_BC_V) ? gy : by);
        if (bound && (m & (CGP_BC_U | CGP_BC_V)) != (CGP_BC_U | CGP_BC_V))
            gmax = 1.f + off / fabsf(A32[kd]);
    }
    if (bound) {
        const unsigned int gb = __reduce_max_sync(0xffffffffu, __float_as_uint(gmax));
        if ((threadIdx.x & 31) == 0) atomicMax(bound, gb);
    }
}

}  // namespace

// Entry -> contribution lists of the fine pattern (host, once per context).
int assemble_gather_build(cgp_ctx_s* c) {
    const HostElems& h = c->hm.ef;
    const int nnz = c->F.nnz;
    const size_t nc = h.slot.size();   // 9 per element
    std::vector<int> ip(nnz + 1, 0), idx(nc);
    for (size_t m = 0; m < nc; ++m) ip[h.slot[m] + 1] += 1;
    for (int k = 0; k < nnz; ++k) ip[k + 1] += ip[k];
    std::vector<int> pos(ip.begin(), ip.end() - 1);
    for (size_t m = 0; m < nc; ++m) idx[pos[h.slot[m]]++] = (int)m;   // element order within an entry
    void *d_ip = nullptr, *d_idx = nullptr, *d_ev = nullptr;
    if (cudaMalloc(&d_ip, sizeof(int) * ip.size()) != cudaSuccess) return CGP_ERR_NOMEM;
    c->allocs.push_back(d_ip);
    if (cudaMalloc(&d_idx, sizeof(int) * idx.size()) != cudaSuccess) return CGP_ERR_NOMEM;
    c->allocs.push_back(d_idx);
    if (cudaMalloc(&d_ev, sizeof(double) * nc) != cudaSuccess) return CGP_ERR_NOMEM;
    c->allocs.push_back(d_ev);
    if (cudaMemcpy(d_ip, ip.data(), sizeof(int) * ip.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_idx, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return CGP_ERR_CUDA;
    c->asm_ip = (int*)d_ip;
    c->asm_idx = (int*)d_idx;
    c->asm_ev = (double*)d_ev;
    return CGP_OK;
}

cudaError_t launch_assemble_step(cgp_ctx_s* c, const double* u, cudaStream_t s, const double* gpn) {
    const int t = c->EF.t, nnz = c->F.nnz, nf = c->nf;
    unsigned int* bound = c->prm.momentum_degree >= 2 ? c->mom_bound : nullptr;
    k_conv_elements<<<(t + 255) / 256, 256, 0, s>>>(t, c->EF.tri, c->EF.conv, u, c->asm_ev, bound);
    k_gather_entries<<<(nnz + 255) / 256, 256, 0, s>>>(nnz, c->asm_ip, c->asm_idx, c->asm_ev, c->A0, c->A,
                                                      c->fp32_A ? c->A32 : nullptr, c->ell_on ? c->ell_pos : nullptr,
                                                      c->ell_A, c->fp32_A ? c->ell_A32 : nullptr);
    // with FP32 inner iterations nothing reads the FP64 inverse diagonal
    double* dinv64 = c->prm.precision == CGP_MIXED ? nullptr : c->dinvA;
    k_rows<<<(nf + 255) / 256, 256, 0, s>>>(nf, c->F.rp, c->F.ci, c->F.diag, c->A, c->A32, c->M, u, c->vel_mask,
                                          c->g, c->prm.rho, dinv64, c->fp32_A ? c->dinvA32 : nullptr, c->b_mom,
                                          bound, gpn, c->prm.dt);
    return cudaGetLastError();
}

// The colour-scheduled persistent assembly, one cooperative launch (the batched step's form).
cudaError_t launch_assemble_step_coloured(cgp_ctx_s* c, const double* u, cudaStream_t s) {
    Launch<StepAsmArgs> L;
    L.single = asm_args(c, u, c->sync + SYNC_ASM);
    L.table = nullptr;
    L.map = {nullptr, nullptr, nullptr};
    cudaError_t e = cudaMemsetAsync(L.single.sw, 0, sizeof(SyncWords), s);
    if (e != cudaSuccess) return e;
    return coop_launch(k_assemble_step, c->sh_f.blocks, c->sh_f.threads, L, s);
}

cudaError_t batch_asm_build(cgp_batch_s* b) {
    std::vector<StepAsmArgs> tab(b->n);
    for (int i = 0; i < b->n; ++i) tab[i] = asm_args(b->ctx[i], batch_u_work(b, i), b->sync + (size_t)i * SYNC_COUNT + SYNC_ASM);
    void* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(StepAsmArgs) * tab.size());
    if (e != cudaSuccess) return e;
    b->allocs.push_back(d);
    b->tab_asm = d;
    return cudaMemcpy(d, tab.data(), sizeof(StepAsmArgs) * tab.size(), cudaMemcpyHostToDevice);
}

cudaError_t batch_asm_launch(cgp_batch_s* b, cudaStream_t s) {
    Launch<StepAsmArgs> L;
    L.single = StepAsmArgs();
    L.table = (const StepAsmArgs*)b->tab_asm;
    L.map = b->map_f;
    return coop_launch(k_assemble_step, b->blocks_f, b->threads, L, s);
}

}  // namespace cgp
