// Persistent Krylov solvers of the CGP step: one cooperative launch per solve.
//
// Every solve is an FP64 iterative-refinement loop around an inner Krylov method in type TI:
//   repeat:  r = b - A x  (FP64);  stop if ||r|| <= rtol ||b||  (per right-hand side)
//            solve A d = r approximately in TI from d = 0;  x += d  (FP64)
// With TI = double (CGP_FP64) one pass normally suffices and the FP64 true residual is the
// final check; with TI = float (CGP_MIXED) the inner solve runs in FP32 with FP32 accumulation
// and the FP64 passes recover full accuracy.
//
// Inner methods, both Jacobi (diagonal) preconditioned:
//  * CG in the Chronopoulos-Gear form (one grid reduction per iteration), for the SPD coarse
//    Poisson matrix (Eq. 21) and the consistent mass matrix of the correction (Eq. 23);
//  * BiCGStab (van der Vorst 1992) for the non-symmetric momentum matrix (Eq. 19), two
//    right-hand sides (the velocity components) at once, Dirichlet rows applied as identity rows
//    per component inside the operator.
// Replaces the paper's ILU(0)-GMRES(m) (Sect. 2.3), whose triangular solves are sequential.
//
// Rows are split into one contiguous slice per block. Grid-wide reductions are deterministic:
// each block writes its partial sums, and after a bounded grid barrier every block adds all
// partials in the same order, so all blocks take identical branch decisions.
#include <algorithm>
#include <mutex>

#include "ctx.h"
#include "krylov_kernels.cuh"

namespace cgp {


namespace {

// ---- argument builders, shared by the single-instance launchers and the batched stages -------
template <typename TI>
CgArgs<TI> poisson_args(cgp_ctx_s* c, const double* b, double* x, SyncWords* sw, double* part) {
    const bool mixed = sizeof(TI) == sizeof(float);
    const int n = c->nc;
    char* p = (char*)c->ws;
    CgArgs<TI> a;
    a.n = n;
    a.rp = c->C.rp;
    a.ci = c->C.ci;
    a.val64 = c->Kc;
    a.valI = mixed ? (const TI*)(const void*)c->Kc32 : (const TI*)(const void*)c->Kc;
    a.dinvI = mixed ? (const TI*)(const void*)c->dinvK32 : (const TI*)(const void*)c->dinvK;
    a.b = b;
    a.x = x;
    a.r = carve<TI>(p, n); a.u = carve<TI>(p, n); a.w = carve<TI>(p, n);
    a.p = carve<TI>(p, n); a.s = carve<TI>(p, n); a.d = carve<TI>(p, n);
    a.part = part;
    a.sw = sw;
    a.rtol = c->prm.rtol;
    a.inner_rtol = mixed ? c->prm.inner_rtol : 0.0;
    a.max_iter = c->prm.max_iter;
    a.max_outer = c->prm.max_outer;
    a.lanes = c->sh_c.lanes;
    a.st_iters = &c->stats->poi_iters; a.st_outer = &c->stats->poi_outer; a.st_status = &c->stats->poi_status;
    a.st_rel = &c->stats->poi_rel; a.st_barrier = &c->stats->barrier_status;
    return a;
}

template <typename TI>
CgArgs<TI> mass_args(cgp_ctx_s* c, const double* b, double* x, SyncWords* sw, double* part, bool ell) {
    const bool mixed = sizeof(TI) == sizeof(float);
    const size_t n2 = 2 * (size_t)c->nf;
    char* p = (char*)c->ws;
    CgArgs<TI> a;
    a.n = c->nf; a.rp = c->F.rp; a.ci = c->F.ci; a.val64 = c->M;
    a.valI = mixed ? (const TI*)(const void*)c->M32 : (const TI*)(const void*)c->M;
    a.dinvI = mixed ? (const TI*)(const void*)c->dinvM32 : (const TI*)(const void*)c->dinvM;
    a.b = b; a.x = x;
    a.r = carve<TI>(p, n2); a.u = carve<TI>(p, n2); a.w = carve<TI>(p, n2);
    a.p = carve<TI>(p, n2); a.s = carve<TI>(p, n2); a.d = carve<TI>(p, n2);
    a.part = part; a.sw = sw; a.rtol = c->prm.rtol; a.inner_rtol = mixed ? c->prm.inner_rtol : 0.0;
    a.max_iter = c->prm.max_iter; a.max_outer = c->prm.max_outer; a.lanes = c->sh_f.lanes;
    a.st_iters = &c->stats->mass_iters; a.st_outer = &c->stats->mass_outer; a.st_status = &c->stats->mass_status;
    a.st_rel = &c->stats->mass_rel; a.st_barrier = &c->stats->barrier_status;
    // Chebyshev preconditioner: for P1 triangles every element matrix D_e^-1 M_e has the
    // eigenvalues 1/2, 1/2, 2, so the spectrum of D^-1 M lies in [1/2, 2] on any mesh
    a.pdeg = c->prm.mass_degree;
    if (a.pdeg >= 2) {
        a.plmin = 0.5;
        a.plmax = 2.0;
        a.valP = c->M32;
        a.dinvP = c->dinvM32;
        a.zc0 = carve<float>(p, n2); a.zc1 = carve<float>(p, n2); a.dc = carve<float>(p, n2);
    }
    if (ell) {
        a.eptr = c->ell_ptr;
        a.ecol = c->ell_col;
        a.eval64 = c->ell_M;
        a.evalI = mixed ? (const TI*)(const void*)c->ell_M32 : (const TI*)(const void*)c->ell_M;
        a.evalP = c->ell_M32;
    }
    return a;
}

template <typename TI>
BicgArgs<TI> momentum_args(cgp_ctx_s* c, const double* u_in, double* x, SyncWords* sw, double* part, bool ell) {
    const bool mixed = sizeof(TI) == sizeof(float);
    const size_t n2 = 2 * (size_t)c->nf;
    char* p = (char*)c->ws;
    BicgArgs<TI> a;
    a.n = c->nf; a.rp = c->F.rp; a.ci = c->F.ci; a.val64 = c->A;
    a.valI = mixed ? (const TI*)(const void*)c->A32 : (const TI*)(const void*)c->A;
    a.dinvI = mixed ? (const TI*)(const void*)c->dinvA32 : (const TI*)(const void*)c->dinvA;
    a.mask = c->vel_mask; a.diag = c->F.diag; a.g = c->g; a.b = c->b_mom; a.x_in = u_in; a.x = x;
    const bool pred = c->prm.warm_start >= 1;
    a.dx = pred ? c->mom_dx : nullptr;
    a.dx_flag = pred ? c->mom_flag : nullptr;
    a.dx2 = c->prm.warm_start >= 3 ? c->mom_dx2 : nullptr;
    a.pdeg = c->prm.momentum_degree;
    a.r = carve<TI>(p, n2); a.rh = carve<TI>(p, n2); a.p = carve<TI>(p, n2);
    a.v = carve<TI>(p, n2); a.y = carve<TI>(p, n2); a.s = carve<TI>(p, n2);
    a.z = carve<TI>(p, n2); a.t = carve<TI>(p, n2); a.d = carve<TI>(p, n2);
    a.part = part; a.sw = sw; a.rtol = c->prm.momentum_rtol; a.inner_rtol = mixed ? c->prm.inner_rtol : 0.0;
    a.max_iter = c->prm.max_iter; a.max_outer = c->prm.max_outer; a.lanes = c->sh_f.lanes;
    a.st_iters = &c->stats->mom_iters; a.st_outer = &c->stats->mom_outer; a.st_status = &c->stats->mom_status;
    a.st_rel = &c->stats->mom_rel; a.st_barrier = &c->stats->barrier_status;
    if (a.pdeg >= 2) {
        // the real parts of the spectrum of D^-1 A lie near [1/2, 2] while the mass matrix
        // dominates; the upper end is the assembly's Gershgorin bound, and an underestimated lower
        // end only leaves those components to the Krylov iteration
        a.plmin = 0.5;
        a.pbound = c->mom_bound;
        a.valP = c->A32;
        a.dinvP = c->dinvA32;
        a.zc0 = carve<float>(p, n2); a.zc1 = carve<float>(p, n2); a.dc = carve<float>(p, n2);
    }
    if (ell) {
        a.eptr = c->ell_ptr;
        a.ecol = c->ell_col;
        a.eval64 = c->ell_A;
        a.evalI = mixed ? (const TI*)(const void*)c->ell_A32 : (const TI*)(const void*)c->ell_A;
        a.evalP = c->ell_A32;
    }
    return a;
}

template <typename Args>
Launch<Args> single_launch(const Args& a) {
    Launch<Args> L;
    L.single = a;
    L.table = nullptr;
    L.map = {nullptr, nullptr, nullptr};
    return L;
}

}  // namespace

cudaError_t launch_poisson_cg(cgp_ctx_s* c, const double* b, double* x, cudaStream_t s) {
    if (c->use_pipe) return launch_poisson_pipe(c, b, x, s);
    SyncWords* sw = c->sync + SYNC_POI;
    cudaError_t e = cudaMemsetAsync(sw, 0, sizeof(SyncWords), s);
    if (e != cudaSuccess) return e;
    if (c->prm.precision == CGP_MIXED) {
        auto L = single_launch(poisson_args<float>(c, b, x, sw, c->part));
        return coop_launch(k_cg<float, 1>, c->sh_c.blocks, c->sh_c.threads, L, s, cg_smem<1>(c->sh_c.threads));
    }
    auto L = single_launch(poisson_args<double>(c, b, x, sw, c->part));
    return coop_launch(k_cg<double, 1>, c->sh_c.blocks, c->sh_c.threads, L, s, cg_smem<1>(c->sh_c.threads));
}

cudaError_t launch_mass_cg(cgp_ctx_s* c, const double* b, double* x, cudaStream_t s) {
    SyncWords* sw = c->sync + SYNC_MASS;
    cudaError_t e = cudaMemsetAsync(sw, 0, sizeof(SyncWords), s);
    if (e != cudaSuccess) return e;
    const int B = c->sh_f.blocks, T = c->sh_f.threads;
    if (c->prm.precision == CGP_MIXED) {
        auto L = single_launch(mass_args<float>(c, b, x, sw, c->part, c->ell_on));
        if (c->ell_on) return coop_launch(k_cg<float, 2, 1, true>, B, T, L, s, cg_smem<2>(T));
        return coop_launch(k_cg<float, 2>, B, T, L, s, cg_smem<2>(T));
    }
    auto L = single_launch(mass_args<double>(c, b, x, sw, c->part, c->ell_on));
    if (c->ell_on) return coop_launch(k_cg<double, 2, 1, true>, B, T, L, s, cg_smem<2>(T));
    return coop_launch(k_cg<double, 2>, B, T, L, s, cg_smem<2>(T));
}

cudaError_t launch_momentum_bicgstab(cgp_ctx_s* c, const double* u_in, double* x, cudaStream_t s) {
    SyncWords* sw = c->sync + SYNC_MOM;
    cudaError_t e = cudaMemsetAsync(sw, 0, sizeof(SyncWords), s);
    if (e != cudaSuccess) return e;
    const int B = c->sh_f.blocks, T = c->sh_f.threads;
    if (c->prm.precision == CGP_MIXED) {
        auto L = single_launch(momentum_args<float>(c, u_in, x, sw, c->part, c->ell_on));
        if (c->ell_on) return coop_launch(k_bicgstab<float, 1, true>, B, T, L, s, bicg_smem(T));
        return coop_launch(k_bicgstab<float>, B, T, L, s, bicg_smem(T));
    }
    auto L = single_launch(momentum_args<double>(c, u_in, x, sw, c->part, c->ell_on));
    if (c->ell_on) return coop_launch(k_bicgstab<double, 1, true>, B, T, L, s, bicg_smem(T));
    return coop_launch(k_bicgstab<double>, B, T, L, s, bicg_smem(T));
}

cudaError_t launch_solver_spmv(cgp_ctx_s* c, const float* x, float* y, cudaStream_t s) {
    const int B = c->sh_f.blocks, T = c->sh_f.threads;
    if (c->ell_on)
        k_solver_spmv<true><<<B, T, 0, s>>>(c->nf, c->F.rp, c->F.ci, c->A32, c->ell_ptr, c->ell_col, c->ell_A32, x, y,
                                            c->sh_f.lanes);
    else
        k_solver_spmv<false><<<B, T, 0, s>>>(c->nf, c->F.rp, c->F.ci, c->A32, c->ell_ptr, c->ell_col, c->ell_A32, x,
                                             y, c->sh_f.lanes);
    return cudaGetLastError();
}

// ---- batched solver stages: one cooperative launch per stage for all instances ----------------
namespace {

template <typename Args>
cudaError_t upload_table(cgp_batch_s* b, const std::vector<Args>& tab, void** out) {
    void* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(Args) * tab.size());
    if (e != cudaSuccess) return e;
    b->allocs.push_back(d);
    *out = d;
    return cudaMemcpy(d, tab.data(), sizeof(Args) * tab.size(), cudaMemcpyHostToDevice);
}

SyncWords* bsync(cgp_batch_s* b, int i, int slot) { return b->sync + (size_t)i * SYNC_COUNT + slot; }
double* bpart(cgp_batch_s* b, int i) { return b->part + (size_t)i * 32 * b->max_group; }

template <typename TI>
cudaError_t build_typed(cgp_batch_s* b) {
    std::vector<BicgArgs<TI>> mom(b->n);
    std::vector<CgArgs<TI>> poi(b->n);
    std::vector<CgArgs<TI>> mass(b->n);
    for (int i = 0; i < b->n; ++i) {
        cgp_ctx_s* c = b->ctx[i];
        mom[i] = momentum_args<TI>(c, batch_u_work(b, i), c->ut, bsync(b, i, SYNC_MOM), bpart(b, i), false);
        poi[i] = poisson_args<TI>(c, c->bc, b->pc[i], bsync(b, i, SYNC_POI), bpart(b, i));
        mass[i] = mass_args<TI>(c, c->grad, c->w, bsync(b, i, SYNC_MASS), bpart(b, i), false);
    }
    cudaError_t e = upload_table(b, mom, &b->tab_mom);
    if (e == cudaSuccess) e = upload_table(b, poi, &b->tab_poi);
    if (e == cudaSuccess) e = upload_table(b, mass, &b->tab_mass);
    return e;
}

template <typename Args>
Launch<Args> table_launch(const void* tab, const BatchMap& m) {
    Launch<Args> L;
    L.single = Args();
    L.table = (const Args*)tab;
    L.map = m;
    return L;
}

}  // namespace

cudaError_t batch_solvers_build(cgp_batch_s* b) {
    return b->precision == CGP_MIXED ? build_typed<float>(b) : build_typed<double>(b);
}

cudaError_t batch_momentum_launch(cgp_batch_s* b, cudaStream_t s) {
    if (b->precision == CGP_MIXED) {
        auto L = table_launch<BicgArgs<float>>(b->tab_mom, b->map_f);
        return coop_launch(k_bicgstab<float, 2>, b->blocks_f, b->threads, L, s, bicg_smem(b->threads));
    }
    auto L = table_launch<BicgArgs<double>>(b->tab_mom, b->map_f);
    return coop_launch(k_bicgstab<double, 2>, b->blocks_f, b->threads, L, s, bicg_smem(b->threads));
}

cudaError_t batch_poisson_launch(cgp_batch_s* b, cudaStream_t s) {
    if (b->precision == CGP_MIXED) {
        auto L = table_launch<CgArgs<float>>(b->tab_poi, b->map_c);
        return coop_launch(k_cg<float, 1, 2>, b->blocks_c, b->threads, L, s, cg_smem<1>(b->threads));
    }
    auto L = table_launch<CgArgs<double>>(b->tab_poi, b->map_c);
    return coop_launch(k_cg<double, 1, 2>, b->blocks_c, b->threads, L, s, cg_smem<1>(b->threads));
}

cudaError_t batch_mass_launch(cgp_batch_s* b, cudaStream_t s) {
    if (b->precision == CGP_MIXED) {
        auto L = table_launch<CgArgs<float>>(b->tab_mass, b->map_f);
        return coop_launch(k_cg<float, 2, 2>, b->blocks_f, b->threads, L, s, cg_smem<2>(b->threads));
    }
    auto L = table_launch<CgArgs<double>>(b->tab_mass, b->map_f);
    return coop_launch(k_cg<double, 2, 2>, b->blocks_f, b->threads, L, s, cg_smem<2>(b->threads));
}

// Occupancy of the persistent kernels (blocks per SM at `threads`), the minimum over the family.
// Resident blocks per SM of the generic persistent kernels at `threads` threads (the minimum over
// all of them, with their dynamic shared memory) for single contexts (batch = false) or for the
// batch instantiations; also raises their dynamic shared-memory limit.
int persistent_blocks_per_sm(int threads, bool batch) {
    int m = 1 << 30, v = 0;
    const void* single[] = {(const void*)k_cg<double, 1>, (const void*)k_cg<float, 1>, (const void*)k_cg<double, 2>,
                            (const void*)k_cg<float, 2>, (const void*)k_bicgstab<double>,
                            (const void*)k_bicgstab<float>, (const void*)k_cg<double, 2, 1, true>,
                            (const void*)k_cg<float, 2, 1, true>, (const void*)k_bicgstab<double, 1, true>,
                            (const void*)k_bicgstab<float, 1, true>};
    const void* batched[] = {(const void*)k_cg<double, 1, 2>, (const void*)k_cg<float, 1, 2>,
                             (const void*)k_cg<double, 2, 2>, (const void*)k_cg<float, 2, 2>,
                             (const void*)k_bicgstab<double, 2>, (const void*)k_bicgstab<float, 2>};
    const size_t smem[] = {cg_smem<1>(threads), cg_smem<1>(threads), cg_smem<2>(threads),
                           cg_smem<2>(threads), bicg_smem(threads), bicg_smem(threads),
                           cg_smem<2>(threads), cg_smem<2>(threads), bicg_smem(threads), bicg_smem(threads)};
    const void* const* fns = batch ? batched : single;
    for (int k = 0; k < (batch ? 6 : 10); ++k) {
        if (cudaFuncSetAttribute(fns[k], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem[k]) != cudaSuccess)
            return 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, fns[k], threads, smem[k]) != cudaSuccess) return 0;
        m = v < m ? v : m;
    }
    return m;
}

namespace {

__global__ void k_sell_fill(int total, const int* __restrict__ src, const double* __restrict__ csr_val, double* sell_val) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < total) sell_val[p] = src[p] >= 0 ? csr_val[src[p]] : 0.0;
}

// Sliced-ELL SpMV, two interleaved right-hand sides: one warp per 32-row slice, slot k of all 32
// rows contiguous, so every value and column load of a warp is one coalesced 128/256-byte access.
// Slots are taken four at a time, all column and value loads of a group issued before its x
// gathers; the matrix is streamed with the evict-first hint and y written the same way, so the
// gathered x keeps its place in L2.
__global__ void __launch_bounds__(256) k_spmv_sell2(int nslices, const int* __restrict__ ptr, const int* __restrict__ col,
                                                    const double* __restrict__ val, const int* __restrict__ perm,
                                                    const double* __restrict__ x, double* __restrict__ y) {
    const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (s >= nslices) return;
    const int base = ptr[s], w = (ptr[s + 1] - base) >> 5;
    const double2* x2 = reinterpret_cast<const double2*>(x);
    double a0 = 0.0, a1 = 0.0;
    int k = 0;
    for (; k + 4 <= w; k += 4) {
        int j[4];
        double v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int p = base + ((k + q) << 5) + lane;
            j[q] = __ldcs(col + p);
            v[q] = __ldcs(val + p);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const double2 xv = __ldg(x2 + j[q]);
            a0 += v[q] * xv.x;
            a1 += v[q] * xv.y;
        }
    }
    for (; k < w; ++k) {
        const int p = base + (k << 5) + lane;
        const double2 xv = __ldg(x2 + __ldcs(col + p));
        const double v = __ldcs(val + p);
        a0 += v * xv.x;
        a1 += v * xv.y;
    }
    const int r = perm[(s << 5) + lane];
    if (r >= 0) __stcs(reinterpret_cast<double2*>(y) + r, make_double2(a0, a1));
}

}  // namespace

namespace {
__global__ void k_ell_fill(int total, const int* __restrict__ src, const double* __restrict__ csr_val, double* val,
                           float* val32) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= total) return;
    const double v = src[p] >= 0 ? csr_val[src[p]] : 0.0;
    val[p] = v;
    if (val32) val32[p] = (float)v;
}
}  // namespace

// Copy CSR values into sliced-ELL slot order (padding slots get 0), with an FP32 copy if asked.
cudaError_t ell_fill(int total, const int* src, const double* csr_val, double* val, float* val32, cudaStream_t s) {
    if (total <= 0) return cudaSuccess;
    k_ell_fill<<<(total + 255) / 256, 256, 0, s>>>(total, src, csr_val, val, val32);
    return cudaGetLastError();
}

cudaError_t sell_fill(cgp_ctx_s* c, const double* csr_val, cudaStream_t s) {
    k_sell_fill<<<(c->sell_total + 255) / 256, 256, 0, s>>>(c->sell_total, c->sell_src, csr_val, c->sell_val);
    return cudaGetLastError();
}

cudaError_t launch_spmv_sell(cgp_ctx_s* c, const double* x, double* y, cudaStream_t s) {
    const int threads = 256;
    const int blocks = (int)(((long long)c->sell_nslices * 32 + threads - 1) / threads);
    k_spmv_sell2<<<blocks, threads, 0, s>>>(c->sell_nslices, c->sell_ptr, c->sell_col, c->sell_val, c->sell_perm, x, y);
    return cudaGetLastError();
}

// y = A0 x on the fine mesh for two interleaved right-hand sides (A0 = rho M + dt mu K), x and y
// in the stored fine order: the sliced-ELL kernel when the autotuner chose it, else one row group
// of sh_f.lanes lanes per row.
cudaError_t launch_spmv_fine(cgp_ctx_s* c, const double* x, double* y, cudaStream_t s) {
    if (c->spmv_sell) return launch_spmv_sell(c, x, y, s);
    const int n = c->nf, threads = 256, lanes = c->sh_f.lanes;
    const int rows_per_block = threads / lanes;
    const int blocks = (n + rows_per_block - 1) / rows_per_block;
    k_spmv_probe<2><<<blocks, threads, 0, s>>>(n, c->F.rp, c->F.ci, c->A0, x, y, lanes, rows_per_block);
    return cudaGetLastError();
}

cudaError_t time_spmv_lanes(cgp_ctx_s* c, bool fine, int lanes, cudaStream_t s, float* ms) {
    const int n = fine ? c->nf : c->nc;
    const int threads = 256;
    const int rows_per_block = threads / lanes;
    const int blocks = (n + rows_per_block - 1) / rows_per_block;
    double* x = (double*)c->ws;
    double* y = x + 2 * (size_t)c->nf + 64;
    cudaError_t e = cudaMemsetAsync(x, 0, 2 * sizeof(double) * (size_t)c->nf, s);
    if (e != cudaSuccess) return e;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int reps = 20;
    for (int w = 0; w < 3; ++w) {
        if (fine) k_spmv_probe<2><<<blocks, threads, 0, s>>>(n, c->F.rp, c->F.ci, c->A0, x, y, lanes, rows_per_block);
        else k_spmv_probe<1><<<blocks, threads, 0, s>>>(n, c->C.rp, c->C.ci, c->Kc_raw, x, y, lanes, rows_per_block);
    }
    cudaEventRecord(e0, s);
    for (int w = 0; w < reps; ++w) {
        if (fine) k_spmv_probe<2><<<blocks, threads, 0, s>>>(n, c->F.rp, c->F.ci, c->A0, x, y, lanes, rows_per_block);
        else k_spmv_probe<1><<<blocks, threads, 0, s>>>(n, c->C.rp, c->C.ci, c->Kc_raw, x, y, lanes, rows_per_block);
    }
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    *ms = t / reps;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Allocation-free variant of the classical CG kernel (cgp_cg_solve_noalloc)
// ------------------------------------------------------------------------------------------
namespace {

constexpr int NOALLOC_MAX_ROWS = 65536;
constexpr size_t NOALLOC_VEC_BYTES = (size_t)NOALLOC_MAX_ROWS * sizeof(double);
constexpr size_t NOALLOC_PART_BYTES = 32 * (size_t)CGP_MAX_GRID * sizeof(double);
constexpr size_t NOALLOC_BYTES = 7 * NOALLOC_VEC_BYTES + NOALLOC_PART_BYTES + 512;
// FP64 refinement passes of one allocation-free solve (each ends with an FP64 true residual)
constexpr int NOALLOC_MAX_OUTER = 30;

// All scratch of cgp_cg_solve_noalloc: seven vectors of NOALLOC_MAX_ROWS doubles (r, u, w, p,
// s, d and the inverse diagonal), the per-block partial sums, the grid-barrier words and a
// statistics record. About 3.6 MB, held by every device that loads the library until exit.
__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

struct NoallocStats {
    int iters, outer, status, barrier;
    double rel;
    int arg;   // CGP_ERR_ARG when a row has no positive finite stored diagonal
};

struct NoallocDevice {
    bool ready = false;
    unsigned char* base = nullptr;   // device address of g_noalloc_scratch on this device
    int num_sms = 0;
};
std::mutex g_noalloc_mu;
NoallocDevice g_noalloc_dev[64];

// Jacobi inverse diagonal. A row without a positive finite stored diagonal cannot belong to an
// SPD matrix: it gets 0 (so the solve stays finite) and the call's status becomes CGP_ERR_ARG.
__global__ void k_noalloc_dinv(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                               const double* __restrict__ val, double* dinv, NoallocStats* st) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double d = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k)
        if (ci[k] == i) d = val[k];
    if (d > 0.0 && d <= 1.7976931348623157e308) {
        dinv[i] = 1.0 / d;
    } else {
        dinv[i] = 0.0;
        st->arg = CGP_ERR_ARG;
    }
}

// Folds the solve's statistics into the caller's outputs: an argument error first, then a grid
// barrier that gave up (the solver's own status and residual are then meaningless: the residual
// reads NaN and the iteration count is what the solver had recorded, 0 if nothing), then the
// solver's status.
__global__ void k_noalloc_finish(const NoallocStats* st, int* status, int* iters, double* rel) {
    const int s = st->arg != 0 ? st->arg : (st->barrier != 0 ? st->barrier : st->status);
    if (status) *status = s;
    if (iters) *iters = st->iters;
    if (rel) *rel = st->barrier != 0 ? __longlong_as_double(0x7ff8000000000000ll) : st->rel;
}

}  // namespace

}  // namespace cgp

extern "C" int cgp_cg_solve_noalloc(int n, const int* rp_dev, const int* ci_dev, const double* val_dev,
                                    const double* b_dev, double* x_dev, double rtol, int max_iter,
                                    int* status_dev, int* iters_dev, double* rel_res_dev, void* stream) {
    using namespace cgp;
    if (n <= 0 || n > NOALLOC_MAX_ROWS) return CGP_ERR_ARG;
    if (!rp_dev || !ci_dev || !val_dev || !b_dev || !x_dev || !(rtol > 0.0) || max_iter <= 0) return CGP_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CGP_ERR_CUDA;
    if (dev < 0 || dev >= 64) return CGP_ERR_ARG;
    NoallocDevice* nd = &g_noalloc_dev[dev];
    {
        // once per device, with that device current: the device address of the scratch array
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!nd->ready) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return CGP_ERR_CUDA;
            int sms = 0, occ = 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CGP_ERR_CUDA;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)k_cg<double, 1>, 512, cg_smem<1>(512)) !=
                    cudaSuccess || occ < 1)
                return CGP_ERR_CUDA;
            nd->base = (unsigned char*)p;
            nd->num_sms = sms;
            nd->ready = true;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* base = nd->base;
    double* vec[7];
    for (int k = 0; k < 7; ++k) vec[k] = (double*)(base + k * NOALLOC_VEC_BYTES);
    double* part = (double*)(base + 7 * NOALLOC_VEC_BYTES);
    SyncWords* sw = (SyncWords*)(base + 7 * NOALLOC_VEC_BYTES + NOALLOC_PART_BYTES);
    NoallocStats* st = (NoallocStats*)(base + 7 * NOALLOC_VEC_BYTES + NOALLOC_PART_BYTES + 256);
    // the scratch keeps the previous call's contents: clear the barrier words and statistics
    if (cudaMemsetAsync(sw, 0, 512, s) != cudaSuccess) return CGP_ERR_CUDA;
    k_noalloc_dinv<<<(n + 255) / 256, 256, 0, s>>>(n, rp_dev, ci_dev, val_dev, vec[6], st);
    if (cudaGetLastError() != cudaSuccess) return CGP_ERR_CUDA;
    CgArgs<double> a;
    a.n = n;
    a.rp = rp_dev;
    a.ci = ci_dev;
    a.val64 = val_dev;
    a.valI = val_dev;
    a.dinvI = vec[6];
    a.b = b_dev;
    a.x = x_dev;
    a.r = vec[0];
    a.u = vec[1];
    a.w = vec[2];
    a.p = vec[3];
    a.s = vec[4];
    a.d = vec[5];
    a.part = part;
    a.sw = sw;
    a.rtol = rtol;
    a.inner_rtol = 0.0;
    a.max_iter = max_iter;
    a.max_outer = NOALLOC_MAX_OUTER;
    a.lanes = 4;
    // every statistic goes to the scratch record first, the barrier status in its own word, so a
    // barrier failure recorded by one block is never overwritten by another block's final status
    a.st_iters = &st->iters;
    a.st_outer = &st->outer;
    a.st_status = &st->status;
    a.st_rel = &st->rel;
    a.st_barrier = &st->barrier;
    const int threads = 512;
    int blocks = (n + threads - 1) / threads;
    blocks = std::max(1, std::min(std::min(blocks, nd->num_sms), CGP_MAX_GRID));
    auto La = single_launch(a);
    cudaError_t e = coop_launch(k_cg<double, 1>, blocks, threads, La, s, cg_smem<1>(threads));
    if (e != cudaSuccess) return CGP_ERR_CUDA;
    k_noalloc_finish<<<1, 1, 0, s>>>(st, status_dev, iters_dev, rel_res_dev);
    e = cudaGetLastError();
    return e == cudaSuccess ? CGP_OK : CGP_ERR_CUDA;
}
