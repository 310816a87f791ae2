// Coarse pressure Poisson solve (Eq. 21) as one persistent kernel with on-chip state.
//
// Layout: one block per SM, one thread per matrix row. Each block copies its row slice of the
// coarse matrix into shared memory once per launch as column-major ELL (slot k of all rows is
// contiguous, so a warp reads 32 consecutive words), and every CG vector of a row lives in the
// registers of the thread that owns it. Per iteration the only global traffic is the published
// preconditioned direction m (written by its owner, gathered by neighbours through L2).
//
// Method: Jacobi-preconditioned pipelined CG (Ghysels & Vanroose, "Hiding global synchronization
// latency in the preconditioned Conjugate Gradient algorithm", Parallel Computing 2014): the two
// inner products of an iteration are reduced while the matrix-vector product n = A m runs, so an
// iteration needs a single grid barrier. Published vectors and partial sums are double buffered
// by iteration parity, which is what makes one barrier per iteration race-free. Pipelined CG has a
// larger gap between recursive and true residual than classical CG; the FP64 refinement loop
// around it (true residual r = b - A x, inner solve of A d = r, x += d) removes that gap.
#include <algorithm>

#include "ctx.h"

namespace cgp {

#define PIPE_WMAX 12
#define PIPE_STAGNATION 2000

namespace {

template <typename TI>
struct PipeArgs {
    int n, rows_per_block, width;
    const int* rp;
    const int* ci;
    const double* val64;
    const TI* valI;
    const double* dinv64;
    const TI* dinvI;
    const double* b;
    double* x;
    TI* mbuf;      // [2][n] published m = D^-1 w (double buffered)
    TI* ubuf;      // [n] published u at the start of a refinement pass
    double* part;  // partial sums
    SyncWords* sw;
    double rtol, inner_rtol;
    int max_iter, max_outer;
    int* st_iters;
    int* st_outer;
    int* st_status;
    double* st_rel;
    int* st_barrier;
};

enum { PP_P0 = 0, PP_O1 = 1, PP_I = 2 /* two buffers of 3 */ };

__device__ __forceinline__ bool bad(double v) { return !(fabs(v) <= 1.7976931348623157e308); }

// sum_k val[k] * src[col[k]] over the ELL row of this thread: all column indices are read from
// shared memory first, then all gathers are issued before the first multiply, so one row costs
// one L2 round trip rather than one per entry.
template <typename TI, typename TS>
__device__ __forceinline__ TI ell_row(const int* s_ci, const TI* s_val, int T, int t, int width, const TS* src) {
    int col[PIPE_WMAX];
    TS g[PIPE_WMAX];
#pragma unroll
    for (int k = 0; k < PIPE_WMAX; ++k) col[k] = k < width ? s_ci[k * T + t] : -1;
#pragma unroll
    for (int k = 0; k < PIPE_WMAX; ++k) g[k] = col[k] >= 0 ? src[col[k]] : (TS)0;
    TI acc = (TI)0;
#pragma unroll
    for (int k = 0; k < PIPE_WMAX; ++k)
        if (k < width) acc += s_val[k * T + t] * (TI)g[k];
    return acc;
}

// Sum K values of type T over the block (FP32 partials are added in FP32 inside the block) and
// store the block's totals as doubles at part[k * nblocks + blockIdx.x].
template <int K, typename T>
__device__ __forceinline__ void block_partials_t(const T (&v0)[K], double* part, unsigned int nblocks, T* s_scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = (blockDim.x + 31) >> 5;
    T v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        v[k] = v0[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) s_scratch[k * 32 + warp] = v[k];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            T s = lane < nwarps ? s_scratch[k * 32 + lane] : (T)0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) part[k * nblocks + blockIdx.x] = (double)s;
        }
    }
}

template <typename TI>
__global__ void __launch_bounds__(512) k_pcg_pipe(PipeArgs<TI> a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_red[32 * 4];
    __shared__ double s_bc[4];
    const int T = blockDim.x, t = threadIdx.x;
    const unsigned int nb = gridDim.x;
    unsigned int epoch = 0;
    const int r0 = blockIdx.x * a.rows_per_block;
    const int row = r0 + t;
    const bool own = (t < a.rows_per_block) && (row < a.n);
    TI* s_val = reinterpret_cast<TI*>(smem);
    int* s_ci = reinterpret_cast<int*>(smem + sizeof(TI) * (size_t)a.width * T);

    // the block's ELL slice of A (inner precision); padding entries point at the row itself
    {
        int k0 = 0, len = 0;
        if (own) {
            k0 = a.rp[row];
            len = a.rp[row + 1] - k0;
        }
        for (int k = 0; k < a.width; ++k) {
            const bool in = own && k < len;
            s_ci[k * T + t] = in ? a.ci[k0 + k] : (own ? row : 0);
            s_val[k * T + t] = in ? a.valI[k0 + k] : (TI)0;
        }
    }
    double bi = own ? a.b[row] : 0.0;
    double xi = own ? a.x[row] : 0.0;
    const TI di = own ? a.dinvI[row] : (TI)0;
    __syncthreads();

    double bb;
    {
        double v[1] = {bi * bi}, tt[1];
        block_partials<1>(v, a.part + PP_P0 * nb, nb, s_red);
        if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
        grid_totals<1>(a.part + PP_P0 * nb, nb, tt, s_bc);
        bb = tt[0];
    }
    if (bb == 0.0) xi = 0.0;
    const double rtol2 = a.rtol * a.rtol, itol2 = a.inner_rtol * a.inner_rtol, floor2 = 0.25 * rtol2;
    int iters = 0, outer = 0, status = CGP_OK;
    double rr64 = 0.0;

    for (;;) {
        // ---- refinement pass: publish x, FP64 true residual
        if (own) a.x[row] = xi;
        if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
        TI r = (TI)0, u = (TI)0, w = (TI)0;
        {
            double ax = 0.0;
            if (own) {
                for (int k = a.rp[row]; k < a.rp[row + 1]; ++k) ax += a.val64[k] * a.x[a.ci[k]];
            }
            const double r64 = own ? bi - ax : 0.0;
            r = (TI)r64;
            u = di * r;
            if (own) a.ubuf[row] = u;
            double v[1] = {r64 * r64}, tt[1];
            block_partials<1>(v, a.part + PP_O1 * nb, nb, s_red);
            if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
            grid_totals<1>(a.part + PP_O1 * nb, nb, tt, s_bc);
            rr64 = tt[0];
        }
        if (bad(rr64)) { status = CGP_ERR_NAN; break; }
        if (bb == 0.0 || rr64 <= rtol2 * bb) break;
        if (outer >= a.max_outer || iters >= a.max_iter) { status = CGP_ERR_NOT_CONVERGED; break; }
        const double tgt = fmax(itol2 * rr64, floor2 * bb);
        // w = A u, then the pipelined iteration from d = 0
        w = own ? ell_row<TI, TI>(s_ci, s_val, T, t, a.width, a.ubuf) : (TI)0;
        TI d = (TI)0, z = (TI)0, q = (TI)0, s = (TI)0, p = (TI)0;
        double alpha = 0.0, gam_old = 0.0;
        double rho_ref = 1.7976931348623157e308;
        int it_ref = iters;
        int par = 0;
        bool first = true, nan = false;
        for (;;) {
            // m = D^-1 w published; partial (r,u), (w,u), (r,r)
            const TI m = di * w;
            if (own) a.mbuf[(size_t)par * a.n + row] = m;
            {
                double v[3] = {(double)(r * u), (double)(w * u), (double)(r * r)};
                block_partials<3>(v, a.part + (PP_I + 3 * par) * nb, nb, s_red);
            }
            if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
            // n = A m overlaps the reduction
            const TI nn = own ? ell_row<TI, TI>(s_ci, s_val, T, t, a.width, a.mbuf + (size_t)par * a.n) : (TI)0;
            double tot[3];
            {
                const int slot[3] = {PP_I + 3 * par, PP_I + 3 * par + 1, PP_I + 3 * par + 2};
                grid_totals_at<3>(a.part, slot, nb, tot, s_bc);
            }
            const double gam = tot[0], del = tot[1], rho = tot[2];
            if (bad(gam) || bad(del) || bad(rho)) { nan = true; break; }
            if (rho <= tgt || iters >= a.max_iter) break;
            // stagnation of the recursive residual (no halving in PIPE_STAGNATION iterations):
            // end the pass; the next one restarts from the FP64 true residual
            if (rho < 0.25 * rho_ref) {
                rho_ref = rho;
                it_ref = iters;
            } else if (iters - it_ref > PIPE_STAGNATION) {
                break;
            }
            double beta, al;
            if (first) {
                beta = 0.0;
                al = del != 0.0 ? gam / del : 0.0;
            } else {
                beta = gam_old != 0.0 ? gam / gam_old : 0.0;
                const double den = del - beta * gam / alpha;
                al = den != 0.0 ? gam / den : 0.0;
            }
            if (al == 0.0) break;     // breakdown: restart from the true residual
            const TI B = (TI)beta, A = (TI)al;
            z = first ? nn : nn + B * z;
            q = first ? m : m + B * q;
            s = first ? w : w + B * s;
            p = first ? u : u + B * p;
            d += A * p;
            r -= A * s;
            u -= A * q;
            w -= A * z;
            alpha = al;
            gam_old = gam;
            first = false;
            par ^= 1;
            iters += 1;
        }
        if (nan) { status = CGP_ERR_NAN; break; }
        xi += (double)d;
        outer += 1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *a.st_iters = iters;
        *a.st_outer = outer;
        *a.st_status = status;
        *a.st_rel = bb > 0.0 ? sqrt(rr64 / bb) : 0.0;
    }
}

// Classical (Chronopoulos-Gear) CG with the same on-chip layout: two grid barriers per
// iteration (one publishes u for the matrix-vector product, one completes the reduction) but
// the stable recurrences of classical CG, which also converge in FP32, and fewer arithmetic
// operations per row (about 17 against 21 for the pipelined form).
enum { PC_P0 = 0, PC_O1 = 1 /* 2 slots */, PC_I0 = 3, PC_I = 4 /* two buffers of 3 */ };

template <typename TI>
__global__ void __launch_bounds__(512) k_pcg_onchip(PipeArgs<TI> a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_red[32 * 4];
    __shared__ TI s_redT[32 * 4];
    __shared__ double s_bc[4];
    __shared__ TI s_ctl[2];
    __shared__ int s_flag;
    const int T = blockDim.x, t = threadIdx.x;
    const unsigned int nb = gridDim.x;
    unsigned int epoch = 0;
    const int row = blockIdx.x * a.rows_per_block + t;
    const bool own = (t < a.rows_per_block) && (row < a.n);
    TI* s_val = reinterpret_cast<TI*>(smem);
    int* s_ci = reinterpret_cast<int*>(smem + sizeof(TI) * (size_t)a.width * T);
    {
        int k0 = 0, len = 0;
        if (own) {
            k0 = a.rp[row];
            len = a.rp[row + 1] - k0;
        }
        for (int k = 0; k < a.width; ++k) {
            const bool in = own && k < len;
            s_ci[k * T + t] = in ? a.ci[k0 + k] : (own ? row : 0);
            s_val[k * T + t] = in ? a.valI[k0 + k] : (TI)0;
        }
    }
    const double bi = own ? a.b[row] : 0.0;
    double xi = own ? a.x[row] : 0.0;
    const TI di = own ? a.dinvI[row] : (TI)0;
    __syncthreads();
    double bb;
    {
        double v[1] = {bi * bi}, tt[1];
        block_partials<1>(v, a.part + PC_P0 * nb, nb, s_red);
        if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
        grid_totals<1>(a.part + PC_P0 * nb, nb, tt, s_bc);
        bb = tt[0];
    }
    if (bb == 0.0) xi = 0.0;
    const double rtol2 = a.rtol * a.rtol, itol2 = a.inner_rtol * a.inner_rtol, floor2 = 0.25 * rtol2;
    int iters = 0, outer = 0, status = CGP_OK;
    double rr64 = 0.0;
    for (;;) {
        // ---- refinement pass: publish x, FP64 true residual, r = (TI) r64, u = D^-1 r
        if (own) a.x[row] = xi;
        if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
        TI r, u;
        double gam;
        {
            double ax = 0.0;
            if (own)
                for (int k = a.rp[row]; k < a.rp[row + 1]; ++k) ax += a.val64[k] * a.x[a.ci[k]];
            const double r64 = own ? bi - ax : 0.0;
            r = (TI)r64;
            u = di * r;
            if (own) a.ubuf[row] = u;
            double v[2] = {r64 * r64, (double)(r * u)}, tt[2];
            block_partials<2>(v, a.part + PC_O1 * nb, nb, s_red);
            if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
            grid_totals<2>(a.part + PC_O1 * nb, nb, tt, s_bc);
            rr64 = tt[0];
            gam = tt[1];
        }
        if (bad(rr64) || bad(gam)) { status = CGP_ERR_NAN; break; }
        if (bb == 0.0 || rr64 <= rtol2 * bb) break;
        if (outer >= a.max_outer || iters >= a.max_iter) { status = CGP_ERR_NOT_CONVERGED; break; }
        const double tgt = fmax(itol2 * rr64, floor2 * bb);
        // ---- w = A u, delta = (w, u)
        TI w = own ? ell_row<TI, TI>(s_ci, s_val, T, t, a.width, a.ubuf) : (TI)0;
        double alpha, beta = 0.0;
        {
            double v[1] = {(double)(w * u)}, tt[1];
            block_partials<1>(v, a.part + PC_I0 * nb, nb, s_red);
            if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
            grid_totals<1>(a.part + PC_I0 * nb, nb, tt, s_bc);
            if (bad(tt[0])) { status = CGP_ERR_NAN; break; }
            alpha = tt[0] != 0.0 ? gam / tt[0] : 0.0;
        }
        TI d = (TI)0, p = (TI)0, s = (TI)0;
        int par = 0;
        bool first = true, nan = false;
        TI A = (TI)alpha, B = (TI)0;
        // every thread leaves this loop on the same broadcast flag (or the same initial alpha)
        while (alpha != 0.0 || !first) {
            // ---- local: p = u + beta p, s = w + beta s, d += alpha p, r -= alpha s, u = D^-1 r
            p = first ? u : u + B * p;
            s = first ? w : w + B * s;
            d += A * p;
            r -= A * s;
            u = di * r;
            if (own) a.ubuf[row] = u;
            const int base = PC_I + 3 * par;
            {
                const TI v[2] = {r * u, r * r};
                block_partials_t<2, TI>(v, a.part + base * nb, nb, s_redT);
            }
            if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
            // ---- w = A u, delta = (w, u)
            w = own ? ell_row<TI, TI>(s_ci, s_val, T, t, a.width, a.ubuf) : (TI)0;
            {
                const TI v[1] = {w * u};
                block_partials_t<1, TI>(v, a.part + (base + 2) * nb, nb, s_redT);
            }
            if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
            {
                const int slot[3] = {base, base + 1, base + 2};
                grid_totals_shared<3>(a.part, slot, nb, s_bc);
            }
            iters += 1;
            first = false;
            par ^= 1;
            // scalar recurrences once per block (thread 0), broadcast through shared memory
            if (t == 0) {
                const double gnew = s_bc[0], rho = s_bc[1], del = s_bc[2];
                int flag = 0;
                if (bad(gnew) || bad(rho) || bad(del)) {
                    flag = 2;
                } else if (rho <= tgt || iters >= a.max_iter || gam == 0.0) {
                    flag = 1;
                } else {
                    const double bnew = gnew / gam;
                    const double den = del - bnew * gnew / alpha;
                    if (den == 0.0 || gnew == 0.0) {
                        flag = 1;
                    } else {
                        beta = bnew;
                        alpha = gnew / den;
                        gam = gnew;
                    }
                }
                s_ctl[0] = (TI)alpha;
                s_ctl[1] = (TI)beta;
                s_flag = flag;
            }
            __syncthreads();
            const int flag = s_flag;
            A = s_ctl[0];
            B = s_ctl[1];
            if (flag == 2) { nan = true; break; }
            if (flag == 1) break;
        }
        if (nan) { status = CGP_ERR_NAN; break; }
        xi += (double)d;
        outer += 1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *a.st_iters = iters;
        *a.st_outer = outer;
        *a.st_status = status;
        *a.st_rel = bb > 0.0 ? sqrt(rr64 / bb) : 0.0;
    }
}

}  // namespace

// Shape of the on-chip Poisson kernel for n rows of maximal length `width`; false if it does
// not fit (rows per block above 1024, rows longer than PIPE_WMAX, or shared memory).
bool pipe_shape(int n, int width, int num_sms, size_t elem, int* blocks, int* threads, size_t* smem) {
    if (width > PIPE_WMAX || n <= 0) return false;
    int nb = std::min(std::min(num_sms, CGP_MAX_GRID), std::max(1, (n + 255) / 256));
    int rpb = (n + nb - 1) / nb;
    if (rpb > 512) return false;
    int T = std::max(128, ((rpb + 31) / 32) * 32);
    size_t sm = (size_t)width * T * (elem + sizeof(int));
    if (sm > 200 * 1024) return false;
    *blocks = nb;
    *threads = T;
    *smem = sm;
    return true;
}

template <typename TI>
static cudaError_t launch_pipe_t(cgp_ctx_s* c, const double* b, double* x, cudaStream_t s, const TI* valI,
                                 const TI* dinvI, int blocks, int threads, size_t smem) {
    PipeArgs<TI> a;
    a.n = c->nc;
    a.rows_per_block = (c->nc + blocks - 1) / blocks;
    a.width = c->width_c;
    a.rp = c->C.rp;
    a.ci = c->C.ci;
    a.val64 = c->Kc;
    a.valI = valI;
    a.dinv64 = c->dinvK;
    a.dinvI = dinvI;
    a.b = b;
    a.x = x;
    char* p = (char*)c->ws;
    a.mbuf = reinterpret_cast<TI*>(p);
    p += ((2 * sizeof(TI) * (size_t)c->nc + 255) / 256) * 256;
    a.ubuf = reinterpret_cast<TI*>(p);
    a.part = c->part;
    a.sw = c->sync + SYNC_POI;
    a.rtol = c->prm.rtol;
    a.inner_rtol = sizeof(TI) == 4 ? c->prm.inner_rtol : 0.0;
    a.max_iter = c->prm.max_iter;
    a.max_outer = c->prm.max_outer;
    a.st_iters = &c->stats->poi_iters;
    a.st_outer = &c->stats->poi_outer;
    a.st_status = &c->stats->poi_status;
    a.st_rel = &c->stats->poi_rel;
    a.st_barrier = &c->stats->barrier_status;
    const void* fn = c->onchip_pipelined ? (const void*)k_pcg_pipe<TI> : (const void*)k_pcg_onchip<TI>;
    cudaError_t e = cudaMemsetAsync(a.sw, 0, sizeof(SyncWords), s);
    if (e != cudaSuccess) return e;
    void* kargs[] = {(void*)&a};
    if (blocks == 1) return cudaLaunchKernel(fn, dim3(1), dim3(threads), kargs, smem, s);
    return cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(threads), kargs, smem, s);
}

// Decide whether the coarse Poisson solve runs on the on-chip kernel and raise its dynamic
// shared-memory limit (once per context, outside any stream capture).
cudaError_t pipe_prepare(cgp_ctx_s* c) {
    int b64, t64, b32, t32;
    size_t s64, s32;
    c->use_pipe = false;
    c->onchip_pipelined = false;
    if (c->prm.coarse_solver == 1) return cudaSuccess;
    // The pipelined form only in FP64: in FP32 its recurrences drift too far from the true
    // residual for the inner solve to reach its target.
    const bool pipelined = c->prm.coarse_solver == 2 && c->prm.precision == CGP_FP64;
    if (!pipe_shape(c->nc, c->width_c, c->num_sms, sizeof(double), &b64, &t64, &s64)) return cudaSuccess;
    if (!pipe_shape(c->nc, c->width_c, c->num_sms, sizeof(float), &b32, &t32, &s32)) return cudaSuccess;
    const void* f64 = pipelined ? (const void*)k_pcg_pipe<double> : (const void*)k_pcg_onchip<double>;
    const void* f32 = pipelined ? (const void*)k_pcg_pipe<float> : (const void*)k_pcg_onchip<float>;
    cudaError_t e = cudaFuncSetAttribute(f64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s64);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s32);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, f64, t64, s64);
    if (e != cudaSuccess || occ < 1) return e;
    c->onchip_pipelined = pipelined;
    c->pipe_c.blocks = b64;
    c->pipe_c.threads = t64;
    c->pipe_smem64 = s64;
    c->pipe_smem32 = s32;
    c->use_pipe = true;
    return cudaSuccess;
}

cudaError_t launch_poisson_pipe(cgp_ctx_s* c, const double* b, double* x, cudaStream_t s) {
    const bool mixed = c->prm.precision == CGP_MIXED;
    if (mixed)
        return launch_pipe_t<float>(c, b, x, s, c->Kc32, c->dinvK32, c->pipe_c.blocks, c->pipe_c.threads,
                                    c->pipe_smem32);
    return launch_pipe_t<double>(c, b, x, s, c->Kc, c->dinvK, c->pipe_c.blocks, c->pipe_c.threads, c->pipe_smem64);
}

}  // namespace cgp
