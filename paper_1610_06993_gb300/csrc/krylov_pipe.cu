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
#include <cmath>
#include <cstdint>
#include <vector>

#include "ctx.h"
#include "subdomain.h"

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

// ---------------------------------------------------------------------------------------------
// Two-level additive Schwarz preconditioned CG, on chip
// ---------------------------------------------------------------------------------------------
// The system is renumbered along a Hilbert curve of the node coordinates so that the contiguous
// row slice of each block is a compact patch (a subdomain). The preconditioner is
//     M^-1 r = sum_a R_a^T q(D_a^-1 A_aa) D_a^-1 R_a r  +  R_0^T A_0^-1 R_0 r
// with q the fixed-degree Chebyshev polynomial for the spectrum bounds [lmin, lmax] of D^-1 A
// (Saad, "Iterative Methods for Sparse Linear Systems", Sect. 12.3, Chebyshev acceleration),
// applied to the block's own rows in shared memory, and a coarse space of three functions per
// subdomain a, its restrictions of 1, (x - xbar_a) / H_a and (y - ybar_a) / H_a (centroid xbar_a,
// ybar_a and RMS radius H_a of the subdomain's nodes): R_0 r holds the three moments of r over
// every subdomain and A_0 = R_0 A R_0^T is the Galerkin matrix, inverted once on the host. The
// linear functions capture the smooth error that a constant per subdomain leaves to the local
// solves, which roughly halves the iteration count again. lmax bounds the spectrum of every D_a^-1 A_aa from
// above (Cauchy interlacing), which keeps q positive on it, so both parts are symmetric positive
// definite and M^-1 is a valid CG preconditioner. The local solve overlaps the grid barrier that
// gathers R_0 r. TI is the precision of the CG iteration, TP that of the preconditioner; with
// TP = float inside FP64 iterations the preconditioner is a slightly inexact fixed operator,
// which slows CG a little but leaves its recursive residual exact (it is built from A p alone).
template <typename TI, typename TP>
struct SchwarzArgs {
    int n, rows_per_block, width, degree;
    const int* perm;        // [n] renumbered row -> caller row
    const int* rp;          // renumbered CSR
    const int* ci;
    const double* val64;
    const TI* valI;
    const TP* valP;
    const TP* dinvP;        // [n] renumbered inverse diagonal
    const TP* fxy;          // [n][2] renumbered values of the two linear coarse functions
    const TP* ainv;         // [3 nb][3 nb] inverse of the coarse Galerkin matrix
    double lmin, lmax;
    const double* b;        // [n] caller numbering
    double* x;              // [n] caller numbering
    double* xp;             // [n] published x, renumbered
    TI* ubuf;               // [n] published u, renumbered
    double* part;
    SyncWords* sw;
    double rtol, inner_rtol;
    int max_iter, max_outer;
    int* st_iters;
    int* st_outer;
    int* st_status;
    double* st_rel;
    int* st_barrier;
};

// Subdomains per block: consecutive parts of ceil(rpb / SZ_SUB) rows of the block's row slice.
// Coarse index of function f on subdomain h of block b: f * (SZ_SUB nb) + SZ_SUB b + h.
#ifndef SZ_SUB
#define SZ_SUB 3
#endif

enum { PS_P0 = 0, PS_O1 = 1 /* 2 slots */, PS_I0 = 3, PS_R = 4 /* SZ_NC SZ_SUB slots */,
       PS_F = 4 + SZ_NC * SZ_SUB /* 3 products, then 3 SZ_NC SZ_SUB moments */,
       PS_END = PS_F + 3 + 3 * SZ_NC * SZ_SUB };
static_assert(PS_END <= CGP_PART_SLOTS, "partial-sum slots");

// Subdomain of every renumbered row: the part of its block's slice of rpb rows.
std::vector<int> onchip_subdomains(int n, int rpb) {
    const int hs = (rpb + SZ_SUB - 1) / SZ_SUB;
    std::vector<int> sub(n);
    for (int i = 0; i < n; ++i) sub[i] = SZ_SUB * (i / rpb) + (i % rpb) / hs;
    return sub;
}

// One entry of the subdomain matrix A_aa in shared memory: column local to the block, value.
template <typename TP> struct LocEnt;
template <> struct __align__(8) LocEnt<float> { int c; float v; };
template <> struct __align__(16) LocEnt<double> { int c; int pad; double v; };

// Dynamic shared memory of k_pcg_schwarz: the block's ELL slice of A (values in TI, global
// columns), the compact ELL slice of A_aa (local columns, values in TP), two Chebyshev buffers,
// the FP64 reduction buffer (three values per thread), the block's SZ_NC SZ_SUB rows of A_0^-1,
// R_0 r, the gathered moments R_0 w, R_0 r, R_0 s of the last reduction and the per-thread
// moments of that reduction (9 per thread). T is a multiple of 32, so every region before the TP
// arrays ends on a 128-byte boundary.
size_t schwarz_smem(int width, int T, int nb, size_t sti, size_t stp) {
    const size_t wt = (size_t)width * T;
    const size_t ncs = (size_t)SZ_NC * SZ_SUB * nb;
    const size_t loc = stp == sizeof(float) ? sizeof(LocEnt<float>) : sizeof(LocEnt<double>);
    return wt * (sti + sizeof(int)) + wt * loc + 2 * (size_t)T * stp + 3 * (size_t)T * sizeof(double) +
           (SZ_NC * SZ_SUB + 1 + 3) * ncs * stp + 3 * SZ_NC * (size_t)T * stp;
}

// Iteration (Chronopoulos-Gear CG with the two-level Schwarz preconditioner M^-1 = local
// Chebyshev solves + R_0^T A_0^-1 R_0; two grid barriers per iteration):
//   reduction of (r,u), (r,r), (w,u) and of the coarse moments R_0 w, R_0 r, R_0 s | barrier
//   totals and every block's moments; alpha, beta (thread 0)
//   p = u + beta p,  s = w + beta s,  d += alpha p,  r -= alpha s                         (local)
//   R_0 s <- R_0 w + beta R_0 s,  R_0 r <- R_0 r - alpha R_0 s  (one step from exact moments)
//   u = Chebyshev(A_aa, r) + R_0^T A_0^-1 R_0 r;  publish u | barrier | w = A u
// The moments of the new residual follow from the exact moments of the vectors it is formed
// from, so the coarse correction needs no reduction of its own, and they never drift: each
// reduction recomputes them from the vectors.
template <typename TI, typename TP>
__global__ void __launch_bounds__(512) k_pcg_schwarz(SchwarzArgs<TI, TP> a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ TP s_redP[32 * SZ_NC * SZ_SUB];
    __shared__ double s_bc[4];
    __shared__ double s_ctl[2];
    __shared__ int s_flag;
    __shared__ TP s_y[SZ_NC * SZ_SUB];   // [f][h]
    const int T = blockDim.x, t = threadIdx.x, lane = t & 31, warp = t >> 5, nwarps = T >> 5;
    const unsigned int nb = gridDim.x;
    unsigned int epoch = 0;
    const int r0 = min(a.n, (int)blockIdx.x * a.rows_per_block);
    const int r1 = min(a.n, r0 + a.rows_per_block);
    const int row = r0 + t;
    const bool own = row < r1;
    const size_t wt = (size_t)a.width * T;
    TI* s_val = reinterpret_cast<TI*>(smem);
    int* s_ci = reinterpret_cast<int*>(smem + sizeof(TI) * wt);
    LocEnt<TP>* s_loc = reinterpret_cast<LocEnt<TP>*>(smem + (sizeof(TI) + sizeof(int)) * wt);
    TP* s_z = reinterpret_cast<TP*>(s_loc + wt);                                  // [2][T]
    double* s_lean = reinterpret_cast<double*>(s_z + 2 * T);                      // [3][T]
    const unsigned int nsub = SZ_SUB * nb, ncs = SZ_NC * nsub;
    TP* s_ainv = reinterpret_cast<TP*>(s_lean + 3 * T);   // [SZ_NC SZ_SUB][ncs]: rows (f, h)
    TP* s_rc = s_ainv + SZ_NC * SZ_SUB * ncs;             // [ncs] R_0 r of the current residual
    TP* s_Rw = s_rc + ncs;                                // [ncs] moments of the last reduction
    TP* s_Rr = s_Rw + ncs;
    TP* s_Rs = s_Rr + ncs;
    TP* s_mom = s_Rs + ncs;                               // [3 SZ_NC][T] this thread's moments
    const int hs = (a.rows_per_block + SZ_SUB - 1) / SZ_SUB;   // rows per part of the slice
    const int hh = t / hs;                                     // this row's part
    int wl, wloc;   // longest row / longest A_aa row among this warp's rows (warp-uniform loop ends)
    {
        int k0 = 0, len = 0, m = 0;
        if (own) {
            k0 = a.rp[row];
            len = a.rp[row + 1] - k0;
        }
        wl = __reduce_max_sync(0xffffffffu, len);
        for (int k = 0; k < a.width; ++k) {
            const bool in = own && k < len;
            const int c = in ? a.ci[k0 + k] : -1;
            s_ci[k * T + t] = c;
            s_val[k * T + t] = in ? a.valI[k0 + k] : (TI)0;
            if (c >= r0 && c < r1) {
                LocEnt<TP> e;
                e.c = c - r0;
                e.v = a.valP[k0 + k];
                s_loc[m * T + t] = e;
                m += 1;
            }
        }
        wloc = __reduce_max_sync(0xffffffffu, m);
        for (int k = m; k < a.width; ++k) {   // padding: own slot, zero weight
            LocEnt<TP> e;
            e.c = t;
            e.v = (TP)0;
            s_loc[k * T + t] = e;
        }
        for (unsigned int j = t; j < SZ_NC * SZ_SUB * ncs; j += T) {
            const unsigned int k = j / ncs, col = j - k * ncs, f = k / SZ_SUB, h = k - f * SZ_SUB;
            s_ainv[j] = a.ainv[(size_t)(f * nsub + SZ_SUB * blockIdx.x + h) * ncs + col];
        }
    }
    const int crow = own ? a.perm[row] : 0;
    const double bi = own ? a.b[crow] : 0.0;
    double xi = own ? a.x[crow] : 0.0;
    const TP di = own ? a.dinvP[row] : (TP)0;
    const TP fx = own ? a.fxy[2 * row] : (TP)0, fy = own ? a.fxy[2 * row + 1] : (TP)0;
    const TP theta = (TP)(0.5 * (a.lmax + a.lmin)), delta = (TP)(0.5 * (a.lmax - a.lmin));
    const TP sigma = theta / delta;
    __syncthreads();

    // local part: Chebyshev iteration on A_aa z = r from z = 0 (s_z double buffered)
    auto chebyshev = [&](TI rI) -> TP {
        const TP r = (TP)rI;
        TP rho = (TP)1 / sigma;
        TP d = di * r / theta;
        TP z = d;
        for (int j = 1; j < a.degree; ++j) {
            TP* zb = s_z + (j & 1) * T;
            zb[t] = z;
            __syncthreads();
            TP az = (TP)0;
#pragma unroll
            for (int k = 0; k < PIPE_WMAX; ++k) {
                if (k < wloc) {
                    const LocEnt<TP> e = s_loc[k * T + t];
                    az += e.v * zb[e.c];
                }
            }
            const TP rn = (TP)1 / ((TP)2 * sigma - rho);
            d = rn * rho * d + ((TP)2 * rn / delta) * di * (r - az);
            z += d;
            rho = rn;
        }
        return z;
    };
    // coarse part: s_y = the block's SZ_NC SZ_SUB entries of A_0^-1 (R_0 r) from s_rc, warp w
    // taking entries w, w + warps, ... (a 128-thread block has fewer warps than entries)
    auto coarse_solve = [&]() {
        for (int k = warp; k < SZ_NC * SZ_SUB; k += nwarps) {
            const TP* arow = s_ainv + k * ncs;
            TP acc = (TP)0;
            for (unsigned int j = lane; j < ncs; j += 32) acc += arow[j] * s_rc[j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) s_y[k] = acc;
        }
        __syncthreads();
    };
    auto coarse_value = [&]() -> TP { return s_y[hh] + fx * s_y[SZ_SUB + hh] + fy * s_y[2 * SZ_SUB + hh]; };

    // u = M^-1 r with the moments of r reduced explicitly (the refinement pass); every thread of
    // every block calls it the same number of times. False if the grid barrier inside failed.
    auto precondition = [&](TI rI, TI& u) -> bool {
        {
            // slot PS_R + 3 h + f holds function f on part h of every block
            const TP r = (TP)rI, rf[SZ_NC] = {r, fx * r, fy * r};
            TP v[SZ_NC * SZ_SUB];
#pragma unroll
            for (int h = 0; h < SZ_SUB; ++h)
#pragma unroll
                for (int f = 0; f < SZ_NC; ++f) v[SZ_NC * h + f] = hh == h ? rf[f] : (TP)0;
            block_partials_t<SZ_NC * SZ_SUB, TP>(v, a.part + PS_R * nb, nb, s_redP);
        }
        grid_arrive(a.sw, nb, epoch);
        const TP z = chebyshev(rI);
        if (!grid_wait(a.sw, nb, epoch)) return false;
        constexpr int GQ = 4;   // all loads of a round in flight before the first store
        for (unsigned int j0 = t; j0 < ncs; j0 += GQ * T) {
            double m[GQ];
#pragma unroll
            for (int q = 0; q < GQ; ++q) {
                const unsigned int j = j0 + q * T;
                m[q] = 0.0;
                if (j < ncs) {
                    const unsigned int f = j / nsub, rem = j - f * nsub, b = rem / SZ_SUB, h = rem - b * SZ_SUB;
                    m[q] = __ldcg(a.part + (size_t)(PS_R + SZ_NC * h + f) * nb + b);
                }
            }
#pragma unroll
            for (int q = 0; q < GQ; ++q)
                if (j0 + q * T < ncs) s_rc[j0 + q * T] = (TP)m[q];
        }
        __syncthreads();
        coarse_solve();
        u = own ? (TI)(z + coarse_value()) : (TI)0;
        return true;
    };

    // One reduction of the products (r,u), (r,r), (w,u) and the moments of w, r, s on this
    // block's parts: slot PS_F + q for product q; from slot PS_F + 3 on, the moments (stored in
    // TP) in coarse order, entry (3 v + f) nsub + SZ_SUB b + h for function f of vector v (w, r,
    // s) on part h of block b, so that every block gathers them with one contiguous copy. Warp w sums tasks w,
    // w + warps, ...: a product over the whole block (FP64 for FP64 iterations), a moment over one
    // part (in TP); fixed order.
    auto reduce_fused = [&](TI rI, TI uI, TI wI, TI sI) {
        __syncthreads();   // earlier readers of s_lean / s_mom are done
        if constexpr (sizeof(TI) == sizeof(double)) {
            s_lean[t] = (double)(rI * uI);
            s_lean[T + t] = (double)(rI * rI);
            s_lean[2 * T + t] = (double)(wI * uI);
        } else {
            TI* sl = reinterpret_cast<TI*>(s_lean);
            sl[t] = rI * uI;
            sl[T + t] = rI * rI;
            sl[2 * T + t] = wI * uI;
        }
        {
            const TP vec[3] = {(TP)wI, (TP)rI, (TP)sI};
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                s_mom[(3 * v) * T + t] = vec[v];
                s_mom[(3 * v + 1) * T + t] = fx * vec[v];
                s_mom[(3 * v + 2) * T + t] = fy * vec[v];
            }
        }
        __syncthreads();
        // with 8 or more warps the three products (the longer sums) go to the last three warps
        // and the moments to the others; fewer warps take the tasks in order
        const bool split = nwarps >= 8;
        const int w0 = split ? (warp >= nwarps - 3 ? warp - (nwarps - 3) : 3 + warp) : warp;
        const int stride = split ? (warp >= nwarps - 3 ? 1 << 30 : nwarps - 3) : nwarps;
        for (int q = w0; q < 3 + 3 * SZ_NC * SZ_SUB; q += stride) {
            double tot;
            if (q < 3) {
                if constexpr (sizeof(TI) == sizeof(double)) {
                    const double* b = s_lean + q * T;
                    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
                    int j = lane;
                    for (; j + 96 < T; j += 128) {
                        a0 += b[j];
                        a1 += b[j + 32];
                        a2 += b[j + 64];
                        a3 += b[j + 96];
                    }
                    for (; j < T; j += 32) a0 += b[j];
                    double acc = (a0 + a1) + (a2 + a3);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                    tot = acc;
                } else {
                    const TI* b = reinterpret_cast<const TI*>(s_lean) + q * T;
                    TI acc = (TI)0;
                    for (int j = lane; j < T; j += 32) acc += b[j];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                    tot = (double)acc;
                }
            } else {
                const int m = q - 3, k = m / SZ_SUB, h = m - k * SZ_SUB;
                const TP* b = s_mom + k * T;
                const int j1 = min(T, (h + 1) * hs);
                TP acc = (TP)0;
                for (int j = h * hs + lane; j < j1; j += 32) acc += b[j];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (lane == 0)
                    reinterpret_cast<TP*>(a.part + (size_t)(PS_F + 3) * nb)[(size_t)k * nsub + SZ_SUB * blockIdx.x + h] = acc;
                continue;
            }
            if (lane == 0) a.part[(size_t)(PS_F + q) * nb + blockIdx.x] = tot;
        }
    };
    // after the barrier: the three totals into s_bc, every block's moments into s_Rw, s_Rr, s_Rs
    // in coarse order (index f nsub + SZ_SUB b + h)
    auto gather_fused = [&]() {
        if (warp < 3) {
            const double* pp = a.part + (size_t)(PS_F + warp) * nb;
            double v[CGP_MAX_GRID / 32];
#pragma unroll
            for (int q = 0; q < CGP_MAX_GRID / 32; ++q) {
                const unsigned int b = lane + 32u * q;
                v[q] = b < nb ? __ldcg(pp + b) : 0.0;
            }
            double tt = 0.0;
#pragma unroll
            for (int q = 0; q < CGP_MAX_GRID / 32; ++q) tt += v[q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) tt += __shfl_xor_sync(0xffffffffu, tt, o);
            if (lane == 0) s_bc[warp] = tt;
        }
        // the moments: a contiguous copy into s_Rw, s_Rr, s_Rs (consecutive [3][ncs]), all loads
        // of a round in flight before the first store (16-byte loads for FP32 moments: the
        // region starts at a multiple of 128 nb bytes)
        const TP* src = reinterpret_cast<const TP*>(a.part + (size_t)(PS_F + 3) * nb);
        const unsigned int lim = 3 * ncs;
        if constexpr (sizeof(TP) == sizeof(float)) {
            const unsigned int n4 = lim / 4;
            const float4* s4 = reinterpret_cast<const float4*>(src);
            constexpr int GQ = 4;
            for (unsigned int i0 = t; i0 < n4; i0 += GQ * T) {
                float4 m[GQ];
#pragma unroll
                for (int q = 0; q < GQ; ++q) {
                    const unsigned int i = i0 + q * T;
                    m[q] = i < n4 ? __ldcg(s4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int q = 0; q < GQ; ++q) {
                    const unsigned int i = i0 + q * T;
                    if (i < n4) {
                        s_Rw[4 * i] = m[q].x;
                        s_Rw[4 * i + 1] = m[q].y;
                        s_Rw[4 * i + 2] = m[q].z;
                        s_Rw[4 * i + 3] = m[q].w;
                    }
                }
            }
            for (unsigned int i = 4 * n4 + t; i < lim; i += T) s_Rw[i] = __ldcg(src + i);
        } else {
            constexpr int GQ = 10;
            for (unsigned int i0 = t; i0 < lim; i0 += GQ * T) {
                TP m[GQ];
#pragma unroll
                for (int q = 0; q < GQ; ++q) {
                    const unsigned int i = i0 + q * T;
                    m[q] = i < lim ? __ldcg(src + i) : (TP)0;
                }
#pragma unroll
                for (int q = 0; q < GQ; ++q) {
                    const unsigned int i = i0 + q * T;
                    if (i < lim) s_Rw[i] = m[q];
                }
            }
        }
        __syncthreads();
    };

    const double rtol2 = a.rtol * a.rtol, itol2 = a.inner_rtol * a.inner_rtol, floor2 = 0.25 * rtol2;
    int iters = 0, outer = 0, status = CGP_OK;
    double rr64 = 0.0, bb = -1.0;   // ||b||^2, taken in the first pass's reduction
    for (;;) {
        // ---- refinement pass: publish x, FP64 true residual and its norm (with ||b||^2), stop if
        // converged; else u = M^-1 r, published for w = A u
        if (own) a.xp[row] = xi;
        if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
        TI r, u;
        double r64;
        {
            double ax = 0.0;
            if (own)
                for (int k = a.rp[row]; k < a.rp[row + 1]; ++k) ax += a.val64[k] * a.xp[a.ci[k]];
            r64 = own ? bi - ax : 0.0;
            r = (TI)r64;
        }
        {
            double v[2] = {r64 * r64, bi * bi}, tt[2];
            block_partials_lean<2>(v, a.part + PS_O1 * nb, nb, blockIdx.x, s_lean);
            if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
            grid_totals<2>(a.part + PS_O1 * nb, nb, tt, s_bc);
            rr64 = tt[0];
            if (bb < 0.0) bb = tt[1];
        }
        if (bb == 0.0) {   // zero right-hand side: the zero solution
            xi = 0.0;
            rr64 = 0.0;
            break;
        }
        if (bad(rr64)) { status = CGP_ERR_NAN; break; }
        if (rr64 <= rtol2 * bb) break;
        if (outer >= a.max_outer || iters >= a.max_iter) { status = CGP_ERR_NOT_CONVERGED; break; }
        const double tgt = fmax(itol2 * rr64, floor2 * bb);
        if (!precondition(r, u)) return record_failure(a.sw, a.st_barrier);
        if (own) a.ubuf[row] = u;
        if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
        TI w = own ? ell_row<TI, TI>(s_ci, s_val, T, t, wl, a.ubuf) : (TI)0;
        TI d = (TI)0, p = (TI)0, s = (TI)0;
        double alpha = 0.0, beta = 0.0, gam = 0.0;
        bool first = true, nan = false, fail = false;
        for (;;) {
            reduce_fused(r, u, w, s);
            if (!grid_sync(a.sw, nb, epoch)) { fail = true; break; }
            gather_fused();
            if (!first) iters += 1;
            if (t == 0) {
                const double gnew = s_bc[0], rho = s_bc[1], del = s_bc[2];
                int flag = 0;
                if (bad(gnew) || bad(rho) || bad(del)) {
                    flag = 2;
                } else if (first) {
                    if (del == 0.0 || gnew == 0.0) {
                        flag = 1;
                    } else {
                        gam = gnew;
                        alpha = gnew / del;
                        beta = 0.0;
                    }
                } else if (rho <= tgt || iters >= a.max_iter || gam == 0.0) {
                    flag = 1;
                } else {
                    // beta = gnew / gam and alpha' = gnew / (del - gnew^2 / (gam alpha))
                    // = gnew gam alpha / (del gam alpha - gnew^2): two independent divisions
                    // (a dependent FP64 operation costs tens of cycles on this GPU)
                    const double ga = gam * alpha;
                    const double den = fma(del, ga, -gnew * gnew);
                    if (den == 0.0 || gnew == 0.0) {
                        flag = 1;
                    } else {
                        beta = gnew / gam;
                        alpha = (gnew * ga) / den;
                        gam = gnew;
                    }
                }
                s_ctl[0] = alpha;
                s_ctl[1] = beta;
                s_flag = flag;
            }
            __syncthreads();
            const int flag = s_flag;
            alpha = s_ctl[0];
            beta = s_ctl[1];
            if (flag == 2) { nan = true; break; }
            if (flag == 1) break;
            const TI A = (TI)alpha, B = (TI)beta;
            p = first ? u : u + B * p;
            s = first ? w : w + B * s;
            d += A * p;
            r -= A * s;
            {
                const TP Ap = (TP)alpha, Bp = (TP)beta;
                for (unsigned int j = t; j < ncs; j += T) {
                    const TP rs = first ? s_Rw[j] : s_Rw[j] + Bp * s_Rs[j];
                    s_rc[j] = s_Rr[j] - Ap * rs;
                }
            }
            __syncthreads();
            coarse_solve();
            const TP z = chebyshev(r);
            u = own ? (TI)(z + coarse_value()) : (TI)0;
            // publish u (a pure barrier), then w = A u
            if (own) a.ubuf[row] = u;
            if (!grid_sync(a.sw, nb, epoch)) { fail = true; break; }
            w = own ? ell_row<TI, TI>(s_ci, s_val, T, t, wl, a.ubuf) : (TI)0;
            first = false;
        }
        if (fail) return record_failure(a.sw, a.st_barrier);
        if (nan) { status = CGP_ERR_NAN; break; }
        xi += (double)d;
        outer += 1;
    }
    if (own) a.x[crow] = xi;
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

namespace {

template <typename T>
cudaError_t sz_alloc(cgp_ctx_s* c, T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    c->allocs.push_back(q);
    *p = (T*)q;
    return cudaSuccess;
}

template <typename T>
cudaError_t sz_upload(T* dst, const std::vector<T>& v) {
    return cudaMemcpy(dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

// Renumbering of the coarse nodes along a Hilbert curve of their coordinates (one scale for
// both axes, so a subdomain is compact in physical space), the renumbered CSR pattern and the
// device buffers of the Schwarz solver.
cudaError_t schwarz_structure(cgp_ctx_s* c) {
    const HostCsr& H = c->hm.coarse;
    const std::vector<double>& xy = c->hm.lv[0].xy;
    const int n = c->nc, nb = c->pipe_c.blocks;
    std::vector<int> perm = hilbert_order(xy, n), iperm(n);
    // within each subdomain, longest rows first: the warps of a block then see nearly uniform row
    // lengths and their ELL loops stop at the warp's own longest row
    {
        const int rpb0 = (n + nb - 1) / nb, hs = (rpb0 + SZ_SUB - 1) / SZ_SUB;
        auto len = [&](int i) { return H.rp[i + 1] - H.rp[i]; };
        for (int b0 = 0; b0 < n; b0 += rpb0)
            for (int h0 = b0; h0 < std::min(n, b0 + rpb0); h0 += hs)   // within each part (subdomain)
                std::stable_sort(perm.begin() + h0, perm.begin() + std::min({n, b0 + rpb0, h0 + hs}),
                                 [&](int p, int q) { return len(p) > len(q); });
    }
    for (int i = 0; i < n; ++i) iperm[perm[i]] = i;
    c->sz_rp_h.assign(1, 0);
    c->sz_ci_h.clear();
    c->sz_src.clear();
    for (int i = 0; i < n; ++i) {
        const int o = perm[i];
        for (int k = H.rp[o]; k < H.rp[o + 1]; ++k) {
            c->sz_ci_h.push_back(iperm[H.ci[k]]);
            c->sz_src.push_back(k);
        }
        c->sz_rp_h.push_back((int)c->sz_ci_h.size());
    }
    const size_t nnz = c->sz_ci_h.size();
    // linear coarse functions (x - xbar_a) / H_a, (y - ybar_a) / H_a of each subdomain a
    const int rpb = (n + nb - 1) / nb;
    c->sz_fxy_h = linear_functions(xy, perm, onchip_subdomains(n, rpb), n, SZ_SUB * nb);
    const std::vector<float> fxy32(c->sz_fxy_h.begin(), c->sz_fxy_h.end());
    const size_t ncs = (size_t)SZ_NC * SZ_SUB * nb;
    cudaError_t e;
    if ((e = sz_alloc(c, &c->sz_perm, n)) != cudaSuccess) return e;
    if ((e = sz_alloc(c, &c->sz_rp, n + 1)) != cudaSuccess) return e;
    if ((e = sz_alloc(c, &c->sz_ci, nnz)) != cudaSuccess) return e;
    if ((e = sz_alloc(c, &c->sz_val64, nnz)) != cudaSuccess) return e;
    if ((e = sz_alloc(c, &c->sz_val32, nnz)) != cudaSuccess) return e;
    if ((e = sz_alloc(c, &c->sz_dinv64, n)) != cudaSuccess) return e;
    if ((e = sz_alloc(c, &c->sz_dinv32, n)) != cudaSuccess) return e;
    if ((e = sz_alloc(c, &c->sz_ainv64, ncs * ncs)) != cudaSuccess) return e;
    if ((e = sz_alloc(c, &c->sz_ainv32, ncs * ncs)) != cudaSuccess) return e;
    if ((e = sz_alloc(c, &c->sz_fxy64, 2 * (size_t)n)) != cudaSuccess) return e;
    if ((e = sz_alloc(c, &c->sz_fxy32, 2 * (size_t)n)) != cudaSuccess) return e;
    if ((e = sz_upload(c->sz_fxy64, c->sz_fxy_h)) != cudaSuccess) return e;
    if ((e = sz_upload(c->sz_fxy32, fxy32)) != cudaSuccess) return e;
    if ((e = sz_upload(c->sz_perm, perm)) != cudaSuccess) return e;
    if ((e = sz_upload(c->sz_rp, c->sz_rp_h)) != cudaSuccess) return e;
    return sz_upload(c->sz_ci, c->sz_ci_h);
}

template <typename TI, typename TP>
const void* schwarz_kernel() {
    return (const void*)k_pcg_schwarz<TI, TP>;
}

const void* schwarz_kernel_for(const cgp_ctx_s* c) {
    if (c->prm.precision == CGP_MIXED) return schwarz_kernel<float, float>();
    return c->schwarz_fp32 ? schwarz_kernel<double, float>() : schwarz_kernel<double, double>();
}

}  // namespace

// Decide whether the coarse Poisson solve runs on an on-chip kernel and raise its dynamic
// shared-memory limit (once per context, outside any stream capture).
cudaError_t pipe_prepare(cgp_ctx_s* c) {
    int b64, t64, b32, t32;
    size_t s64, s32;
    c->use_pipe = false;
    c->onchip_pipelined = false;
    c->use_schwarz = false;
    if (c->prm.coarse_solver == 1) return cudaSuccess;
    const bool schwarz = c->prm.coarse_solver == 0 || c->prm.coarse_solver == 3 || c->prm.coarse_solver == 4;
    if (schwarz) {
        const bool mixed = c->prm.precision == CGP_MIXED;
        c->schwarz_fp32 = mixed || c->prm.coarse_solver != 4;
        const size_t sti = mixed ? sizeof(float) : sizeof(double);
        const size_t stp = c->schwarz_fp32 ? sizeof(float) : sizeof(double);
        int nb = 0, T = 0;
        size_t sm0 = 0, sm = 0;
        const bool fits = pipe_shape(c->nc, c->width_c, c->num_sms, sti, &nb, &T, &sm0) &&
                          (sm = schwarz_smem(c->width_c, T, nb, sti, stp)) <= 200 * 1024;
        const void* fn = schwarz_kernel_for(c);
        int occ = 0;
        if (fits) {
            cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return e;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, T, sm);
            if (e != cudaSuccess) return e;
        }
        if (fits && occ >= 1) {
            c->pipe_c.blocks = nb;
            c->pipe_c.threads = T;
            c->sz_smem = sm;
            c->sz_degree = c->prm.precond_degree > 0 ? c->prm.precond_degree : 6;
            c->sz_ratio = c->prm.precond_ratio > 1.0 ? c->prm.precond_ratio : 30.0;
            cudaError_t e = schwarz_structure(c);
            if (e != cudaSuccess) return e;
            c->use_schwarz = true;
            c->use_pipe = true;
            return cudaSuccess;
        }
        // automatic choice: the Jacobi on-chip kernel next, then the generic kernel
        if (c->prm.coarse_solver != 0) return cudaSuccess;
    }
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

// Values of the Schwarz solver for the current boundary conditions (after the symmetric
// elimination of the pressure-Dirichlet rows): renumbered FP64/FP32 matrix values and inverse
// diagonal, the spectrum bound of D^-1 A for the Chebyshev polynomial, and the inverse of the
// Galerkin coarse matrix A_0 = R_0 A R_0^T by Cholesky factorisation. A coarse function that
// vanishes on its subdomain (all nodes at one point) gets a unit diagonal and no coupling.
int schwarz_values(cgp_ctx_s* c) {
    if (!c->use_schwarz) return CGP_OK;
    const int n = c->nc, nb = c->pipe_c.blocks;
    const int rpb = (n + nb - 1) / nb;
    const std::vector<int>& rp = c->sz_rp_h;
    const std::vector<int>& ci = c->sz_ci_h;
    const size_t nnz = ci.size();
    std::vector<double> K(c->hm.coarse.nnz), v(nnz), dg(n, 0.0);
    if (cudaMemcpy(K.data(), c->Kc, K.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
        return CGP_ERR_CUDA;
    for (size_t k = 0; k < nnz; ++k) v[k] = K[c->sz_src[k]];
    for (int i = 0; i < n; ++i)
        for (int k = rp[i]; k < rp[i + 1]; ++k)
            if (ci[k] == i) dg[i] = v[k];
    for (int i = 0; i < n; ++i)
        if (!(dg[i] > 0.0)) return CGP_ERR_ARG;   // not symmetric positive definite
    // upper bound of the spectrum of D^-1 A: the smaller of the Gershgorin bound and 1.2 times a
    // power-iteration estimate on D^-1/2 A D^-1/2 (same spectrum)
    double gersh = 0.0;
    for (int i = 0; i < n; ++i) {
        double sum = 0.0;
        for (int k = rp[i]; k < rp[i + 1]; ++k) sum += std::fabs(v[k]);
        gersh = std::max(gersh, sum / dg[i]);
    }
    std::vector<double> z(n), w(n), sq(n);
    for (int i = 0; i < n; ++i) {
        sq[i] = 1.0 / std::sqrt(dg[i]);
        z[i] = 1.0 + 0.5 * std::sin(1.0 + 12.9898 * i);   // fixed, non-smooth start
    }
    double lam = 0.0;
    for (int it = 0; it < 100; ++it) {
        double zz = 0.0, zw = 0.0;
        for (int i = 0; i < n; ++i) {
            double acc = 0.0;
            for (int k = rp[i]; k < rp[i + 1]; ++k) acc += v[k] * sq[ci[k]] * z[ci[k]];
            w[i] = sq[i] * acc;
            zz += z[i] * z[i];
            zw += z[i] * w[i];
        }
        lam = zw / zz;
        double ww = 0.0;
        for (int i = 0; i < n; ++i) ww += w[i] * w[i];
        const double inv = ww > 0.0 ? 1.0 / std::sqrt(ww) : 0.0;
        for (int i = 0; i < n; ++i) z[i] = w[i] * inv;
    }
    c->sz_lmax = std::min(gersh, 1.2 * lam);
    c->sz_lmin = c->sz_lmax / c->sz_ratio;
    std::vector<double> Ai;
    {
        const int st = galerkin_inverse(rp, ci, v, c->sz_fxy_h, onchip_subdomains(n, rpb), n, SZ_SUB * nb, Ai);
        if (st != CGP_OK) return st;
    }
    std::vector<double> dinv(n);
    for (int i = 0; i < n; ++i) dinv[i] = 1.0 / dg[i];
    std::vector<float> v32(v.begin(), v.end()), dinv32(dinv.begin(), dinv.end()), ai32(Ai.begin(), Ai.end());
    if (sz_upload(c->sz_val64, v) != cudaSuccess || sz_upload(c->sz_val32, v32) != cudaSuccess ||
        sz_upload(c->sz_dinv64, dinv) != cudaSuccess || sz_upload(c->sz_dinv32, dinv32) != cudaSuccess ||
        sz_upload(c->sz_ainv64, Ai) != cudaSuccess || sz_upload(c->sz_ainv32, ai32) != cudaSuccess)
        return CGP_ERR_CUDA;
    return CGP_OK;
}

template <typename TI, typename TP>
static cudaError_t launch_schwarz_t(cgp_ctx_s* c, const double* b, double* x, cudaStream_t s, const TI* valI,
                                    const TP* valP, const TP* dinvP, const TP* fxy, const TP* ainv) {
    SchwarzArgs<TI, TP> a;
    const int nb = c->pipe_c.blocks;
    a.n = c->nc;
    a.rows_per_block = (c->nc + nb - 1) / nb;
    a.width = c->width_c;
    a.degree = c->sz_degree;
    a.perm = c->sz_perm;
    a.rp = c->sz_rp;
    a.ci = c->sz_ci;
    a.val64 = c->sz_val64;
    a.valI = valI;
    a.valP = valP;
    a.dinvP = dinvP;
    a.fxy = fxy;
    a.ainv = ainv;
    a.lmin = c->sz_lmin;
    a.lmax = c->sz_lmax;
    a.b = b;
    a.x = x;
    char* p = (char*)c->ws;
    a.xp = reinterpret_cast<double*>(p);
    p += ((sizeof(double) * (size_t)c->nc + 255) / 256) * 256;
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
    cudaError_t e = cudaMemsetAsync(a.sw, 0, sizeof(SyncWords), s);
    if (e != cudaSuccess) return e;
    void* kargs[] = {(void*)&a};
    const void* fn = (const void*)k_pcg_schwarz<TI, TP>;
    if (nb == 1) return cudaLaunchKernel(fn, dim3(1), dim3(c->pipe_c.threads), kargs, c->sz_smem, s);
    return cudaLaunchCooperativeKernel(fn, dim3(nb), dim3(c->pipe_c.threads), kargs, c->sz_smem, s);
}

cudaError_t launch_poisson_pipe(cgp_ctx_s* c, const double* b, double* x, cudaStream_t s) {
    const bool mixed = c->prm.precision == CGP_MIXED;
    if (c->use_schwarz) {
        if (mixed)
            return launch_schwarz_t<float, float>(c, b, x, s, c->sz_val32, c->sz_val32, c->sz_dinv32, c->sz_fxy32,
                                                  c->sz_ainv32);
        if (c->schwarz_fp32)
            return launch_schwarz_t<double, float>(c, b, x, s, c->sz_val64, c->sz_val32, c->sz_dinv32,
                                                   c->sz_fxy32, c->sz_ainv32);
        return launch_schwarz_t<double, double>(c, b, x, s, c->sz_val64, c->sz_val64, c->sz_dinv64, c->sz_fxy64,
                                                c->sz_ainv64);
    }
    if (mixed)
        return launch_pipe_t<float>(c, b, x, s, c->Kc32, c->dinvK32, c->pipe_c.blocks, c->pipe_c.threads,
                                    c->pipe_smem32);
    return launch_pipe_t<double>(c, b, x, s, c->Kc, c->dinvK, c->pipe_c.blocks, c->pipe_c.threads, c->pipe_smem64);
}

}  // namespace cgp
