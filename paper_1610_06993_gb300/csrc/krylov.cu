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

namespace cgp {

namespace {

// y = A x over the block's rows, `lanes` consecutive threads per row. emit(row, acc0, acc1) runs
// on the first lane of each row group. Every thread of the block runs the same number of passes
// so the group shuffles always see full warps.
template <int NR, typename TV, typename TX, typename Emit>
__device__ __forceinline__ void spmv_block(RowRange rr, const int* __restrict__ rp, const int* __restrict__ ci,
                                           const TV* __restrict__ val, const TX* x, int lanes, Emit emit) {
    const int groups = blockDim.x / lanes;
    const int g = threadIdx.x / lanes;
    const int l = threadIdx.x & (lanes - 1);
    for (int base = rr.r0; base < rr.r1; base += groups) {
        const int row = base + g;
        TX a0 = 0, a1 = 0;
        if (row < rr.r1) {
            const int k1 = __ldg(rp + row + 1);
            for (int k = __ldg(rp + row) + l; k < k1; k += lanes) {
                const int j = __ldg(ci + k);
                const TX v = (TX)__ldg(val + k);
                if (NR == 1) {
                    a0 += v * x[j];
                } else {
                    TX x0, x1;
                    load2(x, j, x0, x1);
                    a0 += v * x0;
                    a1 += v * x1;
                }
            }
        }
        a0 = group_sum(a0, lanes);
        if (NR == 2) a1 = group_sum(a1, lanes);
        if (l == 0 && row < rr.r1) emit(row, a0, a1);
    }
}

__device__ __forceinline__ bool bad(double v) { return !(fabs(v) <= 1.7976931348623157e308); }

// ------------------------------------------------------------------------------------------
// CG (Chronopoulos-Gear) inside FP64 iterative refinement
// ------------------------------------------------------------------------------------------
template <typename TI>
struct CgArgs {
    int n;
    const int* rp;
    const int* ci;
    const double* val64;
    const TI* valI;
    const TI* dinvI;      // [n]
    const double* b;      // [n][NR]
    double* x;            // [n][NR] initial guess in, solution out
    TI *r, *u, *w, *p, *s, *d;
    double* part;         // [32][nblocks]
    SyncWords* sw;
    double rtol, inner_rtol;
    int max_iter, max_outer, lanes;
    int* st_iters;
    int* st_outer;
    int* st_status;
    double* st_rel;
    int* st_barrier;
};

// partial-sum regions (units of nblocks doubles)
enum { CG_P0 = 0, CG_O1 = 2, CG_I0 = 8, CG_I1 = 10 /* two buffers of 4 */, CG_I2 = 18 };

template <typename TI, int NR>
__global__ void __launch_bounds__(1024) k_cg(CgArgs<TI> a) {
    __shared__ double s_red[32 * 8];
    __shared__ double s_bc[8];
    const unsigned int nb = gridDim.x;
    unsigned int epoch = 0;
    const RowRange rr = block_rows(a.n);
    const int tpb = blockDim.x;
    double bb[NR], rr64[NR];
    int iters = 0, outer = 0, status = CGP_OK;
#pragma unroll
    for (int c = 0; c < NR; ++c) rr64[c] = 0.0;

    // ||b||^2 per right-hand side; a zero right-hand side has the zero solution
    {
        double v[NR];
#pragma unroll
        for (int c = 0; c < NR; ++c) v[c] = 0.0;
        for (int i = rr.r0 + threadIdx.x; i < rr.r1; i += tpb)
#pragma unroll
            for (int c = 0; c < NR; ++c) {
                const double bi = a.b[(size_t)i * NR + c];
                v[c] += bi * bi;
            }
        block_partials<NR>(v, a.part + CG_P0 * nb, nb, s_red);
        if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
        grid_totals<NR>(a.part + CG_P0 * nb, nb, bb, s_bc);
        bool any_zero = false;
#pragma unroll
        for (int c = 0; c < NR; ++c) any_zero |= (bb[c] == 0.0);
        if (any_zero) {
            for (int i = rr.r0 + threadIdx.x; i < rr.r1; i += tpb)
#pragma unroll
                for (int c = 0; c < NR; ++c)
                    if (bb[c] == 0.0) a.x[(size_t)i * NR + c] = 0.0;
            if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
        }
    }
    const double rtol2 = a.rtol * a.rtol, itol2 = a.inner_rtol * a.inner_rtol;
    const double floor2 = 0.25 * rtol2;

    for (;;) {
        // ---- refinement pass: FP64 true residual, inner start r = (TI) r64, u = D^-1 r, d = 0
        double t1[3 * NR];
        {
            double v[3 * NR];
#pragma unroll
            for (int k = 0; k < 3 * NR; ++k) v[k] = 0.0;
            spmv_block<NR, double, double>(rr, a.rp, a.ci, a.val64, a.x, a.lanes, [&](int i, double s0, double s1) {
                const double acc[2] = {s0, s1};
                const TI di = a.dinvI[i];
#pragma unroll
                for (int c = 0; c < NR; ++c) {
                    const size_t idx = (size_t)i * NR + c;
                    const double ri = a.b[idx] - acc[c];
                    v[c] += ri * ri;
                    const TI rI = (TI)ri, uI = di * rI;
                    a.r[idx] = rI;
                    a.u[idx] = uI;
                    a.d[idx] = (TI)0;
                    v[NR + c] += (double)(rI * uI);
                }
            });
            block_partials<3 * NR>(v, a.part + CG_O1 * nb, nb, s_red);
            if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
            grid_totals<3 * NR>(a.part + CG_O1 * nb, nb, t1, s_bc);
        }
        bool act[NR], any = false, nan = false;
        double tgt[NR], gam[NR], alpha[NR], beta[NR];
#pragma unroll
        for (int c = 0; c < NR; ++c) {
            rr64[c] = t1[c];
            nan |= bad(t1[c]) | bad(t1[NR + c]);
            act[c] = !(bb[c] == 0.0 || rr64[c] <= rtol2 * bb[c]);
            any |= act[c];
            tgt[c] = fmax(itol2 * rr64[c], floor2 * bb[c]);
            gam[c] = t1[NR + c];
        }
        if (nan) { status = CGP_ERR_NAN; break; }
        if (!any) break;
        if (outer >= a.max_outer || iters >= a.max_iter) { status = CGP_ERR_NOT_CONVERGED; break; }

        // ---- w = A u, delta = (w, u); alpha_0 = gamma_0 / delta_0
        {
            double v[NR], t0[NR];
#pragma unroll
            for (int c = 0; c < NR; ++c) v[c] = 0.0;
            spmv_block<NR, TI, TI>(rr, a.rp, a.ci, a.valI, a.u, a.lanes, [&](int i, TI s0, TI s1) {
                const TI acc[2] = {s0, s1};
#pragma unroll
                for (int c = 0; c < NR; ++c) {
                    const size_t idx = (size_t)i * NR + c;
                    a.w[idx] = acc[c];
                    v[c] += (double)(acc[c] * a.u[idx]);
                }
            });
            block_partials<NR>(v, a.part + CG_I0 * nb, nb, s_red);
            if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
            grid_totals<NR>(a.part + CG_I0 * nb, nb, t0, s_bc);
#pragma unroll
            for (int c = 0; c < NR; ++c) {
                if (act[c] && t0[c] != 0.0 && !bad(t0[c])) {
                    alpha[c] = gam[c] / t0[c];
                } else {
                    act[c] = false;
                    alpha[c] = 0.0;
                }
                beta[c] = 0.0;
            }
        }
        bool first = true;
        for (;;) {
            // ---- local update: p = u + beta p, s = w + beta s, d += alpha p, r -= alpha s, u = D^-1 r
            {
                TI vg[NR], vr[NR];
#pragma unroll
                for (int c = 0; c < NR; ++c) vg[c] = vr[c] = (TI)0;
                TI al[NR], be[NR];
#pragma unroll
                for (int c = 0; c < NR; ++c) {
                    al[c] = (TI)alpha[c];
                    be[c] = (TI)beta[c];
                }
                for (int i = rr.r0 + threadIdx.x; i < rr.r1; i += tpb) {
                    const TI di = a.dinvI[i];
#pragma unroll
                    for (int c = 0; c < NR; ++c) {
                        const size_t idx = (size_t)i * NR + c;
                        const TI uo = a.u[idx], wo = a.w[idx];
                        const TI p = first ? uo : uo + be[c] * a.p[idx];
                        const TI s = first ? wo : wo + be[c] * a.s[idx];
                        a.p[idx] = p;
                        a.s[idx] = s;
                        a.d[idx] += al[c] * p;
                        const TI r = a.r[idx] - al[c] * s;
                        a.r[idx] = r;
                        const TI u = di * r;
                        a.u[idx] = u;
                        vg[c] += r * u;
                        vr[c] += r * r;
                    }
                }
                double v[2 * NR];
#pragma unroll
                for (int c = 0; c < NR; ++c) {
                    v[c] = (double)vg[c];
                    v[NR + c] = (double)vr[c];
                }
                block_partials<2 * NR>(v, a.part + (CG_I1 + 4 * (iters & 1)) * nb, nb, s_red);
                if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
            }
            // ---- w = A u, delta = (w, u)
            double tg[2 * NR], td[NR];
            {
                TI vv[NR];
#pragma unroll
                for (int c = 0; c < NR; ++c) vv[c] = (TI)0;
                spmv_block<NR, TI, TI>(rr, a.rp, a.ci, a.valI, a.u, a.lanes, [&](int i, TI s0, TI s1) {
                    const TI acc[2] = {s0, s1};
#pragma unroll
                    for (int c = 0; c < NR; ++c) {
                        const size_t idx = (size_t)i * NR + c;
                        a.w[idx] = acc[c];
                        vv[c] += acc[c] * a.u[idx];
                    }
                });
                double v[NR];
#pragma unroll
                for (int c = 0; c < NR; ++c) v[c] = (double)vv[c];
                block_partials<NR>(v, a.part + CG_I2 * nb, nb, s_red);
                if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
                int slot[3 * NR];
                double t3[3 * NR];
#pragma unroll
                for (int k = 0; k < 2 * NR; ++k) slot[k] = CG_I1 + 4 * (iters & 1) + k;
#pragma unroll
                for (int k = 0; k < NR; ++k) slot[2 * NR + k] = CG_I2 + k;
                grid_totals_at<3 * NR>(a.part, slot, nb, t3, s_bc);
#pragma unroll
                for (int k = 0; k < 2 * NR; ++k) tg[k] = t3[k];
#pragma unroll
                for (int k = 0; k < NR; ++k) td[k] = t3[2 * NR + k];
            }
            iters += 1;
            first = false;
            bool more = false;
#pragma unroll
            for (int c = 0; c < NR; ++c) {
                nan |= bad(tg[c]) | bad(tg[NR + c]) | bad(td[c]);
                if (act[c] && tg[NR + c] <= tgt[c]) act[c] = false;
                if (act[c]) {
                    const double gnew = tg[c];
                    const double bnew = gnew / gam[c];
                    const double den = td[c] - bnew * gnew / alpha[c];
                    if (den != 0.0 && gam[c] != 0.0) {
                        beta[c] = bnew;
                        alpha[c] = gnew / den;
                        gam[c] = gnew;
                    } else {
                        act[c] = false;
                    }
                }
                if (!act[c]) alpha[c] = beta[c] = 0.0;
                more |= act[c];
            }
            if (nan || !more || iters >= a.max_iter) break;
        }
        if (nan) { status = CGP_ERR_NAN; break; }
        // ---- x += d (FP64)
        for (int i = rr.r0 + threadIdx.x; i < rr.r1; i += tpb)
#pragma unroll
            for (int c = 0; c < NR; ++c) {
                const size_t idx = (size_t)i * NR + c;
                a.x[idx] += (double)a.d[idx];
            }
        if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
        outer += 1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double rel = 0.0;
#pragma unroll
        for (int c = 0; c < NR; ++c)
            if (bb[c] > 0.0) rel = fmax(rel, sqrt(rr64[c] / bb[c]));
        *a.st_iters = iters;
        *a.st_outer = outer;
        *a.st_status = status;
        *a.st_rel = rel;
    }
}

// ------------------------------------------------------------------------------------------
// BiCGStab, two right-hand sides, identity rows at Dirichlet nodes, inside FP64 refinement
// ------------------------------------------------------------------------------------------
template <typename TI>
struct BicgArgs {
    int n;
    const int* rp;
    const int* ci;
    const double* val64;
    const TI* valI;
    const TI* dinvI;              // [n][2]
    const unsigned char* mask;    // CGP_BC_U / CGP_BC_V per node
    const int* diag;              // [n] CSR slot of the diagonal
    const double* g;              // [n][2] prescribed values
    const double* b;              // [n][2]
    const double* x_in;           // [n][2] initial guess (Dirichlet entries are replaced by g)
    double* x;                    // [n][2] solution
    TI *r, *rh, *p, *v, *y, *s, *z, *t, *d;
    double* part;
    SyncWords* sw;
    double rtol, inner_rtol;
    int max_iter, max_outer, lanes;
    int* st_iters;
    int* st_outer;
    int* st_status;
    double* st_rel;
    int* st_barrier;
};

enum { BI_P0 = 0, BI_O1 = 2, BI_B2 = 6, BI_B3 = 8, BI_B4 = 10, BI_B5 = 14 };

template <typename TI>
__global__ void __launch_bounds__(1024) k_bicgstab(BicgArgs<TI> a) {
    __shared__ double s_red[32 * 8];
    __shared__ double s_bc[8];
    const unsigned int nb = gridDim.x;
    unsigned int epoch = 0;
    const RowRange rr = block_rows(a.n);
    const int tpb = blockDim.x;
    double bb[2], rr64[2] = {0.0, 0.0};
    int iters = 0, outer = 0, status = CGP_OK;

    // initial guess with prescribed values, ||b||^2
    {
        double v[2] = {0.0, 0.0};
        for (int i = rr.r0 + threadIdx.x; i < rr.r1; i += tpb) {
            const unsigned char m = a.mask[i];
            double x0, x1, g0, g1, b0, b1;
            load2(a.x_in, i, x0, x1);
            load2(a.g, i, g0, g1);
            store2(a.x, i, (m & CGP_BC_U) ? g0 : x0, (m & CGP_BC_V) ? g1 : x1);
            load2(a.b, i, b0, b1);
            // ||b|| of the row-scaled system: a Dirichlet row counts as A_ii x_i = A_ii g_i, so
            // O(1) boundary values do not swamp the O(h^2) interior right-hand side. Those rows
            // hold x_i = g_i exactly and never carry residual.
            if (m) {
                const double aii = a.val64[a.diag[i]];
                if (m & CGP_BC_U) b0 *= aii;
                if (m & CGP_BC_V) b1 *= aii;
            }
            v[0] += b0 * b0;
            v[1] += b1 * b1;
        }
        block_partials<2>(v, a.part + BI_P0 * nb, nb, s_red);
        if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
        grid_totals<2>(a.part + BI_P0 * nb, nb, bb, s_bc);
        if (bb[0] == 0.0 || bb[1] == 0.0) {
            for (int i = rr.r0 + threadIdx.x; i < rr.r1; i += tpb)
                for (int c = 0; c < 2; ++c)
                    if (bb[c] == 0.0) a.x[2 * (size_t)i + c] = 0.0;
            if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
        }
    }
    const double rtol2 = a.rtol * a.rtol, itol2 = a.inner_rtol * a.inner_rtol;
    const double floor2 = 0.25 * rtol2;
    auto masked = [&](int i, int c, TI acc, const TI* src) -> TI {
        return (a.mask[i] & (1 << c)) ? src[2 * (size_t)i + c] : acc;
    };

    for (;;) {
        double t1[4];
        {
            double v[4] = {0.0, 0.0, 0.0, 0.0};
            spmv_block<2, double, double>(rr, a.rp, a.ci, a.val64, a.x, a.lanes, [&](int i, double s0, double s1) {
                const double acc[2] = {s0, s1};
                const unsigned char m = a.mask[i];
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const size_t idx = 2 * (size_t)i + c;
                    const double ax = (m & (1 << c)) ? a.x[idx] : acc[c];
                    const double ri = a.b[idx] - ax;
                    v[c] += ri * ri;
                    const TI rI = (TI)ri;
                    a.r[idx] = rI;
                    a.rh[idx] = rI;
                    a.d[idx] = (TI)0;
                    v[2 + c] += (double)(rI * rI);
                }
            });
            block_partials<4>(v, a.part + BI_O1 * nb, nb, s_red);
            if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
            grid_totals<4>(a.part + BI_O1 * nb, nb, t1, s_bc);
        }
        bool act[2], any = false, nan = false;
        double tgt[2], rho[2], alpha[2] = {0.0, 0.0}, omega[2] = {0.0, 0.0}, beta[2] = {0.0, 0.0};
        for (int c = 0; c < 2; ++c) {
            rr64[c] = t1[c];
            nan |= bad(t1[c]) | bad(t1[2 + c]);
            act[c] = !(bb[c] == 0.0 || rr64[c] <= rtol2 * bb[c]);
            any |= act[c];
            tgt[c] = fmax(itol2 * rr64[c], floor2 * bb[c]);
            rho[c] = t1[2 + c];
        }
        if (nan) { status = CGP_ERR_NAN; break; }
        if (!any) break;
        if (outer >= a.max_outer || iters >= a.max_iter) { status = CGP_ERR_NOT_CONVERGED; break; }

        bool first = true;
        for (;;) {
            TI al[2], om[2], be[2];
            // ---- p = r + beta (p - omega v), y = D^-1 p
            for (int c = 0; c < 2; ++c) {
                om[c] = (TI)omega[c];
                be[c] = (TI)beta[c];
            }
            for (int i = rr.r0 + threadIdx.x; i < rr.r1; i += tpb) {
                TI d0, d1;
                load2(a.dinvI, i, d0, d1);
                const TI dd[2] = {d0, d1};
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const size_t idx = 2 * (size_t)i + c;
                    const TI r = a.r[idx];
                    const TI p = first ? r : r + be[c] * (a.p[idx] - om[c] * a.v[idx]);
                    a.p[idx] = p;
                    a.y[idx] = dd[c] * p;
                }
            }
            if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
            // ---- v = A y, sigma = (rh, v)
            {
                TI vs[2] = {(TI)0, (TI)0};
                spmv_block<2, TI, TI>(rr, a.rp, a.ci, a.valI, a.y, a.lanes, [&](int i, TI s0, TI s1) {
                    const TI acc[2] = {s0, s1};
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const size_t idx = 2 * (size_t)i + c;
                        const TI vv = masked(i, c, acc[c], a.y);
                        a.v[idx] = vv;
                        vs[c] += a.rh[idx] * vv;
                    }
                });
                double v[2] = {(double)vs[0], (double)vs[1]}, ts[2];
                block_partials<2>(v, a.part + BI_B2 * nb, nb, s_red);
                if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
                grid_totals<2>(a.part + BI_B2 * nb, nb, ts, s_bc);
                for (int c = 0; c < 2; ++c) {
                    nan |= bad(ts[c]);
                    if (act[c] && ts[c] != 0.0) alpha[c] = rho[c] / ts[c];
                    else { act[c] = false; alpha[c] = 0.0; }
                    al[c] = (TI)alpha[c];
                }
            }
            // ---- s = r - alpha v, z = D^-1 s, d += alpha y, (s, s)
            {
                TI vs[2] = {(TI)0, (TI)0};
                for (int i = rr.r0 + threadIdx.x; i < rr.r1; i += tpb) {
                    TI d0, d1;
                    load2(a.dinvI, i, d0, d1);
                    const TI dd[2] = {d0, d1};
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const size_t idx = 2 * (size_t)i + c;
                        const TI s = a.r[idx] - al[c] * a.v[idx];
                        a.s[idx] = s;
                        a.z[idx] = dd[c] * s;
                        a.d[idx] += al[c] * a.y[idx];
                        vs[c] += s * s;
                    }
                }
                double v[2] = {(double)vs[0], (double)vs[1]};
                block_partials<2>(v, a.part + BI_B3 * nb, nb, s_red);
                if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
            }
            // ---- t = A z, omega = (t, s) / (t, t)
            {
                TI vts[2] = {(TI)0, (TI)0}, vtt[2] = {(TI)0, (TI)0};
                spmv_block<2, TI, TI>(rr, a.rp, a.ci, a.valI, a.z, a.lanes, [&](int i, TI s0, TI s1) {
                    const TI acc[2] = {s0, s1};
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const size_t idx = 2 * (size_t)i + c;
                        const TI tv = masked(i, c, acc[c], a.z);
                        a.t[idx] = tv;
                        vts[c] += tv * a.s[idx];
                        vtt[c] += tv * tv;
                    }
                });
                double v[4] = {(double)vts[0], (double)vts[1], (double)vtt[0], (double)vtt[1]}, t4[4], tss[2];
                block_partials<4>(v, a.part + BI_B4 * nb, nb, s_red);
                if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
                {
                    const int slot[6] = {BI_B4, BI_B4 + 1, BI_B4 + 2, BI_B4 + 3, BI_B3, BI_B3 + 1};
                    double t6[6];
                    grid_totals_at<6>(a.part, slot, nb, t6, s_bc);
                    for (int k = 0; k < 4; ++k) t4[k] = t6[k];
                    tss[0] = t6[4];
                    tss[1] = t6[5];
                }
                for (int c = 0; c < 2; ++c) {
                    nan |= bad(t4[c]) | bad(t4[2 + c]) | bad(tss[c]);
                    if (act[c] && tss[c] <= tgt[c]) {          // converged at the half step
                        act[c] = false;
                        omega[c] = 0.0;
                    } else if (act[c] && t4[2 + c] != 0.0) {
                        omega[c] = t4[c] / t4[2 + c];
                    } else {
                        act[c] = false;
                        omega[c] = 0.0;
                    }
                    om[c] = (TI)omega[c];
                }
            }
            // ---- d += omega z, r = s - omega t, rho' = (rh, r), (r, r)
            {
                TI vr[2] = {(TI)0, (TI)0}, vq[2] = {(TI)0, (TI)0};
                for (int i = rr.r0 + threadIdx.x; i < rr.r1; i += tpb) {
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const size_t idx = 2 * (size_t)i + c;
                        a.d[idx] += om[c] * a.z[idx];
                        const TI r = a.s[idx] - om[c] * a.t[idx];
                        a.r[idx] = r;
                        vr[c] += a.rh[idx] * r;
                        vq[c] += r * r;
                    }
                }
                double v[4] = {(double)vr[0], (double)vr[1], (double)vq[0], (double)vq[1]}, t5[4];
                block_partials<4>(v, a.part + BI_B5 * nb, nb, s_red);
                if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
                grid_totals<4>(a.part + BI_B5 * nb, nb, t5, s_bc);
                iters += 1;
                first = false;
                bool more = false;
                for (int c = 0; c < 2; ++c) {
                    nan |= bad(t5[c]) | bad(t5[2 + c]);
                    if (act[c] && t5[2 + c] <= tgt[c]) act[c] = false;
                    if (act[c]) {
                        if (t5[c] != 0.0 && omega[c] != 0.0 && rho[c] != 0.0) {
                            beta[c] = (t5[c] / rho[c]) * (alpha[c] / omega[c]);
                            rho[c] = t5[c];
                        } else {
                            act[c] = false;            // breakdown: restart in the next pass
                        }
                    }
                    if (!act[c]) beta[c] = 0.0;
                    more |= act[c];
                }
                if (nan || !more || iters >= a.max_iter) break;
            }
        }
        if (nan) { status = CGP_ERR_NAN; break; }
        for (int i = rr.r0 + threadIdx.x; i < rr.r1; i += tpb)
            for (int c = 0; c < 2; ++c) a.x[2 * (size_t)i + c] += (double)a.d[2 * (size_t)i + c];
        if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
        outer += 1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double rel = 0.0;
        for (int c = 0; c < 2; ++c)
            if (bb[c] > 0.0) rel = fmax(rel, sqrt(rr64[c] / bb[c]));
        *a.st_iters = iters;
        *a.st_outer = outer;
        *a.st_status = status;
        *a.st_rel = rel;
    }
}

// Stand-alone SpMV used by the autotuner: y = A x over all rows, one row slice per block.
template <int NR>
__global__ void __launch_bounds__(1024) k_spmv_probe(int n, const int* rp, const int* ci, const double* val,
                                                     const double* x, double* y, int lanes, int rows_per_block) {
    RowRange rr;
    rr.r0 = min(n, blockIdx.x * rows_per_block);
    rr.r1 = min(n, rr.r0 + rows_per_block);
    spmv_block<NR, double, double>(rr, rp, ci, val, x, lanes, [&](int i, double s0, double s1) {
        if (NR == 1) y[i] = s0;
        else store2(y, i, s0, s1);
    });
}

template <typename T>
T* carve(char*& p, size_t count) {
    T* r = reinterpret_cast<T*>(p);
    p += ((count * sizeof(T) + 255) / 256) * 256;
    return r;
}

}  // namespace

cudaError_t launch_poisson_cg(cgp_ctx_s* c, const double* b, double* x, cudaStream_t s) {
    if (c->use_pipe) return launch_poisson_pipe(c, b, x, s);
    SyncWords* sw = c->sync + SYNC_POI;
    cudaError_t e = cudaMemsetAsync(sw, 0, sizeof(SyncWords), s);
    if (e != cudaSuccess) return e;
    const bool mixed = c->prm.precision == CGP_MIXED;
    const int n = c->nc;
    char* p = (char*)c->ws;
    if (mixed) {
        CgArgs<float> a;
        a.n = n; a.rp = c->C.rp; a.ci = c->C.ci; a.val64 = c->Kc; a.valI = c->Kc32; a.dinvI = c->dinvK32;
        a.b = b; a.x = x;
        a.r = carve<float>(p, n); a.u = carve<float>(p, n); a.w = carve<float>(p, n);
        a.p = carve<float>(p, n); a.s = carve<float>(p, n); a.d = carve<float>(p, n);
        a.part = c->part; a.sw = sw; a.rtol = c->prm.rtol; a.inner_rtol = c->prm.inner_rtol;
        a.max_iter = c->prm.max_iter; a.max_outer = c->prm.max_outer; a.lanes = c->sh_c.lanes;
        a.st_iters = &c->stats->poi_iters; a.st_outer = &c->stats->poi_outer; a.st_status = &c->stats->poi_status;
        a.st_rel = &c->stats->poi_rel; a.st_barrier = &c->stats->barrier_status;
        return coop_launch((const void*)k_cg<float, 1>, c->sh_c.blocks, c->sh_c.threads, a, s);
    }
    CgArgs<double> a;
    a.n = n; a.rp = c->C.rp; a.ci = c->C.ci; a.val64 = c->Kc; a.valI = c->Kc; a.dinvI = c->dinvK;
    a.b = b; a.x = x;
    a.r = carve<double>(p, n); a.u = carve<double>(p, n); a.w = carve<double>(p, n);
    a.p = carve<double>(p, n); a.s = carve<double>(p, n); a.d = carve<double>(p, n);
    a.part = c->part; a.sw = sw; a.rtol = c->prm.rtol; a.inner_rtol = 0.0;
    a.max_iter = c->prm.max_iter; a.max_outer = c->prm.max_outer; a.lanes = c->sh_c.lanes;
    a.st_iters = &c->stats->poi_iters; a.st_outer = &c->stats->poi_outer; a.st_status = &c->stats->poi_status;
    a.st_rel = &c->stats->poi_rel; a.st_barrier = &c->stats->barrier_status;
    return coop_launch((const void*)k_cg<double, 1>, c->sh_c.blocks, c->sh_c.threads, a, s);
}

cudaError_t launch_mass_cg(cgp_ctx_s* c, const double* b, double* x, cudaStream_t s) {
    SyncWords* sw = c->sync + SYNC_MASS;
    cudaError_t e = cudaMemsetAsync(sw, 0, sizeof(SyncWords), s);
    if (e != cudaSuccess) return e;
    const int n = c->nf;
    char* p = (char*)c->ws;
    CgArgs<double> a;
    a.n = n; a.rp = c->F.rp; a.ci = c->F.ci; a.val64 = c->M; a.valI = c->M; a.dinvI = c->dinvM;
    a.b = b; a.x = x;
    a.r = carve<double>(p, 2 * (size_t)n); a.u = carve<double>(p, 2 * (size_t)n); a.w = carve<double>(p, 2 * (size_t)n);
    a.p = carve<double>(p, 2 * (size_t)n); a.s = carve<double>(p, 2 * (size_t)n); a.d = carve<double>(p, 2 * (size_t)n);
    a.part = c->part; a.sw = sw; a.rtol = c->prm.rtol; a.inner_rtol = 0.0;
    a.max_iter = c->prm.max_iter; a.max_outer = c->prm.max_outer; a.lanes = c->sh_f.lanes;
    a.st_iters = &c->stats->mass_iters; a.st_outer = &c->stats->mass_outer; a.st_status = &c->stats->mass_status;
    a.st_rel = &c->stats->mass_rel; a.st_barrier = &c->stats->barrier_status;
    return coop_launch((const void*)k_cg<double, 2>, c->sh_f.blocks, c->sh_f.threads, a, s);
}

cudaError_t launch_momentum_bicgstab(cgp_ctx_s* c, const double* u_in, double* x, cudaStream_t s) {
    SyncWords* sw = c->sync + SYNC_MOM;
    cudaError_t e = cudaMemsetAsync(sw, 0, sizeof(SyncWords), s);
    if (e != cudaSuccess) return e;
    const bool mixed = c->prm.precision == CGP_MIXED;
    const size_t n2 = 2 * (size_t)c->nf;
    char* p = (char*)c->ws;
    if (mixed) {
        BicgArgs<float> a;
        a.n = c->nf; a.rp = c->F.rp; a.ci = c->F.ci; a.val64 = c->A; a.valI = c->A32; a.dinvI = c->dinvA32;
        a.mask = c->vel_mask; a.diag = c->F.diag; a.g = c->g; a.b = c->b_mom; a.x_in = u_in; a.x = x;
        a.r = carve<float>(p, n2); a.rh = carve<float>(p, n2); a.p = carve<float>(p, n2);
        a.v = carve<float>(p, n2); a.y = carve<float>(p, n2); a.s = carve<float>(p, n2);
        a.z = carve<float>(p, n2); a.t = carve<float>(p, n2); a.d = carve<float>(p, n2);
        a.part = c->part; a.sw = sw; a.rtol = c->prm.rtol; a.inner_rtol = c->prm.inner_rtol;
        a.max_iter = c->prm.max_iter; a.max_outer = c->prm.max_outer; a.lanes = c->sh_f.lanes;
        a.st_iters = &c->stats->mom_iters; a.st_outer = &c->stats->mom_outer; a.st_status = &c->stats->mom_status;
        a.st_rel = &c->stats->mom_rel; a.st_barrier = &c->stats->barrier_status;
        return coop_launch((const void*)k_bicgstab<float>, c->sh_f.blocks, c->sh_f.threads, a, s);
    }
    BicgArgs<double> a;
    a.n = c->nf; a.rp = c->F.rp; a.ci = c->F.ci; a.val64 = c->A; a.valI = c->A; a.dinvI = c->dinvA;
    a.mask = c->vel_mask; a.diag = c->F.diag; a.g = c->g; a.b = c->b_mom; a.x_in = u_in; a.x = x;
    a.r = carve<double>(p, n2); a.rh = carve<double>(p, n2); a.p = carve<double>(p, n2);
    a.v = carve<double>(p, n2); a.y = carve<double>(p, n2); a.s = carve<double>(p, n2);
    a.z = carve<double>(p, n2); a.t = carve<double>(p, n2); a.d = carve<double>(p, n2);
    a.part = c->part; a.sw = sw; a.rtol = c->prm.rtol; a.inner_rtol = 0.0;
    a.max_iter = c->prm.max_iter; a.max_outer = c->prm.max_outer; a.lanes = c->sh_f.lanes;
    a.st_iters = &c->stats->mom_iters; a.st_outer = &c->stats->mom_outer; a.st_status = &c->stats->mom_status;
    a.st_rel = &c->stats->mom_rel; a.st_barrier = &c->stats->barrier_status;
    return coop_launch((const void*)k_bicgstab<double>, c->sh_f.blocks, c->sh_f.threads, a, s);
}

// Occupancy of the persistent kernels (blocks per SM at `threads`), the minimum over the family.
int persistent_blocks_per_sm(int threads) {
    int m = 1 << 30, v = 0;
    const void* fns[] = {(const void*)k_cg<double, 1>, (const void*)k_cg<float, 1>, (const void*)k_cg<double, 2>,
                         (const void*)k_bicgstab<double>, (const void*)k_bicgstab<float>};
    for (const void* f : fns) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, f, threads, 0) != cudaSuccess) return 0;
        m = v < m ? v : m;
    }
    return m;
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

// All scratch of cgp_cg_solve_noalloc: seven vectors of NOALLOC_MAX_ROWS doubles (r, u, w, p,
// s, d and the inverse diagonal), the per-block partial sums, the grid-barrier words and a
// statistics record. About 3.6 MB, held by every device that loads the library until exit.
__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

struct NoallocStats {
    int iters, outer, status, barrier;
    double rel;
};

struct NoallocDevice {
    bool ready = false;
    unsigned char* base = nullptr;   // device address of g_noalloc_scratch on this device
    int num_sms = 0;
};
std::mutex g_noalloc_mu;
NoallocDevice g_noalloc_dev[64];

__global__ void k_noalloc_dinv(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                               const double* __restrict__ val, double* dinv) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double d = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k)
        if (ci[k] == i) d = val[k];
    dinv[i] = 1.0 / d;
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
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)k_cg<double, 1>, 512, 0) !=
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
    if (status_dev && cudaMemsetAsync(status_dev, 0, sizeof(int), s) != cudaSuccess) return CGP_ERR_CUDA;
    k_noalloc_dinv<<<(n + 255) / 256, 256, 0, s>>>(n, rp_dev, ci_dev, val_dev, vec[6]);
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
    a.max_outer = 30;
    a.lanes = 4;
    a.st_iters = iters_dev ? iters_dev : &st->iters;
    a.st_outer = &st->outer;
    a.st_status = status_dev ? status_dev : &st->status;
    a.st_rel = rel_res_dev ? rel_res_dev : &st->rel;
    a.st_barrier = status_dev ? status_dev : &st->barrier;
    const int threads = 512;
    int blocks = (n + threads - 1) / threads;
    blocks = std::max(1, std::min(std::min(blocks, nd->num_sms), CGP_MAX_GRID));
    cudaError_t e = coop_launch((const void*)k_cg<double, 1>, blocks, threads, a, s);
    return e == cudaSuccess ? CGP_OK : CGP_ERR_CUDA;
}
