// Persistent Krylov kernels of the CGP step, shared by the single-instance launchers
// (krylov.cu) and the batched multi-instance step (batch.cu). See krylov.cu for the method.
#pragma once
#include "ctx.h"

#ifndef CGP_ROWS_F32
#define CGP_ROWS_F32 2        // rows in flight per thread in the FP32 CSR product (4 measured no faster)
#endif
#ifndef CGP_ELL_CHUNK_F32
#define CGP_ELL_CHUNK_F32 4   // slots per load group of the FP32 sliced-ELL product
#endif

namespace cgp {

namespace {

// CNT consecutive entries (from k) of R rows (row q starts at ka[q] and has na[q] entries): all
// column and value loads first, then the x gathers and products; entries past a row's end are
// skipped per lane. The fine-mesh products (two right-hand sides) stream their matrix with the
// evict-first hint, so that it does not push the Krylov vectors out of L2; the scalar coarse
// products keep theirs cached, since a coarse CG re-reads it every iteration (the 64-cavity
// batch's coarse matrices, 50 MB in FP32, ran 6 % slower when streamed).
template <int R, int CNT, int NR, typename TV, typename TX>
__device__ __forceinline__ void spmv_rows_chunk(int k, const int (&ka)[R], const int (&na)[R],
                                                const int* __restrict__ ci, const TV* __restrict__ val, const TX* x,
                                                TX (&acc0)[R], TX (&acc1)[R]) {
    int j[R][CNT];
    TX v[R][CNT];
#pragma unroll
    for (int q = 0; q < R; ++q)
#pragma unroll
        for (int e = 0; e < CNT; ++e) {
            const bool in = k + e < na[q];
            if (NR == 2) {
                j[q][e] = in ? __ldcs(ci + ka[q] + k + e) : -1;
                v[q][e] = in ? (TX)__ldcs(val + ka[q] + k + e) : (TX)0;
            } else {
                j[q][e] = in ? __ldg(ci + ka[q] + k + e) : -1;
                v[q][e] = in ? (TX)__ldg(val + ka[q] + k + e) : (TX)0;
            }
        }
#pragma unroll
    for (int q = 0; q < R; ++q)
#pragma unroll
        for (int e = 0; e < CNT; ++e) {
            if (j[q][e] >= 0) {
                if (NR == 1) {
                    acc0[q] += v[q][e] * x[j[q][e]];
                } else {
                    TX x0, x1;
                    load2(x, j[q][e], x0, x1);
                    acc0[q] += v[q][e] * x0;
                    acc1[q] += v[q][e] * x1;
                }
            }
        }
}

// y = A x over the block's rows with one thread per row and R rows per thread in flight: the
// block's range is cut into R equal parts and a thread takes row i of every part at once, so that
// every pass but the last has all R rows in all lanes. The entries of the R rows go CNT at a time
// (all column and value loads of a group before its x gathers), and the warp stops at its longest
// row exactly: the products of a warp issue once per entry slot that some lane needs. A product is
// bound by the dependent column -> x round trips of a thread, so R rows in flight divide their
// number by R (measured on the 1M-row cylinder mesh: four rows per thread were no faster than two;
// with perfectly coalesced x reads a product was only a fifth faster, so it is bound by the
// matrix stream at this occupancy rather than by the gathers). x is written by other blocks during
// the launch, so it is read with ordinary (coherent) loads; the fine-mesh matrices are streamed
// with the evict-first hint (on the 1M-row cylinder mesh the momentum products fell from ~44 to
// ~35 us). CGP_ROWS_F32 sets R for the single-context FP32 products, the rest take two
// (registers).
template <int NR, typename TV, typename TX, int R = 2, typename Emit>
__device__ __forceinline__ void spmv_rows(RowRange rr, const int* __restrict__ rp, const int* __restrict__ ci,
                                          const TV* __restrict__ val, const TX* x, Emit emit) {
    const int T = blockDim.x;
    const int Q = (rr.r1 - rr.r0 + R - 1) / R;
    for (int i0 = rr.r0 + threadIdx.x; i0 < rr.r0 + Q; i0 += T) {
        int ka[R], na[R];
        int mx = 0;
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int i = i0 + q * Q;
            const bool h = i < rr.r1;
            ka[q] = h ? __ldg(rp + i) : 0;
            na[q] = h ? __ldg(rp + i + 1) - ka[q] : 0;
            mx = max(mx, na[q]);
        }
        // the longest row among the lanes here; each lane's own rows are no longer than that
        const int mw = (int)__reduce_max_sync(__activemask(), (unsigned)mx);
        TX a0[R], a1[R];
#pragma unroll
        for (int q = 0; q < R; ++q) a0[q] = a1[q] = (TX)0;
        int k = 0;
        for (; k + 4 <= mw; k += 4) spmv_rows_chunk<R, 4, NR, TV, TX>(k, ka, na, ci, val, x, a0, a1);
        switch (mw - k) {
            case 3: spmv_rows_chunk<R, 3, NR, TV, TX>(k, ka, na, ci, val, x, a0, a1); break;
            case 2: spmv_rows_chunk<R, 2, NR, TV, TX>(k, ka, na, ci, val, x, a0, a1); break;
            case 1: spmv_rows_chunk<R, 1, NR, TV, TX>(k, ka, na, ci, val, x, a0, a1); break;
            default: break;
        }
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int i = i0 + q * Q;
            if (i < rr.r1) emit(i, a0[q], a1[q]);
        }
    }
}

// y = A x over the block's rows, `lanes` consecutive threads per row. emit(row, acc0, acc1) runs
// on the first lane of each row group. Every thread of the block runs the same number of passes
// so the group shuffles always see full warps. Plain loop: for kernels with many resident warps
// (the stand-alone product), where occupancy hides the latency.
template <int NR, typename TV, typename TX, typename Emit>
__device__ __forceinline__ void spmv_lanes(RowRange rr, const int* __restrict__ rp, const int* __restrict__ ci,
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

// The product of the persistent Krylov kernels (one block per SM): one lane per row takes the
// spmv_rows path, more lanes the group loop.
template <int NR, typename TV, typename TX, int R = 2, typename Emit>
__device__ __forceinline__ void spmv_block(RowRange rr, const int* __restrict__ rp, const int* __restrict__ ci,
                                           const TV* __restrict__ val, const TX* x, int lanes, Emit emit) {
    if (lanes == 1) spmv_rows<NR, TV, TX, R>(rr, rp, ci, val, x, emit);
    else spmv_lanes<NR, TV, TX>(rr, rp, ci, val, x, lanes, emit);
}

// CNT consecutive slots (from k) of two 32-row slices of the sliced-ELL layout (slot k of a slice's
// rows contiguous, so every column and value load of a warp is one coalesced access): column and
// value loads of both slices first, then the x gathers. Slice widths are warp-uniform, so the
// bounds below never diverge. pa, pb: the lane's first slot in slices a and b.
template <int CNT, int NR, typename TV, typename TX>
__device__ __forceinline__ void ell_pair_chunk(int k, int pa, int wa, int pb, int wb, const int* __restrict__ col,
                                               const TV* __restrict__ val, const TX* x, TX& a0, TX& a1, TX& b0,
                                               TX& b1) {
    int ja[CNT], jb[CNT];
    TX va[CNT], vb[CNT];
#pragma unroll
    for (int q = 0; q < CNT; ++q) {
        const int o = (k + q) << 5;
        const bool ia = k + q < wa, ib = k + q < wb;
        ja[q] = ia ? __ldcs(col + pa + o) : 0;
        va[q] = ia ? (TX)__ldcs(val + pa + o) : (TX)0;
        jb[q] = ib ? __ldcs(col + pb + o) : 0;
        vb[q] = ib ? (TX)__ldcs(val + pb + o) : (TX)0;
    }
#pragma unroll
    for (int q = 0; q < CNT; ++q) {
        if (k + q < wa) {
            if (NR == 1) {
                a0 += va[q] * x[ja[q]];
            } else {
                TX x0, x1;
                load2(x, ja[q], x0, x1);
                a0 += va[q] * x0;
                a1 += va[q] * x1;
            }
        }
        if (k + q < wb) {
            if (NR == 1) {
                b0 += vb[q] * x[jb[q]];
            } else {
                TX x0, x1;
                load2(x, jb[q], x0, x1);
                b0 += vb[q] * x0;
                b1 += vb[q] * x1;
            }
        }
    }
}

// y = A x over the block's rows in the sliced-ELL layout of the natural row order: 32-row slices,
// the slots of slice s at ptr[s] .. ptr[s + 1], slot k of its rows contiguous (padding slots hold
// a zero value and a valid column). The block's rows are whole slices (group_rows_aligned). One
// warp takes two slices at a time (the first half of the block's slices paired with the second),
// one lane per row, four slots of both slices per load group: the matrix streams in 128-byte
// (FP32, columns) or 256-byte (FP64) coalesced accesses, with the evict-first hint so the vectors
// keep their place in L2. emit(row, acc0, acc1) runs once per row.
template <int NR, typename TV, typename TX, typename Emit>
__device__ __forceinline__ void spmv_ell(RowRange rr, const int* __restrict__ ptr, const int* __restrict__ col,
                                         const TV* __restrict__ val, const TX* x, Emit emit) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int s0 = rr.r0 >> 5, s1 = (rr.r1 + 31) >> 5;
    const int half = (s1 - s0 + 1) >> 1;
    for (int sa = s0 + warp; sa < s0 + half; sa += nw) {
        const int sb = sa + half;
        const bool hb = sb < s1;
        const int qa = __ldg(ptr + sa), wa = (__ldg(ptr + sa + 1) - qa) >> 5;
        const int qb = hb ? __ldg(ptr + sb) : 0, wb = hb ? (__ldg(ptr + sb + 1) - qb) >> 5 : 0;
        const int pa = qa + lane, pb = qb + lane;
        const int mw = max(wa, wb);
        TX a0 = 0, a1 = 0, b0 = 0, b1 = 0;
        // CH slots of both slices per load group (the guards inside skip slots past a slice's
        // width, warp-uniformly); 4 measured faster than 8 on the 1M-row cylinder mesh
        constexpr int CH = sizeof(TX) == sizeof(float) ? CGP_ELL_CHUNK_F32 : 4;
        for (int k = 0; k < mw; k += CH) ell_pair_chunk<CH, NR, TV, TX>(k, pa, wa, pb, wb, col, val, x, a0, a1, b0, b1);
        const int ia = (sa << 5) + lane, ib = (sb << 5) + lane;
        if (ia < rr.r1) emit(ia, a0, a1);
        if (hb && ib < rr.r1) emit(ib, b0, b1);
    }
}

// The product of a persistent Krylov kernel on the layout it was compiled for: sliced ELL (ELL,
// the launch's eptr / ecol / eval arrays) or CSR through spmv_block. One layout per instantiation
// keeps each kernel within its register budget.
template <bool ELL, int NR, typename TV, typename TX, int R = 2, typename Emit>
__device__ __forceinline__ void spmv_sel(RowRange rr, const int* eptr, const int* ecol, const TV* eval,
                                         const int* __restrict__ rp, const int* __restrict__ ci,
                                         const TV* __restrict__ val, const TX* x, int lanes, Emit emit) {
    if constexpr (ELL) spmv_ell<NR, TV, TX>(rr, eptr, ecol, eval, x, emit);
    else spmv_block<NR, TV, TX, R>(rr, rp, ci, val, x, lanes, emit);
}

// Rows of the persistent kernels: whole 32-row slices per block with the sliced-ELL layout.
template <bool ELL>
__device__ __forceinline__ RowRange solver_rows(int n, const Grp& g) {
    if constexpr (ELL) return group_rows_aligned(n, g);
    else return group_rows(n, g);
}

__device__ __forceinline__ bool bad(double v) { return !(fabs(v) <= 1.7976931348623157e308); }

// The fine solvers' FP32 product as a launch of its own, in their shape (one block per SM, the
// same row ranges, layout and rows in flight): y = A x for two interleaved right-hand sides.
template <bool ELL>
__global__ void __launch_bounds__(512, 1) k_solver_spmv(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                                       const float* __restrict__ val, const int* eptr, const int* ecol,
                                                       const float* evalf, const float* x, float* __restrict__ y,
                                                       int lanes) {
    const Grp g{gridDim.x, blockIdx.x, 0};
    const RowRange rr = solver_rows<ELL>(n, g);
    spmv_sel<ELL, 2, float, float, CGP_ROWS_F32>(rr, eptr, ecol, evalf, rp, ci, val, x, lanes,
                                                 [&](int i, float s0, float s1) { store2(y, i, s0, s1); });
}

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
    // Chebyshev polynomial preconditioner (pdeg >= 2; else Jacobi): u = p(D^-1 A) D^-1 r for a
    // spectrum of D^-1 A inside [plmin, plmax], applied in FP32
    int pdeg = 0;
    double plmin = 0.0, plmax = 0.0;
    const float* valP = nullptr;    // FP32 matrix values and inverse diagonal
    const float* dinvP = nullptr;
    float *zc0 = nullptr, *zc1 = nullptr, *dc = nullptr;   // [n][NR] iterates (double buffered), direction
    // sliced-ELL copy of the matrix (eptr != nullptr selects it for every product): slice offsets,
    // columns, and the values matching val64, valI and valP
    const int* eptr = nullptr;
    const int* ecol = nullptr;
    const double* eval64 = nullptr;
    const TI* evalI = nullptr;
    const float* evalP = nullptr;
};

// partial-sum regions (units of nblocks doubles)
enum { CG_O1 = 2 /* 3 NR: residual norms, (r, u), ||b||^2 */, CG_I1 = 10 /* 3 NR */ };

// Dynamic shared memory of k_cg: the lean FP64 reduction buffer, 3 NR doubles per thread.
template <int NR>
constexpr size_t cg_smem(int threads) {
    return (size_t)3 * NR * threads * sizeof(double);
}

// Iteration (Chronopoulos-Gear form, two grid barriers per iteration, one of them a reduction):
//   p = u + beta p,  s = w + beta s,  d += alpha p,  r -= alpha s,  u = D^-1 r     (local)
//   publish u | barrier | w = A u; partials (r,u), (r,r), (w,u) | barrier
// With the polynomial preconditioner, u = p(D^-1 A) D^-1 r is the Chebyshev iteration on A z = r
// from z = 0 (pdeg - 1 products with the FP32 copy of A, a barrier before each), and (r, u) is
// taken in the product w = A u.
// MINB: resident blocks per SM the launch is compiled for: 1 for a single context (128 registers
// per thread, no spills), 2 for batches, whose many small block groups gain more from twice the
// threads per SM than from registers. ELL: products in the sliced-ELL layout (the launch's eptr,
// ecol and eval* arrays; rows in whole 32-row slices per block) instead of CSR.
template <typename TI, int NR, int MINB = 1, bool ELL = false>
__global__ void __launch_bounds__(512, MINB) k_cg(Launch<CgArgs<TI>> L) {
    // rows in flight per thread of the CSR products: more for FP32 in the single-context kernels
    constexpr int RP = MINB == 1 ? CGP_ROWS_F32 : 2;
    constexpr int RI = sizeof(TI) == sizeof(float) ? RP : 2;
    extern __shared__ double s_lean[];   // [3 NR][blockDim.x]
    __shared__ double s_bc[8];
    __shared__ float s_f32[32 * 3 * NR];
    __shared__ double s_sc[2 * NR];
    __shared__ int s_fl[2 * NR];
    const Grp g = group_of(L.map);
    const CgArgs<TI>& a = L.table ? L.table[g.inst] : L.single;
    const unsigned int nb = g.nb;
    unsigned int epoch = 0;
    const RowRange rr = solver_rows<ELL>(a.n, g);
    const int tpb = blockDim.x;
    double bb[NR], rr64[NR];
    int iters = 0, outer = 0, status = CGP_OK;
#pragma unroll
    for (int c = 0; c < NR; ++c) rr64[c] = 0.0;

    // ||b||^2 per right-hand side is taken in the first refinement pass's reduction (bb < 0 until
    // then); a zero right-hand side has the zero solution
#pragma unroll
    for (int c = 0; c < NR; ++c) bb[c] = -1.0;
    const double rtol2 = a.rtol * a.rtol, itol2 = a.inner_rtol * a.inner_rtol;
    const double floor2 = 0.25 * rtol2;
    const bool poly = a.pdeg >= 2;
    const float thetaP = poly ? (float)(0.5 * (a.plmax + a.plmin)) : 1.f;
    const float deltaP = poly ? (float)(0.5 * (a.plmax - a.plmin)) : 1.f;
    const float sigmaP = thetaP / deltaP;
    // Chebyshev steps 1 .. pdeg - 1 from the first iterate z_1 = D^-1 r / theta (in zc0 and dc,
    // written by the caller before a barrier); the last step writes u. Every block calls it the
    // same number of times; false if a barrier failed.
    auto poly_apply = [&]() -> bool {
        float rho = 1.f / sigmaP;
        for (int j = 1; j < a.pdeg; ++j) {
            const float* zin = (j & 1) ? a.zc0 : a.zc1;
            float* zout = (j & 1) ? a.zc1 : a.zc0;
            const bool last = j == a.pdeg - 1;
            const float rn = 1.f / (2.f * sigmaP - rho);
            const float c1 = rn * rho, c2 = 2.f * rn / deltaP;
            if (!grid_sync(a.sw, nb, epoch)) return false;
            spmv_sel<ELL, NR, float, float, RP>(rr, a.eptr, a.ecol, a.evalP, a.rp, a.ci, a.valP, zin, a.lanes, [&](int i, float s0, float s1) {
                const float acc[2] = {s0, s1};
                const float di = a.dinvP[i];
#pragma unroll
                for (int c = 0; c < NR; ++c) {
                    const size_t idx = (size_t)i * NR + c;
                    const float dn = c1 * a.dc[idx] + c2 * di * ((float)a.r[idx] - acc[c]);
                    const float zn = zin[idx] + dn;
                    if (last) {
                        a.u[idx] = (TI)zn;
                    } else {
                        a.dc[idx] = dn;
                        zout[idx] = zn;
                    }
                }
            });
            rho = rn;
        }
        return true;
    };

    for (;;) {
        // ---- refinement pass: FP64 true residual, inner start r = (TI) r64, u = D^-1 r, d = 0
        double t1[3 * NR];
        {
            double v[3 * NR];
#pragma unroll
            for (int k = 0; k < 3 * NR; ++k) v[k] = 0.0;
            spmv_sel<ELL, NR, double, double, 2>(rr, a.eptr, a.ecol, a.eval64, a.rp, a.ci, a.val64, a.x, a.lanes, [&](int i, double s0, double s1) {
                const double acc[2] = {s0, s1};
                const TI di = a.dinvI[i];
#pragma unroll
                for (int c = 0; c < NR; ++c) {
                    const size_t idx = (size_t)i * NR + c;
                    const double bi = a.b[idx];
                    const double ri = bi - acc[c];
                    v[c] += ri * ri;
                    v[2 * NR + c] += bi * bi;
                    const TI rI = (TI)ri, uI = di * rI;
                    a.r[idx] = rI;
                    a.d[idx] = (TI)0;
                    if (poly) {
                        const float z1 = a.dinvP[i] * (float)ri / thetaP;
                        a.zc0[idx] = z1;
                        a.dc[idx] = z1;
                    } else {
                        a.u[idx] = uI;
                        v[NR + c] += (double)(rI * uI);
                    }
                }
            });
            block_partials_lean<3 * NR>(v, a.part + CG_O1 * nb, nb, g.bid, s_lean);
            if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
            grid_totals<3 * NR>(a.part + CG_O1 * nb, nb, t1, s_bc);
            if (bb[0] < 0.0) {
#pragma unroll
                for (int c = 0; c < NR; ++c) bb[c] = t1[2 * NR + c];
                // zero right-hand sides: x = 0 (those components stay inactive, so no other
                // row's update reads the old values)
                for (int i = rr.r0 + threadIdx.x; i < rr.r1; i += tpb)
#pragma unroll
                    for (int c = 0; c < NR; ++c)
                        if (bb[c] == 0.0) a.x[(size_t)i * NR + c] = 0.0;
            }
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

        // ---- w = A u, delta = (w, u) (and gamma_0 = (r, u) with the polynomial); alpha_0
        {
            if (poly) {
                if (!poly_apply()) return record_failure(a.sw, a.st_barrier);
                if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
            }
            TI vv[2 * NR];
#pragma unroll
            for (int c = 0; c < 2 * NR; ++c) vv[c] = (TI)0;
            spmv_sel<ELL, NR, TI, TI, RI>(rr, a.eptr, a.ecol, a.evalI, a.rp, a.ci, a.valI, a.u, a.lanes, [&](int i, TI s0, TI s1) {
                const TI acc[2] = {s0, s1};
#pragma unroll
                for (int c = 0; c < NR; ++c) {
                    const size_t idx = (size_t)i * NR + c;
                    const TI ui = a.u[idx];
                    a.w[idx] = acc[c];
                    vv[c] += acc[c] * ui;
                    if (poly) vv[NR + c] += a.r[idx] * ui;
                }
            });
            double t0[2 * NR];
            block_partials_it<2 * NR, TI>(vv, a.part + CG_I1 * nb, nb, g.bid, s_lean, s_f32);
            if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
            grid_totals<2 * NR>(a.part + CG_I1 * nb, nb, t0, s_bc);
            if (poly) {
#pragma unroll
                for (int c = 0; c < NR; ++c) {
                    gam[c] = t0[NR + c];
                    if (bad(gam[c])) {
                        nan = true;
                        act[c] = false;
                    }
                }
            }
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
            // (two rows per thread: all loads of both rows before the first store)
            TI vg[NR], vr[NR], vd[NR];
#pragma unroll
            for (int c = 0; c < NR; ++c) vg[c] = vr[c] = vd[c] = (TI)0;
            {
                TI al[NR], be[NR];
#pragma unroll
                for (int c = 0; c < NR; ++c) {
                    al[c] = (TI)alpha[c];
                    be[c] = (TI)beta[c];
                }
                for (int i0 = rr.r0 + threadIdx.x; i0 < rr.r1; i0 += 2 * tpb) {
                    const int i1 = i0 + tpb;
                    const bool h1 = i1 < rr.r1;
                    const int row[2] = {i0, h1 ? i1 : i0};
                    TI di[2], uo[2][NR], wo[2][NR], po[2][NR], so[2][NR], dd[2][NR], ro[2][NR];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        di[h] = a.dinvI[row[h]];
#pragma unroll
                        for (int c = 0; c < NR; ++c) {
                            const size_t idx = (size_t)row[h] * NR + c;
                            uo[h][c] = a.u[idx];
                            wo[h][c] = a.w[idx];
                            po[h][c] = first ? (TI)0 : a.p[idx];
                            so[h][c] = first ? (TI)0 : a.s[idx];
                            dd[h][c] = a.d[idx];
                            ro[h][c] = a.r[idx];
                        }
                    }
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        if (h == 1 && !h1) break;
#pragma unroll
                        for (int c = 0; c < NR; ++c) {
                            const size_t idx = (size_t)row[h] * NR + c;
                            const TI p = uo[h][c] + be[c] * po[h][c];
                            const TI sv = wo[h][c] + be[c] * so[h][c];
                            a.p[idx] = p;
                            a.s[idx] = sv;
                            a.d[idx] = dd[h][c] + al[c] * p;
                            const TI r = ro[h][c] - al[c] * sv;
                            a.r[idx] = r;
                            vr[c] += r * r;
                            if (poly) {
                                const float z1 = a.dinvP[row[h]] * (float)r / thetaP;
                                a.zc0[idx] = z1;
                                a.dc[idx] = z1;
                            } else {
                                const TI u = di[h] * r;
                                a.u[idx] = u;
                                vg[c] += r * u;
                            }
                        }
                    }
                }
            }
            if (poly && !poly_apply()) return record_failure(a.sw, a.st_barrier);
            if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
            // ---- w = A u; (r, u), (r, r), (w, u) in one reduction
            spmv_sel<ELL, NR, TI, TI, RI>(rr, a.eptr, a.ecol, a.evalI, a.rp, a.ci, a.valI, a.u, a.lanes, [&](int i, TI s0, TI s1) {
                const TI acc[2] = {s0, s1};
#pragma unroll
                for (int c = 0; c < NR; ++c) {
                    const size_t idx = (size_t)i * NR + c;
                    const TI ui = a.u[idx];
                    a.w[idx] = acc[c];
                    vd[c] += acc[c] * ui;
                    if (poly) vg[c] += a.r[idx] * ui;
                }
            });
            {
                TI v[3 * NR];
#pragma unroll
                for (int c = 0; c < NR; ++c) {
                    v[c] = vg[c];
                    v[NR + c] = vr[c];
                    v[2 * NR + c] = vd[c];
                }
                block_partials_it<3 * NR, TI>(v, a.part + CG_I1 * nb, nb, g.bid, s_lean, s_f32);
                if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
                int slot[3 * NR];
#pragma unroll
                for (int k = 0; k < 3 * NR; ++k) slot[k] = CG_I1 + k;
                grid_totals_shared<3 * NR>(a.part, slot, nb, s_bc);
            }
            iters += 1;
            first = false;
            // scalar recurrences once per block, one thread per right-hand side (thread 32 c for
            // component c, carrying its recurrence state; FP64 division is slow on this GPU, and
            // the components' divisions run side by side), broadcast through shared memory
            if ((threadIdx.x & 31) == 0 && threadIdx.x < 32 * NR) {
#pragma unroll
                for (int c = 0; c < NR; ++c) {
                    if ((int)(threadIdx.x >> 5) != c) continue;
                    const double gnew = s_bc[c], rho = s_bc[NR + c], del = s_bc[2 * NR + c];
                    s_fl[c] = (bad(gnew) | bad(rho) | bad(del)) ? 1 : 0;
                    if (act[c] && rho <= tgt[c]) act[c] = false;
                    if (act[c]) {
                        // beta = gnew / gam and alpha' = gnew gam alpha / (del gam alpha - gnew^2):
                        // two independent divisions (a dependent FP64 operation costs tens of
                        // cycles on this GPU)
                        const double ga = gam[c] * alpha[c];
                        const double den = fma(del, ga, -gnew * gnew);
                        if (den != 0.0 && gam[c] != 0.0) {
                            beta[c] = gnew / gam[c];
                            alpha[c] = (gnew * ga) / den;
                            gam[c] = gnew;
                        } else {
                            act[c] = false;
                        }
                    }
                    if (!act[c]) alpha[c] = beta[c] = 0.0;
                    s_fl[NR + c] = act[c] ? 1 : 0;
                    s_sc[c] = alpha[c];
                    s_sc[NR + c] = beta[c];
                }
            }
            __syncthreads();
            bool more = false;
#pragma unroll
            for (int c = 0; c < NR; ++c) {
                alpha[c] = s_sc[c];
                beta[c] = s_sc[NR + c];
                more |= s_fl[NR + c] != 0;
                nan |= s_fl[c] != 0;
            }
            __syncthreads();   // s_sc / s_fl read by all before they are written again
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
    if (g.bid == 0 && threadIdx.x == 0) {
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
    const double* x_in;           // [n][2] u^n (Dirichlet entries of the guess are replaced by g)
    double* x;                    // [n][2] solution (x == x_in gives a zero increment)
    double* dx;                   // [n][2] increment x - x_in of the last converged solve, or nullptr
    double* dx2 = nullptr;        // [n][2] the increment before it (second-order guess), or nullptr
    int* dx_flag;                 // number of increments recorded, 0 .. 2
    // Chebyshev polynomial preconditioner (pdeg >= 2; else Jacobi): y = p(D^-1 A) D^-1 q for a
    // spectrum of D^-1 A inside [plmin, the float bound at *pbound], applied in FP32
    int pdeg = 0;
    double plmin = 0.0;
    const unsigned int* pbound = nullptr;
    const float* valP = nullptr;  // FP32 matrix values and inverse diagonal ([n][2])
    const float* dinvP = nullptr;
    float *zc0 = nullptr, *zc1 = nullptr, *dc = nullptr;   // [n][2] iterates (double buffered), direction
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
    // sliced-ELL copy of the matrix, as in CgArgs
    const int* eptr = nullptr;
    const int* ecol = nullptr;
    const double* eval64 = nullptr;
    const TI* evalI = nullptr;
    const float* evalP = nullptr;
};

enum { BI_P0 = 0, BI_O1 = 2, BI_B2 = 6, BI_B4 = 8 /* 10 slots */ };

// Dynamic shared memory of k_bicgstab: the lean FP64 reduction buffer, 10 doubles per thread.
constexpr size_t bicg_smem(int threads) { return (size_t)10 * threads * sizeof(double); }

// Iteration, per right-hand side c (four grid barriers, two of them reductions; the scalar
// recurrences run on thread 0 and are broadcast through shared memory):
//   p = r + beta (p - omega v),  y = D^-1 p                      (fused with the r update below)
//   publish y | barrier | v = A y; sigma = (rh, v) | barrier;  alpha = rho / sigma
//   s = r - alpha v,  z = D^-1 s,  d += alpha y
//   publish z | barrier | t = A z; (t, s), (t, t), (rh, t), (rh, s), (s, s) | barrier
//   omega = (t, s) / (t, t);  d += omega z,  r = s - omega t
//   rho' = (rh, s) - omega (rh, t),  (r, r) = (s, s) - 2 omega (t, s) + omega^2 (t, t)
// The next rho and ||r||^2 follow from inner products of s and t taken in the same reduction
// (exact identities for r = s - omega t), which saves the fifth barrier of the textbook form.
// With the polynomial preconditioner, y = K^-1 p and z = K^-1 s are Chebyshev iterations on
// A y = p and A z = s from zero (pdeg - 1 products with the FP32 copy of A, a barrier before
// each; identity rows at Dirichlet components).
template <typename TI, int MINB = 1, bool ELL = false>
__global__ void __launch_bounds__(512, MINB) k_bicgstab(Launch<BicgArgs<TI>> L) {
    constexpr int RP = MINB == 1 ? CGP_ROWS_F32 : 2;
    constexpr int RI = sizeof(TI) == sizeof(float) ? RP : 2;
    extern __shared__ double s_lean[];   // [10][blockDim.x]
    __shared__ double s_bc[10];
    __shared__ float s_f32[32 * 10];
    __shared__ double s_sc[4];
    __shared__ int s_fl[4];
    const Grp g = group_of(L.map);
    const BicgArgs<TI>& a = L.table ? L.table[g.inst] : L.single;
    const unsigned int nb = g.nb;
    unsigned int epoch = 0;
    const RowRange rr = solver_rows<ELL>(a.n, g);
    const int tpb = blockDim.x;
    double bb[2], rr64[2] = {0.0, 0.0};
    int iters = 0, outer = 0, status = CGP_OK;
    // Initial guess u^n + (u~^n - u^(n-1)): the last step's increment, repeated, or with dx2 its
    // linear extrapolation u^n + 2 dx^n - dx^(n-1) once two are recorded. Every block reads the
    // flag before the first grid barrier; block 0 rewrites it only after the last one.
    const int n_dx = a.dx != nullptr ? *a.dx_flag : 0;
    const bool have_dx = n_dx > 0, have_dx2 = a.dx2 != nullptr && n_dx >= 2;
    const bool poly = a.pdeg >= 2;
    float thetaP = 1.f, deltaP = 1.f;
    if (poly) {
        const float lmax = fmaxf(__uint_as_float(*a.pbound), (float)a.plmin * 1.25f);
        thetaP = 0.5f * (lmax + (float)a.plmin);
        deltaP = 0.5f * (lmax - (float)a.plmin);
    }
    const float sigmaP = thetaP / deltaP;
    // y <- K^-1 q: Chebyshev steps 1 .. pdeg - 1 from the first iterate D^-1 q / theta (in zc0 and
    // dc, written by the caller before a barrier); the last step writes y. Every block calls it
    // the same number of times; false if a barrier failed.
    auto poly_apply = [&](const TI* q, TI* y) -> bool {
        float rho = 1.f / sigmaP;
        for (int j = 1; j < a.pdeg; ++j) {
            const float* zin = (j & 1) ? a.zc0 : a.zc1;
            float* zout = (j & 1) ? a.zc1 : a.zc0;
            const bool last = j == a.pdeg - 1;
            const float rn = 1.f / (2.f * sigmaP - rho);
            const float c1 = rn * rho, c2 = 2.f * rn / deltaP;
            if (!grid_sync(a.sw, nb, epoch)) return false;
            spmv_sel<ELL, 2, float, float, RP>(rr, a.eptr, a.ecol, a.evalP, a.rp, a.ci, a.valP, zin, a.lanes, [&](int i, float s0, float s1) {
                const unsigned char m = a.mask[i];
                float z0, z1, d0, d1, i0, i1;
                load2(zin, i, z0, z1);
                load2(a.dc, i, d0, d1);
                load2(a.dinvP, i, i0, i1);
                TI q0, q1;
                load2(q, i, q0, q1);
                const float a0 = (m & 1) ? z0 : s0, a1 = (m & 2) ? z1 : s1;
                const float n0 = c1 * d0 + c2 * i0 * ((float)q0 - a0);
                const float n1 = c1 * d1 + c2 * i1 * ((float)q1 - a1);
                if (last) {
                    store2(y, i, (TI)(z0 + n0), (TI)(z1 + n1));
                } else {
                    store2(a.dc, i, n0, n1);
                    store2(zout, i, z0 + n0, z1 + n1);
                }
            });
            rho = rn;
        }
        return true;
    };

    // initial guess with prescribed values, ||b||^2
    {
        double v[2] = {0.0, 0.0};
        for (int i = rr.r0 + threadIdx.x; i < rr.r1; i += tpb) {
            const unsigned char m = a.mask[i];
            double x0, x1, g0, g1, b0, b1;
            load2(a.x_in, i, x0, x1);
            if (have_dx) {
                double d0, d1;
                load2(a.dx, i, d0, d1);
                if (have_dx2) {
                    double e0, e1;
                    load2(a.dx2, i, e0, e1);
                    d0 = 2.0 * d0 - e0;
                    d1 = 2.0 * d1 - e1;
                }
                x0 += d0;
                x1 += d1;
            }
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
        block_partials_lean<2>(v, a.part + BI_P0 * nb, nb, g.bid, s_lean);
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

    for (;;) {
        double t1[4];
        {
            double v[4] = {0.0, 0.0, 0.0, 0.0};
            spmv_sel<ELL, 2, double, double, 2>(rr, a.eptr, a.ecol, a.eval64, a.rp, a.ci, a.val64, a.x, a.lanes, [&](int i, double s0, double s1) {
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
            block_partials_lean<4>(v, a.part + BI_O1 * nb, nb, g.bid, s_lean);
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
        TI om[2] = {(TI)0, (TI)0};
        for (;;) {
            TI al[2], be[2];
            // ---- (previous omega) d += omega z, r = s - omega t; then p = r + beta (p - omega v),
            //      y = D^-1 p; two rows per thread, all loads of both rows before the first store
            for (int c = 0; c < 2; ++c) be[c] = (TI)beta[c];
            for (int i0 = rr.r0 + threadIdx.x; i0 < rr.r1; i0 += 2 * tpb) {
                const int i1 = i0 + tpb;
                const bool h1 = i1 < rr.r1;
                const int row[2] = {i0, h1 ? i1 : i0};
                TI dv[2][2], rv[2][2], zv[2][2], sv[2][2], tv[2][2], pv[2][2], vv[2][2], dg[2][2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    load2(a.dinvI, row[h], dg[h][0], dg[h][1]);
                    if (first) {
                        load2(a.r, row[h], rv[h][0], rv[h][1]);
                    } else {
                        load2(a.d, row[h], dv[h][0], dv[h][1]);
                        load2(a.z, row[h], zv[h][0], zv[h][1]);
                        load2(a.s, row[h], sv[h][0], sv[h][1]);
                        load2(a.t, row[h], tv[h][0], tv[h][1]);
                        load2(a.p, row[h], pv[h][0], pv[h][1]);
                        load2(a.v, row[h], vv[h][0], vv[h][1]);
                    }
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (h == 1 && !h1) break;
                    TI pn[2], yn[2];
                    if (first) {
#pragma unroll
                        for (int c = 0; c < 2; ++c) pn[c] = rv[h][c];
                    } else {
                        TI dn[2], rn[2];
#pragma unroll
                        for (int c = 0; c < 2; ++c) {
                            dn[c] = dv[h][c] + om[c] * zv[h][c];
                            rn[c] = sv[h][c] - om[c] * tv[h][c];
                            pn[c] = rn[c] + be[c] * (pv[h][c] - om[c] * vv[h][c]);
                        }
                        store2(a.d, row[h], dn[0], dn[1]);
                        store2(a.r, row[h], rn[0], rn[1]);
                    }
                    store2(a.p, row[h], pn[0], pn[1]);
                    if (poly) {
                        float i0, i1;
                        load2(a.dinvP, row[h], i0, i1);
                        const float z0 = i0 * (float)pn[0] / thetaP, z1 = i1 * (float)pn[1] / thetaP;
                        store2(a.zc0, row[h], z0, z1);
                        store2(a.dc, row[h], z0, z1);
                    } else {
#pragma unroll
                        for (int c = 0; c < 2; ++c) yn[c] = dg[h][c] * pn[c];
                        store2(a.y, row[h], yn[0], yn[1]);
                    }
                }
            }
            if (poly && !poly_apply(a.p, a.y)) return record_failure(a.sw, a.st_barrier);
            if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
            // ---- v = A y, sigma = (rh, v); alpha = rho / sigma (thread 0, broadcast)
            {
                TI vs[2] = {(TI)0, (TI)0};
                spmv_sel<ELL, 2, TI, TI, RI>(rr, a.eptr, a.ecol, a.evalI, a.rp, a.ci, a.valI, a.y, a.lanes, [&](int i, TI s0, TI s1) {
                    const TI acc[2] = {s0, s1};
                    TI r0, r1, y0 = (TI)0, y1 = (TI)0;
                    load2(a.rh, i, r0, r1);
                    const unsigned char m = a.mask[i];
                    if (m) load2(a.y, i, y0, y1);
                    const TI v0 = (m & 1) ? y0 : acc[0], v1 = (m & 2) ? y1 : acc[1];
                    store2(a.v, i, v0, v1);
                    vs[0] += r0 * v0;
                    vs[1] += r1 * v1;
                });
                block_partials_it<2, TI>(vs, a.part + BI_B2 * nb, nb, g.bid, s_lean, s_f32);
                if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
                const int slot[2] = {BI_B2, BI_B2 + 1};
                grid_totals_shared<2>(a.part, slot, nb, s_bc);
                // one thread per right-hand side (thread 0: component 0, thread 32: component 1),
                // each carrying its component's recurrence state, so the FP64 divisions of the
                // two components run side by side
                if ((threadIdx.x & 31) == 0 && threadIdx.x < 64) {
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        if ((int)(threadIdx.x >> 5) != c) continue;
                        const double ts = s_bc[c];
                        s_fl[c] = bad(ts) ? 1 : 0;
                        if (act[c] && ts != 0.0) alpha[c] = rho[c] / ts;
                        else { act[c] = false; alpha[c] = 0.0; }
                        s_sc[c] = alpha[c];
                    }
                }
                __syncthreads();
                for (int c = 0; c < 2; ++c) al[c] = (TI)s_sc[c];
                nan |= (s_fl[0] | s_fl[1]) != 0;
            }
            // ---- s = r - alpha v, z = D^-1 s, d += alpha y (two rows per thread)
            for (int i0 = rr.r0 + threadIdx.x; i0 < rr.r1; i0 += 2 * tpb) {
                const int i1 = i0 + tpb;
                const bool h1 = i1 < rr.r1;
                const int row[2] = {i0, h1 ? i1 : i0};
                TI dg[2][2], rv[2][2], vv[2][2], yv[2][2], dv[2][2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    load2(a.dinvI, row[h], dg[h][0], dg[h][1]);
                    load2(a.r, row[h], rv[h][0], rv[h][1]);
                    load2(a.v, row[h], vv[h][0], vv[h][1]);
                    load2(a.y, row[h], yv[h][0], yv[h][1]);
                    load2(a.d, row[h], dv[h][0], dv[h][1]);
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (h == 1 && !h1) break;
                    TI sn[2], zn[2], dn[2];
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        sn[c] = rv[h][c] - al[c] * vv[h][c];
                        zn[c] = dg[h][c] * sn[c];
                        dn[c] = dv[h][c] + al[c] * yv[h][c];
                    }
                    store2(a.s, row[h], sn[0], sn[1]);
                    store2(a.d, row[h], dn[0], dn[1]);
                    if (poly) {
                        float i0, i1;
                        load2(a.dinvP, row[h], i0, i1);
                        const float z0 = i0 * (float)sn[0] / thetaP, z1 = i1 * (float)sn[1] / thetaP;
                        store2(a.zc0, row[h], z0, z1);
                        store2(a.dc, row[h], z0, z1);
                    } else {
                        store2(a.z, row[h], zn[0], zn[1]);
                    }
                }
            }
            if (poly && !poly_apply(a.s, a.z)) return record_failure(a.sw, a.st_barrier);
            if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
            // ---- t = A z; (t, s), (t, t), (rh, t), (rh, s), (s, s) in one reduction
            {
                TI q[10];
#pragma unroll
                for (int k = 0; k < 10; ++k) q[k] = (TI)0;
                spmv_sel<ELL, 2, TI, TI, RI>(rr, a.eptr, a.ecol, a.evalI, a.rp, a.ci, a.valI, a.z, a.lanes, [&](int i, TI s0, TI s1) {
                    const TI acc[2] = {s0, s1};
                    TI z0 = (TI)0, z1 = (TI)0, sv[2], hv[2];
                    const unsigned char m = a.mask[i];
                    if (m) load2(a.z, i, z0, z1);
                    load2(a.s, i, sv[0], sv[1]);
                    load2(a.rh, i, hv[0], hv[1]);
                    const TI tv[2] = {(m & 1) ? z0 : acc[0], (m & 2) ? z1 : acc[1]};
                    store2(a.t, i, tv[0], tv[1]);
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        q[c] += tv[c] * sv[c];
                        q[2 + c] += tv[c] * tv[c];
                        q[4 + c] += hv[c] * tv[c];
                        q[6 + c] += hv[c] * sv[c];
                        q[8 + c] += sv[c] * sv[c];
                    }
                });
                block_partials_it<10, TI>(q, a.part + BI_B4 * nb, nb, g.bid, s_lean, s_f32);
                if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
                {
                    int slot[10];
#pragma unroll
                    for (int k = 0; k < 10; ++k) slot[k] = BI_B4 + k;
                    grid_totals_shared<10>(a.part, slot, nb, s_bc);
                }
                iters += 1;
                first = false;
                // omega, the next rho and beta, convergence: one thread per component (as above),
                // broadcast
                if ((threadIdx.x & 31) == 0 && threadIdx.x < 64) {
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        if ((int)(threadIdx.x >> 5) != c) continue;
                        const double ts = s_bc[c], tt = s_bc[2 + c], ht = s_bc[4 + c], hs = s_bc[6 + c];
                        const double ss = s_bc[8 + c];
                        s_fl[c] = (bad(ts) | bad(tt) | bad(ht) | bad(hs) | bad(ss)) ? 1 : 0;
                        if (act[c] && ss <= tgt[c]) {          // converged at the half step
                            act[c] = false;
                            omega[c] = 0.0;
                        } else if (act[c] && tt != 0.0) {
                            omega[c] = ts / tt;
                        } else {
                            act[c] = false;
                            omega[c] = 0.0;
                        }
                        if (act[c]) {
                            // with omega = ts / tt (tt = (t, t) > 0): rnew tt = hs tt - ts ht,
                            // ||r||^2 tt = ss tt - ts^2 and beta = (rnew / rho)(alpha / omega) =
                            // rnew tt alpha / (rho ts); the three divisions are independent
                            const double q = fma(hs, tt, -ts * ht);
                            const double rr2t = fma(ss, tt, -ts * ts);
                            if (rr2t <= tgt[c] * tt) {
                                act[c] = false;
                            } else if (q != 0.0 && ts != 0.0 && rho[c] != 0.0) {
                                beta[c] = (q * alpha[c]) / (rho[c] * ts);
                                rho[c] = q / tt;
                            } else {
                                act[c] = false;            // breakdown: restart in the next pass
                            }
                        }
                        if (!act[c]) beta[c] = 0.0;
                        s_fl[2 + c] = act[c] ? 1 : 0;
                        s_sc[c] = omega[c];
                        s_sc[2 + c] = beta[c];
                    }
                }
                __syncthreads();
                for (int c = 0; c < 2; ++c) {
                    omega[c] = s_sc[c];
                    beta[c] = s_sc[2 + c];
                    om[c] = (TI)omega[c];
                }
                const bool more = (s_fl[2] | s_fl[3]) != 0;
                nan |= (s_fl[0] | s_fl[1]) != 0;
                __syncthreads();   // s_sc / s_fl read by all before they are written again
                if (nan || !more || iters >= a.max_iter) {
                    // last update of this pass: d += omega z
                    for (int i = rr.r0 + threadIdx.x; i < rr.r1; i += tpb) {
                        TI d0, d1, z0, z1;
                        load2(a.d, i, d0, d1);
                        load2(a.z, i, z0, z1);
                        store2(a.d, i, d0 + om[0] * z0, d1 + om[1] * z1);
                    }
                    break;
                }
            }
        }
        if (nan) { status = CGP_ERR_NAN; break; }
        for (int i = rr.r0 + threadIdx.x; i < rr.r1; i += tpb)
            for (int c = 0; c < 2; ++c) a.x[2 * (size_t)i + c] += (double)a.d[2 * (size_t)i + c];
        if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
        outer += 1;
    }
    if (a.dx != nullptr) {
        // the increment of this solve, kept for the next step's guess (converged solves only;
        // the block's own rows, written by this block before its last barrier)
        if (status == CGP_OK)
            for (int i = rr.r0 + threadIdx.x; i < rr.r1; i += tpb) {
                double x0, x1, u0, u1;
                load2(a.x, i, x0, x1);
                load2(a.x_in, i, u0, u1);
                if (a.dx2) {
                    double d0, d1;
                    load2(a.dx, i, d0, d1);
                    store2(a.dx2, i, d0, d1);
                }
                store2(a.dx, i, x0 - u0, x1 - u1);
            }
        if (g.bid == 0 && threadIdx.x == 0) *a.dx_flag = status == CGP_OK ? min(n_dx + 1, 2) : 0;
    }
    if (g.bid == 0 && threadIdx.x == 0) {
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
    spmv_lanes<NR, double, double>(rr, rp, ci, val, x, lanes, [&](int i, double s0, double s1) {
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

}  // namespace cgp
