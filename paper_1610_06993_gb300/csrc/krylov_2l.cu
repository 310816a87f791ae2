// Batched coarse Poisson solve (Eq. 21) with a two-level additive Schwarz preconditioner.
//
// A batch holds far more coarse rows than the on-chip kernel keeps in shared memory (about a
// million rows of tens of instances on 152 SMs), so this kernel follows the generic persistent
// layout (vectors in global memory, the matrix read through L2) and adds a coarse space:
//     M^-1 r = D^-1 r + R_0^T A_0^-1 R_0 r,
// Jacobi as the local part and three functions per subdomain (1, (x - xbar)/H, (y - ybar)/H) on
// subdomains of CG2_S consecutive rows of a Hilbert-curve renumbering of each instance; A_0 is the
// Galerkin matrix, inverted once on the host. A block group of an instance owns whole
// subdomains; with CG2_S = blockDim.x / 2 and rows strided by blockDim.x, each half of a block
// covers one subdomain per pass, so subdomain sums are block reductions in a fixed order.
//
// Iteration (classical CG, Chronopoulos-Gear form, two grid barriers):
//   p = u + beta p,  s = w + beta s,  d += alpha p,  r -= alpha s
//   R_0 s = R_0 w + beta R_0 s,  R_0 r -= alpha R_0 s     (coarse vectors, every block)
//   u = D^-1 r + R_0^T A_0^-1 R_0 r                         (the block's rows and subdomains)
//   publish u | barrier | w = A u; (r,u), (r,r), (w,u) and the subdomain sums of w, r, s | barrier
// The sums of r and s taken at the second barrier are exact, so the coarse recurrences above span
// one step each and their rounding never accumulates.
#include <algorithm>
#include <vector>

#include "ctx.h"
#include "krylov_kernels.cuh"
#include "subdomain.h"

namespace cgp {

#define CG2_S 256          // rows per subdomain (half of the 512-thread block)
#define CG2_MAXSUB 512     // subdomains per instance (n <= 131,072 rows)

namespace {

template <typename TI>
struct Cg2Args {
    int n, nsub;
    const int* perm;        // [n] renumbered row -> caller row
    const int* rp;          // renumbered CSR
    const int* ci;
    const double* val64;
    const TI* valI;
    const TI* dinvI;        // [n] renumbered
    const float* fxy;       // [n][2] linear coarse functions, renumbered
    const float* ainv;      // [3 nsub][3 nsub]
    const double* b;        // [n] caller numbering
    double* x;              // [n] caller numbering
    double* xp;             // [n] x renumbered (published for the FP64 residual)
    TI *r, *u, *w, *p, *s, *d;
    double* part;           // group partial sums
    double* mom;            // [9][nsub] subdomain sums of w, r, s times (1, fx, fy)
    SyncWords* sw;
    double rtol, inner_rtol;
    int max_iter, max_outer;
    int* st_iters;
    int* st_outer;
    int* st_status;
    double* st_rel;
    int* st_barrier;
};

enum { C2_P0 = 0, C2_O1 = 1 /* 1 */, C2_G = 2 /* 1 */, C2_I0 = 3 /* 1 */, C2_J = 4 /* 3 */ };

// Dynamic shared memory: the lean FP64 reduction buffer (3 per thread), the three coarse vectors
// R_0 w, R_0 r, R_0 s in FP64 and the block's coarse solution entries, for instances of at most
// nsub_max subdomains.
size_t cg2_smem(int threads, int nsub_max) {
    const size_t ncs = (size_t)SZ_NC * nsub_max;
    return 3 * (size_t)threads * sizeof(double) + 3 * ncs * sizeof(double) + ncs * sizeof(float);
}

template <typename TI, int MINB>
__global__ void __launch_bounds__(512, MINB) k_cg2l(Launch<Cg2Args<TI>> L) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_bc[4];
    __shared__ float s_f32[32 * 4];
    __shared__ float s_wm[16 * 9];
    __shared__ double s_sc[2];
    __shared__ int s_fl[2];
    const Grp g = group_of(L.map);
    const Cg2Args<TI>& a = L.table ? L.table[g.inst] : L.single;
    const unsigned int nb = g.nb;
    unsigned int epoch = 0;
    const int T = blockDim.x, t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int ncs = SZ_NC * a.nsub;
    double* s_lean = reinterpret_cast<double*>(smem);          // [3][T]
    double* s_Rw = s_lean + 3 * T;                             // [ncs] each
    double* s_Rr = s_Rw + ncs;
    double* s_Rs = s_Rr + ncs;
    float* s_y = reinterpret_cast<float*>(s_Rs + ncs);         // [3 q]
    // the block's subdomains and rows
    const int q = (a.nsub + (int)nb - 1) / (int)nb;
    const int sub0 = min(a.nsub, (int)g.bid * q), sub1 = min(a.nsub, sub0 + q);
    const int r0 = min(a.n, sub0 * CG2_S), r1 = min(a.n, sub1 * CG2_S);
    const RowRange rr{r0, r1};
    const int passes = (r1 - r0 + T - 1) / T;   // uniform over the block

    // per-subdomain sums of K per-row values, one pass of T rows at a time (half a block per
    // subdomain); warp sums in FP32, then the eight warp sums of a half in a fixed order
    auto subdomain_sums = [&](int k0, int K, auto rowvals) {
        for (int j = 0; j < passes; ++j) {
            const int row = r0 + t + j * T;
            float v[9];
            rowvals(row, row < r1, v);
            for (int k = 0; k < K; ++k) {
                float x = v[k];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                if (lane == 0) s_wm[warp * 9 + k] = x;
            }
            __syncthreads();
            if (t < 2 * K) {
                const int half = t / K, k = t - half * K;
                const int nw = T / 64;
                float acc = 0.f;
                for (int w8 = 0; w8 < nw; ++w8) acc += s_wm[(half * nw + w8) * 9 + k];
                const int sub = sub0 + 2 * j + half;
                if (sub < sub1) a.mom[(size_t)(k0 + k) * a.nsub + sub] = (double)acc;
            }
            __syncthreads();
        }
    };
    auto gather = [&](int k0, double* dst) {
        for (int j = t; j < ncs; j += T) dst[j] = __ldcg(a.mom + (size_t)k0 * a.nsub + j);
    };
    // s_y = the block's entries of A_0^-1 R_0 r (from s_Rr): one warp per row of A_0^-1
    auto coarse = [&]() {
        const int nrow = SZ_NC * (sub1 - sub0);
        for (int i = warp; i < nrow; i += T / 32) {
            const int f = i / (sub1 - sub0), ls = i - f * (sub1 - sub0);
            const float* arow = a.ainv + (size_t)(f * a.nsub + sub0 + ls) * ncs;
            float acc = 0.f;
            for (int j = lane; j < ncs; j += 32) acc += __ldg(arow + j) * (float)s_Rr[j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) s_y[i] = acc;
        }
    };
    // u = D^-1 r + coarse correction for the block's rows (s_y valid)
    auto apply_u = [&](int row) -> TI {
        const int ls = (row - r0) / CG2_S, nl = sub1 - sub0;
        const float fx = a.fxy[2 * row], fy = a.fxy[2 * row + 1];
        const float y = s_y[ls] + fx * s_y[nl + ls] + fy * s_y[2 * nl + ls];
        return a.dinvI[row] * a.r[row] + (TI)y;
    };

    double bb;
    {
        double v[1] = {0.0}, tt[1];
        for (int row = r0 + t; row < r1; row += T) {
            const double bi = a.b[a.perm[row]];
            v[0] += bi * bi;
            a.xp[row] = a.x[a.perm[row]];
        }
        block_partials_lean<1>(v, a.part + C2_P0 * nb, nb, g.bid, s_lean);
        if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
        grid_totals<1>(a.part + C2_P0 * nb, nb, tt, s_bc);
        bb = tt[0];
    }
    if (bb == 0.0)
        for (int row = r0 + t; row < r1; row += T) a.xp[row] = 0.0;
    const double rtol2 = a.rtol * a.rtol, itol2 = a.inner_rtol * a.inner_rtol, floor2 = 0.25 * rtol2;
    int iters = 0, outer = 0, status = CGP_OK;
    double rr64 = 0.0;
    for (;;) {
        // ---- refinement pass: FP64 true residual r = b - A x, d = 0, exact R_0 r
        if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
        {
            double v[1] = {0.0}, tt[1];
            for (int row = r0 + t; row < r1; row += T) {
                double ax = 0.0;
                for (int k = a.rp[row]; k < a.rp[row + 1]; ++k) ax += a.val64[k] * a.xp[a.ci[k]];
                const double r64 = a.b[a.perm[row]] - ax;
                v[0] += r64 * r64;
                a.r[row] = (TI)r64;
                a.d[row] = (TI)0;
            }
            subdomain_sums(3, 3, [&](int row, bool in, float* vv) {
                const float r = in ? (float)a.r[row] : 0.f;
                vv[0] = r;
                vv[1] = in ? a.fxy[2 * row] * r : 0.f;
                vv[2] = in ? a.fxy[2 * row + 1] * r : 0.f;
            });
            block_partials_lean<1>(v, a.part + C2_O1 * nb, nb, g.bid, s_lean);
            if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
            grid_totals<1>(a.part + C2_O1 * nb, nb, tt, s_bc);
            rr64 = tt[0];
            gather(3, s_Rr);
        }
        if (bad(rr64)) { status = CGP_ERR_NAN; break; }
        if (bb == 0.0 || rr64 <= rtol2 * bb) break;
        if (outer >= a.max_outer || iters >= a.max_iter) { status = CGP_ERR_NOT_CONVERGED; break; }
        const double tgt = fmax(itol2 * rr64, floor2 * bb);
        // ---- u = M^-1 r, gamma = (r, u), publish u
        __syncthreads();
        coarse();
        __syncthreads();
        double gam;
        {
            TI vg[1] = {(TI)0};
            for (int row = r0 + t; row < r1; row += T) {
                const TI u = apply_u(row);
                a.u[row] = u;
                vg[0] += a.r[row] * u;
            }
            double tt[1];
            block_partials_it<1, TI>(vg, a.part + C2_G * nb, nb, g.bid, s_lean, s_f32);
            if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
            grid_totals<1>(a.part + C2_G * nb, nb, tt, s_bc);
            gam = tt[0];
        }
        // ---- w = A u, delta = (w, u), R_0 w
        double alpha;
        {
            TI vd[1] = {(TI)0};
            spmv_rows<1, TI, TI>(rr, a.rp, a.ci, a.valI, a.u, [&](int i, TI s0, TI) {
                a.w[i] = s0;
                vd[0] += s0 * a.u[i];
            });
            __syncthreads();   // w of the block's rows, written by other threads of the product
            subdomain_sums(0, 3, [&](int row, bool in, float* vv) {
                const float w = in ? (float)a.w[row] : 0.f;
                vv[0] = w;
                vv[1] = in ? a.fxy[2 * row] * w : 0.f;
                vv[2] = in ? a.fxy[2 * row + 1] * w : 0.f;
            });
            double tt[1];
            block_partials_it<1, TI>(vd, a.part + C2_I0 * nb, nb, g.bid, s_lean, s_f32);
            if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
            grid_totals<1>(a.part + C2_I0 * nb, nb, tt, s_bc);
            gather(0, s_Rw);
            if (bad(gam) || bad(tt[0])) { status = CGP_ERR_NAN; break; }
            alpha = tt[0] != 0.0 && gam != 0.0 ? gam / tt[0] : 0.0;
        }
        double beta = 0.0;
        bool first = true, nan = false;
        // every thread leaves this loop on the same broadcast flag (or the same initial alpha)
        while (alpha != 0.0 || !first) {
            // ---- local update and coarse recurrences
            const TI A = (TI)alpha, B = (TI)beta;
            for (int row = r0 + t; row < r1; row += T) {
                const TI uo = a.u[row], wo = a.w[row];
                const TI p = first ? uo : uo + B * a.p[row];
                const TI sv = first ? wo : wo + B * a.s[row];
                a.p[row] = p;
                a.s[row] = sv;
                a.d[row] += A * p;
                a.r[row] -= A * sv;
            }
            __syncthreads();   // s_Rw, s_Rr, s_Rs complete
            for (int j = t; j < ncs; j += T) {
                const double rs = first ? s_Rw[j] : s_Rw[j] + beta * s_Rs[j];
                s_Rs[j] = rs;
                s_Rr[j] -= alpha * rs;
            }
            __syncthreads();
            coarse();
            __syncthreads();
            for (int row = r0 + t; row < r1; row += T) a.u[row] = apply_u(row);
            if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
            // ---- w = A u; (r,u), (r,r), (w,u); subdomain sums of w, r, s
            TI q3[3] = {(TI)0, (TI)0, (TI)0};
            spmv_rows<1, TI, TI>(rr, a.rp, a.ci, a.valI, a.u, [&](int i, TI s0, TI) {
                a.w[i] = s0;
                const TI r = a.r[i], u = a.u[i];
                q3[0] += r * u;
                q3[1] += r * r;
                q3[2] += s0 * u;
            });
            __syncthreads();   // w of the block's rows, written by other threads of the product
            subdomain_sums(0, 9, [&](int row, bool in, float* vv) {
                const float fx = in ? a.fxy[2 * row] : 0.f, fy = in ? a.fxy[2 * row + 1] : 0.f;
                const float w = in ? (float)a.w[row] : 0.f, r = in ? (float)a.r[row] : 0.f;
                const float sv = in ? (float)a.s[row] : 0.f;
                vv[0] = w; vv[1] = fx * w; vv[2] = fy * w;
                vv[3] = r; vv[4] = fx * r; vv[5] = fy * r;
                vv[6] = sv; vv[7] = fx * sv; vv[8] = fy * sv;
            });
            block_partials_it<3, TI>(q3, a.part + C2_J * nb, nb, g.bid, s_lean, s_f32);
            if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.st_barrier);
            {
                const int slot[3] = {C2_J, C2_J + 1, C2_J + 2};
                grid_totals_shared<3>(a.part, slot, nb, s_bc);
            }
            gather(0, s_Rw);
            gather(3, s_Rr);
            gather(6, s_Rs);
            iters += 1;
            first = false;
            if (t == 0) {
                const double gnew = s_bc[0], rho = s_bc[1], del = s_bc[2];
                int flag = 0;
                if (bad(gnew) || bad(rho) || bad(del)) {
                    flag = 2;
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
                s_sc[0] = alpha;
                s_sc[1] = beta;
                s_fl[0] = flag;
            }
            __syncthreads();
            const int flag = s_fl[0];
            alpha = s_sc[0];
            beta = s_sc[1];
            __syncthreads();
            if (flag == 2) { nan = true; break; }
            if (flag == 1) break;
        }
        if (nan) { status = CGP_ERR_NAN; break; }
        for (int row = r0 + t; row < r1; row += T) a.xp[row] += (double)a.d[row];
        outer += 1;
    }
    for (int row = r0 + t; row < r1; row += T) a.x[a.perm[row]] = a.xp[row];
    if (g.bid == 0 && threadIdx.x == 0) {
        *a.st_iters = iters;
        *a.st_outer = outer;
        *a.st_status = status;
        *a.st_rel = bb > 0.0 ? sqrt(rr64 / bb) : 0.0;
    }
}

template <typename T>
int tl_alloc(cgp_ctx_s* c, T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? CGP_ERR_NOMEM : CGP_ERR_CUDA;
    c->allocs.push_back(q);
    *p = (T*)q;
    return CGP_OK;
}

template <typename T>
int tl_upload(cgp_ctx_s* c, T** p, const std::vector<T>& v) {
    int s = tl_alloc(c, p, v.size());
    if (s) return s;
    return cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) == cudaSuccess ? CGP_OK
                                                                                                 : CGP_ERR_CUDA;
}

template <typename TI>
Cg2Args<TI> cg2_args(cgp_ctx_s* c, double* x, SyncWords* sw, double* part) {
    const bool mixed = sizeof(TI) == sizeof(float);
    const TwoLevel& tl = c->tl;
    const int n = c->nc;
    char* p = (char*)c->ws;
    Cg2Args<TI> a;
    a.n = n;
    a.nsub = tl.nsub;
    a.perm = tl.perm;
    a.rp = tl.rp;
    a.ci = tl.ci;
    a.val64 = tl.val64;
    a.valI = mixed ? (const TI*)(const void*)tl.val32 : (const TI*)(const void*)tl.val64;
    a.dinvI = mixed ? (const TI*)(const void*)tl.dinv32 : (const TI*)(const void*)tl.dinv64;
    a.fxy = tl.fxy32;
    a.ainv = tl.ainv32;
    a.b = c->bc;
    a.x = x;
    a.xp = carve<double>(p, n);
    a.r = carve<TI>(p, n); a.u = carve<TI>(p, n); a.w = carve<TI>(p, n);
    a.p = carve<TI>(p, n); a.s = carve<TI>(p, n); a.d = carve<TI>(p, n);
    a.part = part;
    a.mom = tl.mom;
    a.sw = sw;
    a.rtol = c->prm.rtol;
    a.inner_rtol = mixed ? c->prm.inner_rtol : 0.0;
    a.max_iter = c->prm.max_iter;
    a.max_outer = c->prm.max_outer;
    a.st_iters = &c->stats->poi_iters; a.st_outer = &c->stats->poi_outer; a.st_status = &c->stats->poi_status;
    a.st_rel = &c->stats->poi_rel; a.st_barrier = &c->stats->barrier_status;
    return a;
}

}  // namespace

// Renumbering, renumbered matrix, coarse functions and the inverse Galerkin matrix of the batched
// two-level solver for the context's current pressure boundary conditions.
int twolevel_build(cgp_ctx_s* c) {
    TwoLevel& tl = c->tl;
    const HostCsr& H = c->hm.coarse;
    const std::vector<double>& xy = c->hm.lv[0].xy;
    const int n = c->nc;
    const int nsub = (n + CG2_S - 1) / CG2_S;
    if (nsub > CG2_MAXSUB) return CGP_ERR_ARG;
    std::vector<int> perm = hilbert_order(xy, n), iperm(n);
    for (int i = 0; i < n; ++i) iperm[perm[i]] = i;
    std::vector<double> K(H.nnz);
    if (cudaMemcpy(K.data(), c->Kc, K.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
        return CGP_ERR_CUDA;
    std::vector<int> rp(1, 0), ci;
    std::vector<double> v, dinv(n, 0.0);
    for (int i = 0; i < n; ++i) {
        const int o = perm[i];
        for (int k = H.rp[o]; k < H.rp[o + 1]; ++k) {
            ci.push_back(iperm[H.ci[k]]);
            v.push_back(K[k]);
            if (H.ci[k] == o) dinv[i] = K[k];
        }
        rp.push_back((int)ci.size());
    }
    for (int i = 0; i < n; ++i) {
        if (!(dinv[i] > 0.0)) return CGP_ERR_ARG;
        dinv[i] = 1.0 / dinv[i];
    }
    const std::vector<int> sub = chunk_subdomains(n, CG2_S);
    const std::vector<double> fxy = linear_functions(xy, perm, sub, n, nsub);
    std::vector<double> Ai;
    int st = galerkin_inverse(rp, ci, v, fxy, sub, n, nsub, Ai);
    if (st != CGP_OK) return st;
    if (!tl.ready) {
        if ((st = tl_alloc(c, &tl.mom, 9 * (size_t)nsub))) return st;
    }
    tl.nsub = nsub;
    if ((st = tl_upload(c, &tl.perm, perm)) || (st = tl_upload(c, &tl.rp, rp)) || (st = tl_upload(c, &tl.ci, ci)) ||
        (st = tl_upload(c, &tl.val64, v)) || (st = tl_upload(c, &tl.val32, std::vector<float>(v.begin(), v.end()))) ||
        (st = tl_upload(c, &tl.dinv64, dinv)) ||
        (st = tl_upload(c, &tl.dinv32, std::vector<float>(dinv.begin(), dinv.end()))) ||
        (st = tl_upload(c, &tl.fxy32, std::vector<float>(fxy.begin(), fxy.end()))) ||
        (st = tl_upload(c, &tl.ainv32, std::vector<float>(Ai.begin(), Ai.end()))))
        return st;
    tl.ready = true;
    return CGP_OK;
}

// The batch's coarse Poisson stage on the two-level kernel: argument table, shared-memory limit
// and a residency check (two blocks per SM, as the batch's block count assumes). Returns false
// (and leaves the batch on the Jacobi kernel) if an instance is too large or it does not fit.
bool batch_poisson2l_build(cgp_batch_s* b) {
    b->poisson_2l = false;
    if (b->threads != 2 * CG2_S) return false;
    int nsub_max = 1;
    for (int i = 0; i < b->n; ++i) {
        cgp_ctx_s* c = b->ctx[i];
        if (c->prm.coarse_solver != 0 || twolevel_build(c) != CGP_OK) return false;
        nsub_max = std::max(nsub_max, c->tl.nsub);
    }
    const size_t sm = cg2_smem(b->threads, nsub_max);
    const void* fn = b->precision == CGP_MIXED ? (const void*)k_cg2l<float, 2> : (const void*)k_cg2l<double, 2>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) return false;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, b->threads, sm) != cudaSuccess) return false;
    if (occ * b->ctx[0]->num_sms < b->blocks_c) return false;
    size_t bytes = 0;
    if (b->precision == CGP_MIXED) {
        std::vector<Cg2Args<float>> tab(b->n);
        for (int i = 0; i < b->n; ++i)
            tab[i] = cg2_args<float>(b->ctx[i], b->pc[i], b->sync + (size_t)i * SYNC_COUNT + SYNC_POI,
                                     b->part + (size_t)i * 32 * b->max_group);
        bytes = sizeof(Cg2Args<float>) * tab.size();
        if (cudaMalloc(&b->tab_poi2, bytes) != cudaSuccess) return false;
        b->allocs.push_back(b->tab_poi2);
        if (cudaMemcpy(b->tab_poi2, tab.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) return false;
    } else {
        std::vector<Cg2Args<double>> tab(b->n);
        for (int i = 0; i < b->n; ++i)
            tab[i] = cg2_args<double>(b->ctx[i], b->pc[i], b->sync + (size_t)i * SYNC_COUNT + SYNC_POI,
                                      b->part + (size_t)i * 32 * b->max_group);
        bytes = sizeof(Cg2Args<double>) * tab.size();
        if (cudaMalloc(&b->tab_poi2, bytes) != cudaSuccess) return false;
        b->allocs.push_back(b->tab_poi2);
        if (cudaMemcpy(b->tab_poi2, tab.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) return false;
    }
    b->smem_poi2 = sm;
    b->poisson_2l = true;
    return true;
}

// ---- many right-hand sides of one coarse matrix (cgp_poisson_solve_many) ----------------------
namespace {

// Per-right-hand-side workspace layout (256-byte carved): xp (n doubles), r u w p s d (n TI each),
// mom (9 nsub doubles), part (32 doubles), sync words.
template <typename TI>
size_t many_bytes(int n, int nsub) {
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    return al(sizeof(double) * n) + 6 * al(sizeof(TI) * n) + al(sizeof(double) * 9 * nsub) + al(32 * sizeof(double)) +
           al(sizeof(SyncWords));
}

// Arguments of right-hand side i of the launch: the context's shared template with the
// per-right-hand-side vectors, workspace and statistics (one block per right-hand side).
template <typename TI>
__global__ void k_many_table(int cnt, Cg2Args<TI> tmpl, const double* b, double* x, size_t n, char* ws, size_t per,
                             int* stats, int* rhs_iters, double* rhs_rel, int* rhs_status, int first,
                             Cg2Args<TI>* tab) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    auto al = [](size_t v) { return (v + 255) / 256 * 256; };
    Cg2Args<TI> a = tmpl;
    char* p = ws + (size_t)i * per;
    a.b = b + (size_t)(first + i) * n;
    a.x = x + (size_t)(first + i) * n;
    a.xp = (double*)p; p += al(sizeof(double) * n);
    a.r = (TI*)p; p += al(sizeof(TI) * n);
    a.u = (TI*)p; p += al(sizeof(TI) * n);
    a.w = (TI*)p; p += al(sizeof(TI) * n);
    a.p = (TI*)p; p += al(sizeof(TI) * n);
    a.s = (TI*)p; p += al(sizeof(TI) * n);
    a.d = (TI*)p; p += al(sizeof(TI) * n);
    a.mom = (double*)p; p += al(sizeof(double) * 9 * tmpl.nsub);
    a.part = (double*)p; p += al(32 * sizeof(double));
    a.sw = (SyncWords*)p;
    a.sw->count = 0;
    a.sw->err = 0;
    int* st = stats + 8 * (size_t)i;
    st[3] = 0;
    a.st_iters = rhs_iters ? rhs_iters + first + i : st;
    a.st_outer = st + 1;
    a.st_status = rhs_status ? rhs_status + first + i : st + 2;
    a.st_barrier = st + 3;   // one block per right-hand side: its barriers never wait
    a.st_rel = rhs_rel ? rhs_rel + first + i : (double*)(st + 4);
    tab[i] = a;
}

template <typename TI>
int many_launch(cgp_ctx_s* c, int nrhs, const double* b, double* x, int* iters, double* rel, int* status,
                cudaStream_t s) {
    ManyRhs& m = c->many;
    const int n = c->nc;
    Cg2Args<TI> tmpl = cg2_args<TI>(c, x, nullptr, nullptr);
    for (int w0 = 0; w0 < nrhs; w0 += m.wave) {
        const int cnt = std::min(m.wave, nrhs - w0);
        k_many_table<TI><<<(cnt + 127) / 128, 128, 0, s>>>(cnt, tmpl, b, x, (size_t)n, (char*)m.ws, m.per_rhs, m.stats,
                                                          iters, rel, status, w0, (Cg2Args<TI>*)m.tab);
        if (cudaGetLastError() != cudaSuccess) return CGP_ERR_CUDA;
        Launch<Cg2Args<TI>> L;
        L.single = Cg2Args<TI>();
        L.table = (const Cg2Args<TI>*)m.tab;
        L.map = {m.map_ib, m.map_b0, m.map_nb};
        if (coop_launch(k_cg2l<TI, 2>, cnt, 2 * CG2_S, L, s, m.smem) != cudaSuccess) return CGP_ERR_CUDA;
    }
    return CGP_OK;
}

}  // namespace

// Set-up of the multi-right-hand-side solve: the two-level structures and the per-wave workspace.
int many_prepare(cgp_ctx_s* c) {
    ManyRhs& m = c->many;
    if (m.ws) return CGP_OK;
    int st = c->tl.ready ? CGP_OK : twolevel_build(c);
    if (st != CGP_OK) return st;
    const bool mixed = c->prm.precision == CGP_MIXED;
    const void* fn = mixed ? (const void*)k_cg2l<float, 2> : (const void*)k_cg2l<double, 2>;
    m.smem = cg2_smem(2 * CG2_S, c->tl.nsub);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)m.smem) != cudaSuccess)
        return CGP_ERR_CUDA;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 2 * CG2_S, m.smem) != cudaSuccess || occ < 1)
        return CGP_ERR_CUDA;
    m.wave = std::min(occ * c->num_sms, CGP_MAX_GRID * 4);
    m.per_rhs = mixed ? many_bytes<float>(c->nc, c->tl.nsub) : many_bytes<double>(c->nc, c->tl.nsub);
    const size_t tab_bytes = (mixed ? sizeof(Cg2Args<float>) : sizeof(Cg2Args<double>)) * (size_t)m.wave;
    std::vector<int> ib(m.wave), b0(m.wave), nb(m.wave, 1);
    for (int i = 0; i < m.wave; ++i) ib[i] = b0[i] = i;
    if ((st = tl_alloc(c, (char**)&m.ws, m.per_rhs * (size_t)m.wave)) || (st = tl_alloc(c, (char**)&m.tab, tab_bytes)) ||
        (st = tl_alloc(c, &m.stats, 8 * (size_t)m.wave)) || (st = tl_upload(c, &m.map_ib, ib)) ||
        (st = tl_upload(c, &m.map_b0, b0)) || (st = tl_upload(c, &m.map_nb, nb)))
        return st;
    return CGP_OK;
}

int many_solve(cgp_ctx_s* c, int nrhs, const double* b, double* x, int* iters, double* rel, int* status,
               cudaStream_t s) {
    int st = many_prepare(c);
    if (st != CGP_OK) return st;
    return c->prm.precision == CGP_MIXED ? many_launch<float>(c, nrhs, b, x, iters, rel, status, s)
                                         : many_launch<double>(c, nrhs, b, x, iters, rel, status, s);
}

cudaError_t batch_poisson2l_launch(cgp_batch_s* b, cudaStream_t s) {
    if (b->precision == CGP_MIXED) {
        Launch<Cg2Args<float>> L;
        L.single = Cg2Args<float>();
        L.table = (const Cg2Args<float>*)b->tab_poi2;
        L.map = b->map_c;
        return coop_launch(k_cg2l<float, 2>, b->blocks_c, b->threads, L, s, b->smem_poi2);
    }
    Launch<Cg2Args<double>> L;
    L.single = Cg2Args<double>();
    L.table = (const Cg2Args<double>*)b->tab_poi2;
    L.map = b->map_c;
    return coop_launch(k_cg2l<double, 2>, b->blocks_c, b->threads, L, s, b->smem_poi2);
}

}  // namespace cgp
