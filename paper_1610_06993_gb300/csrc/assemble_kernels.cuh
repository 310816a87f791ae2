// Per-step momentum assembly kernel, shared by the single-instance launcher (assemble.cu)
// and the batched multi-instance step (batch.cu).
#pragma once
#include "ctx.h"

namespace cgp {
namespace {

struct StepAsmArgs {
    int nf, nnz, ncol;
    const int* colptr;           // device copy of the colour offsets
    const int* perm;
    const int* slot;
    const double* conv;          // [t][6] gradients scaled by dt rho |T| / 12
    const int* tri;
    const int* rp;
    const int* ci;
    const int* diag;
    const double* A0;
    const double* M;
    const double* u;             // [nf][2] u^n
    const unsigned char* mask;
    const double* g;
    double* A;
    float* A32;                  // nullptr unless CGP_MIXED
    double* dinv;                // [nf][2]
    float* dinv32;
    double* b;                   // [nf][2]
    unsigned int* bound;         // Gershgorin bound of D^-1 A (float bits, atomic max), or nullptr
    double rho;
    SyncWords* sw;
    int* barrier_status;
};

// Per-step momentum matrix A = A0 + dt rho N(u^n), Jacobi diagonals and right-hand side
// b = rho M u^n (Dirichlet rows: prescribed values). One cooperative launch; grid barriers
// separate the copy, each colour and the row pass.
__global__ void __launch_bounds__(1024) k_assemble_step(Launch<StepAsmArgs> L) {
    const Grp grp = group_of(L.map);
    const StepAsmArgs& a = L.table ? L.table[grp.inst] : L.single;
    unsigned int epoch = 0;
    const unsigned int nb = grp.nb;
    const int tid = grp.bid * blockDim.x + threadIdx.x;
    const int nthreads = grp.nb * blockDim.x;
    if (a.bound && tid == 0) *a.bound = 0u;
    for (int k = tid; k < a.nnz; k += nthreads) a.A[k] = a.A0[k];
    if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.barrier_status);
    for (int c = 0; c < a.ncol; ++c) {
        const int k0 = a.colptr[c], k1 = a.colptr[c + 1];
        for (int k = k0 + tid; k < k1; k += nthreads) {
            const int e = a.perm[k];
            const double* g = a.conv + 6 * (size_t)e;
            double ux[3], uy[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) load2(a.u, a.tri[3 * e + q], ux[q], uy[q]);
            const double sx = ux[0] + ux[1] + ux[2], sy = uy[0] + uy[1] + uy[2];
            double S[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) S[q] = fma(sy, g[3 + q], sx * g[q]);
            const int* sl = a.slot + 9 * (size_t)e;
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int q = 0; q < 3; ++q) a.A[sl[r * 3 + q]] += fma(ux[r], g[q], fma(uy[r], g[3 + q], S[q]));
        }
        if (!grid_sync(a.sw, nb, epoch)) return record_failure(a.sw, a.barrier_status);
    }
    float gmax = 1.f;
    for (int i = tid; i < a.nf; i += nthreads) {
        const unsigned char m = a.mask[i];
        const int kd = a.diag[i];
        const double dg = a.A[kd];
        const double di = 1.0 / dg;
        double dx = (m & CGP_BC_U) ? 1.0 : di, dy = (m & CGP_BC_V) ? 1.0 : di;
        store2(a.dinv, i, dx, dy);
        double mx = 0.0, my = 0.0;
        float off = 0.f;
        for (int k = a.rp[i]; k < a.rp[i + 1]; ++k) {
            double ujx, ujy;
            load2(a.u, a.ci[k], ujx, ujy);
            const double mv = a.M[k];
            mx += mv * ujx;
            my += mv * ujy;
            if (a.A32) {
                const float av = (float)a.A[k];
                a.A32[k] = av;
                if (k != kd) off += fabsf(av);
            }
        }
        double gx, gy;
        load2(a.g, i, gx, gy);
        store2(a.b, i, (m & CGP_BC_U) ? gx : a.rho * mx, (m & CGP_BC_V) ? gy : a.rho * my);
        if (a.dinv32) store2(a.dinv32, i, (float)dx, (float)dy);
        // Gershgorin disc of row i of D^-1 A (identity rows for Dirichlet components)
        if ((m & (CGP_BC_U | CGP_BC_V)) != (CGP_BC_U | CGP_BC_V)) gmax = fmaxf(gmax, 1.f + off / fabsf((float)dg));
    }
    if (a.bound) {
        const unsigned int gb = __reduce_max_sync(0xffffffffu, __float_as_uint(gmax));
        if ((threadIdx.x & 31) == 0) atomicMax(a.bound, gb);
    }
}

}  // namespace
}  // namespace cgp
