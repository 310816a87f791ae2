// Batched multi-instance CGP step: many independent contexts (meshes of uneven size) advanced
// together. Each persistent stage (assembly, momentum BiCGStab, coarse CG, mass CG) is one
// cooperative launch for all instances; the grid is cut into per-instance block groups sized by
// the instance's work, and barriers and reductions stay inside a group, so instances never wait
// for one another inside a stage. The gathers between the stages are launched per instance. A
// whole step can be captured once as a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <new>

#include "ctx.h"

using namespace cgp;

namespace {

// Cut `total` blocks into one group per weight (>= 1 block each, <= CGP_MAX_GRID) by largest
// remainder. Returns false if there are more instances than blocks.
bool apportion(const std::vector<double>& w, int total, std::vector<int>& nb, std::vector<int>& b0) {
    const int n = (int)w.size();
    if (n > total) return false;
    double W = 0.0;
    for (double x : w) W += x;
    std::vector<double> share(n);
    nb.assign(n, 1);
    int sum = 0;
    for (int i = 0; i < n; ++i) {
        share[i] = W > 0.0 ? total * w[i] / W : (double)total / n;
        nb[i] = std::max(1, std::min(CGP_MAX_GRID, (int)std::floor(share[i])));
        sum += nb[i];
    }
    while (sum < total) {
        int best = -1;
        double br = -1e300;
        for (int i = 0; i < n; ++i)
            if (nb[i] < CGP_MAX_GRID && share[i] - nb[i] > br) {
                br = share[i] - nb[i];
                best = i;
            }
        if (best < 0) break;
        nb[best] += 1;
        sum += 1;
    }
    while (sum > total) {
        int best = -1;
        for (int i = 0; i < n; ++i)
            if (nb[i] > 1 && (best < 0 || nb[i] > nb[best])) best = i;
        if (best < 0) return false;
        nb[best] -= 1;
        sum -= 1;
    }
    b0.assign(n, 0);
    for (int i = 1; i < n; ++i) b0[i] = b0[i - 1] + nb[i - 1];
    return true;
}

template <typename T>
int dalloc(cgp_batch_s* b, T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? CGP_ERR_NOMEM : CGP_ERR_CUDA;
    b->allocs.push_back(q);
    *p = (T*)q;
    return CGP_OK;
}

int upload_map(cgp_batch_s* b, const std::vector<int>& nb, const std::vector<int>& b0, int total, BatchMap& m) {
    std::vector<int> inst(total, 0);
    for (size_t i = 0; i < nb.size(); ++i)
        for (int k = 0; k < nb[i]; ++k) inst[b0[i] + k] = (int)i;
    int *d_inst = nullptr, *d_b0 = nullptr, *d_nb = nullptr;
    int s;
    if ((s = dalloc(b, &d_inst, inst.size())) || (s = dalloc(b, &d_b0, b0.size())) || (s = dalloc(b, &d_nb, nb.size())))
        return s;
    if (cudaMemcpy(d_inst, inst.data(), sizeof(int) * inst.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_b0, b0.data(), sizeof(int) * b0.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_nb, nb.data(), sizeof(int) * nb.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return CGP_ERR_CUDA;
    m = {d_inst, d_b0, d_nb};
    return CGP_OK;
}

void destroy_batch(cgp_batch_s* b) {
    if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (void* p : b->allocs) cudaFree(p);
    b->allocs.clear();
}

int create_impl(cgp_ctx* ctxs, int n, double* const* u, double* const* pc, cgp_batch_s* b) {
    b->n = n;
    b->ctx.assign(ctxs, ctxs + n);
    b->u.assign(u, u + n);
    b->pc.assign(pc, pc + n);
    b->precision = ctxs[0]->prm.precision;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i] || !u[i] || !pc[i]) return CGP_ERR_ARG;
        if (!ctxs[i]->bc_set) return CGP_ERR_STATE;
        if (ctxs[i]->prm.precision != b->precision) return CGP_ERR_ARG;
        if (ctxs[i]->device != ctxs[0]->device) return CGP_ERR_ARG;
        if (ctxs[i]->prm.projection != 0) return CGP_ERR_ARG;   // incremental forms: single contexts only
    }
    const int sms = ctxs[0]->num_sms;
    const int bps = std::min(2, persistent_blocks_per_sm(b->threads, true));
    if (bps < 1) return CGP_ERR_CUDA;
    const int total = sms * bps;
    std::vector<double> wf(n), wc(n);
    for (int i = 0; i < n; ++i) {
        wf[i] = (double)ctxs[i]->F.nnz;
        wc[i] = (double)ctxs[i]->C.nnz * std::sqrt((double)ctxs[i]->nc);   // CG iterations grow like sqrt(n)
    }
    if (!apportion(wf, total, b->nb_f, b->b0_f) || !apportion(wc, total, b->nb_c, b->b0_c)) return CGP_ERR_ARG;
    b->blocks_f = total;
    b->blocks_c = total;
    b->max_group = 1;
    for (int i = 0; i < n; ++i) b->max_group = std::max({b->max_group, b->nb_f[i], b->nb_c[i]});
    int s;
    if ((s = upload_map(b, b->nb_f, b->b0_f, total, b->map_f))) return s;
    if ((s = upload_map(b, b->nb_c, b->b0_c, total, b->map_c))) return s;
    if ((s = dalloc(b, &b->sync, (size_t)n * SYNC_COUNT))) return s;
    if ((s = dalloc(b, &b->part, (size_t)n * 32 * b->max_group))) return s;
    if (batch_asm_build(b) != cudaSuccess || batch_solvers_build(b) != cudaSuccess) return CGP_ERR_CUDA;
    // coarse Poisson on the two-level kernel when every instance asks for the automatic coarse
    // solver and fits it; otherwise the Jacobi kernel
    batch_poisson2l_build(b);
    cudaGetLastError();
    if (batch_predict_build(b) != cudaSuccess || batch_perm_build(b) != cudaSuccess) return CGP_ERR_CUDA;
    batch_gather_build(b);
    cudaGetLastError();
    return CGP_OK;
}

cudaError_t enqueue_step(cgp_batch_s* b, cudaStream_t s) {
    for (int i = 0; i < b->n; ++i) {
        // each instance's A is assembled from u^n in its stored order: u_int, or (identity order)
        // the caller's buffer, which the correction overwrites with u^(n+1)
        cgp_ctx_s* c = b->ctx[i];
        c->u_asm = c->fperm ? c->u_int : nullptr;
        c->assembled = true;
    }
    cudaError_t e = cudaMemsetAsync(b->sync, 0, sizeof(SyncWords) * (size_t)b->n * SYNC_COUNT, s);
    if (e == cudaSuccess) e = batch_perm_launch(b, s);   // u^n into the instances' stored fine order
    if (e == cudaSuccess) e = batch_asm_launch(b, s);
    if (e == cudaSuccess) e = batch_predict_launch(b, s);   // p_c and w still hold step n
    if (e == cudaSuccess) e = batch_momentum_launch(b, s);
    if (b->gather) {
        // the gathers between the persistent stages: one launch per stage for every instance
        if (e == cudaSuccess) e = batch_restrict_launch(b, s);
        if (e == cudaSuccess) e = b->poisson_2l ? batch_poisson2l_launch(b, s) : batch_poisson_launch(b, s);
        if (e == cudaSuccess) e = batch_prolong_gradient_launch(b, s);
        if (e == cudaSuccess) e = batch_mass_launch(b, s);
        if (e == cudaSuccess) e = batch_correct_launch(b, s);
        return e;
    }
    for (int i = 0; i < b->n && e == cudaSuccess; ++i) e = launch_restrict_rhs(b->ctx[i], b->ctx[i]->ut, b->ctx[i]->bc, s);
    if (e == cudaSuccess) e = b->poisson_2l ? batch_poisson2l_launch(b, s) : batch_poisson_launch(b, s);
    for (int i = 0; i < b->n && e == cudaSuccess; ++i) {
        cgp_ctx_s* c = b->ctx[i];
        e = launch_prolong(c, b->pc[i], c->pf, s);
        if (e == cudaSuccess) e = launch_gradient(c, c->pf, c->grad, s);
    }
    if (e == cudaSuccess) e = batch_mass_launch(b, s);
    for (int i = 0; i < b->n && e == cudaSuccess; ++i)
        e = launch_correct(b->ctx[i], b->ctx[i]->ut, b->ctx[i]->w, b->u[i], nullptr, s, true);
    return e;
}

}  // namespace

extern "C" {

int cgp_batch_create(cgp_ctx* ctxs, int n, double* const* u_devs, double* const* pc_devs, cgp_batch* out) {
    if (!ctxs || !u_devs || !pc_devs || !out || n <= 0) return CGP_ERR_ARG;
    *out = nullptr;
    cgp_batch_s* b = new (std::nothrow) cgp_batch_s();
    if (!b) return CGP_ERR_NOMEM;
    int s = create_impl(ctxs, n, u_devs, pc_devs, b);
    if (s != CGP_OK) {
        destroy_batch(b);
        delete b;
        return s;
    }
    *out = b;
    return CGP_OK;
}

int cgp_batch_info(cgp_batch b, int* blocks, int* group_fine, int* group_coarse) {
    if (!b) return CGP_ERR_ARG;
    if (blocks) *blocks = b->blocks_f;
    for (int i = 0; i < b->n; ++i) {
        if (group_fine) group_fine[i] = b->nb_f[i];
        if (group_coarse) group_coarse[i] = b->nb_c[i];
    }
    return CGP_OK;
}

int cgp_batch_step(cgp_batch b, void* stream) {
    if (!b) return CGP_ERR_ARG;
    return enqueue_step(b, (cudaStream_t)stream) == cudaSuccess ? CGP_OK : CGP_ERR_CUDA;
}

int cgp_batch_run(cgp_batch b, int steps, void* stream) {
    if (!b || steps < 0) return CGP_ERR_ARG;
    if (!b->graph_exec) {
        if (!b->cap_stream && cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
            return CGP_ERR_CUDA;
        if (cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return CGP_ERR_CUDA;
        cudaError_t e = enqueue_step(b, b->cap_stream);
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &g);
        if (e != cudaSuccess || e2 != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            return CGP_ERR_CUDA;
        }
        b->graph = g;
        if (cudaGraphInstantiate(&b->graph_exec, g, 0) != cudaSuccess) return CGP_ERR_CUDA;
    }
    for (int k = 0; k < steps; ++k)
        if (cudaGraphLaunch(b->graph_exec, (cudaStream_t)stream) != cudaSuccess) return CGP_ERR_CUDA;
    return CGP_OK;
}

int cgp_batch_poisson_solve(cgp_batch b, void* stream) {
    if (!b) return CGP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(b->sync, 0, sizeof(SyncWords) * (size_t)b->n * SYNC_COUNT, s);
    if (e == cudaSuccess) e = b->poisson_2l ? batch_poisson2l_launch(b, s) : batch_poisson_launch(b, s);
    return e == cudaSuccess ? CGP_OK : CGP_ERR_CUDA;
}

int cgp_batch_get_stats(cgp_batch b, void* stream, cgp_stats* per_instance) {
    if (!b || !per_instance) return CGP_ERR_ARG;
    int first = CGP_OK;
    for (int i = 0; i < b->n; ++i) {
        int s = cgp_get_stats(b->ctx[i], stream, &per_instance[i]);
        if (s == CGP_ERR_CUDA || s == CGP_ERR_ARG) return s;
        if (first == CGP_OK) first = s;
    }
    return first;
}

int cgp_batch_destroy(cgp_batch b) {
    if (!b) return CGP_OK;
    cudaDeviceSynchronize();
    destroy_batch(b);
    delete b;
    return CGP_OK;
}

}  // extern "C"
