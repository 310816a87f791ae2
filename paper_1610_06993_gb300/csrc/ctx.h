// Internal state of a CGP context and the kernel launchers shared by the .cu files.
#pragma once
#include <cuda_runtime.h>
#include <vector>
#include "cgp.h"
#include "common.cuh"
#include "host_mesh.h"

#define CGP_MAX_LEVELS 4   // refinement levels a context may have (cgp_mesh_create checks)

namespace cgp {

// Device-side statistics of the latest solves (mirrors cgp_stats).
struct DevStats {
    int mom_iters, mom_outer, mom_status;
    int poi_iters, poi_outer, poi_status;
    int mass_iters, mass_outer, mass_status;
    int barrier_status;
    double mom_rel, poi_rel, mass_rel;
};

struct DevCsr {
    int n = 0, nnz = 0;
    int* rp = nullptr;
    int* ci = nullptr;
    int* diag = nullptr;
};

struct DevElems {
    int t = 0, ncol = 0;
    std::vector<int> colptr;   // host copy of colour offsets
    int* colptr_dev = nullptr; // device copy of colour offsets
    int* tri = nullptr;        // [t][3]
    int* slot = nullptr;       // [t][9]
    int* perm = nullptr;       // [t]
    double* geo = nullptr;     // [t][8]: area, gx[3], gy[3], pad
    double* conv = nullptr;    // [t][6]: c gx[3], c gy[3] with c = dt rho |T| / 12 (fine set)
};

// Launch shape of one persistent (cooperative) kernel family.
struct Shape {
    int blocks = 1, threads = 512, lanes = 4;
};

// Sync words: one slot per persistent launch site, zeroed before every launch.
enum SyncSlot { SYNC_ASM = 0, SYNC_MOM, SYNC_POI, SYNC_MASS, SYNC_COUNT };

// Coarse space of the batched two-level coarse CG (krylov_2l.cu): Hilbert renumbering, the
// renumbered matrix, and 256-row subdomains with three coarse functions each.
struct TwoLevel {
    bool ready = false;
    int nsub = 0;
    int *perm = nullptr, *rp = nullptr, *ci = nullptr;
    double *val64 = nullptr, *dinv64 = nullptr, *mom = nullptr;
    float *val32 = nullptr, *dinv32 = nullptr, *fxy32 = nullptr, *ainv32 = nullptr;
};

// Workspace of the multi-right-hand-side coarse solve (cgp_poisson_solve_many): one block per
// right-hand side, up to `wave` right-hand sides per cooperative launch.
struct ManyRhs {
    int wave = 0;               // right-hand sides per launch (resident blocks of the kernel)
    size_t per_rhs = 0;         // workspace bytes per right-hand side
    void* ws = nullptr;         // [wave][per_rhs]
    void* tab = nullptr;        // [wave] kernel arguments, filled on the device per launch
    int* stats = nullptr;       // [wave][8] iteration count, outer passes, status, barrier, rel (2 ints)
    int *map_ib = nullptr, *map_b0 = nullptr, *map_nb = nullptr;   // identity block-group map
    size_t smem = 0;
};

}  // namespace cgp

struct cgp_ctx_s {
    cgp_params prm;
    int device = 0, num_sms = 0;
    cgp::HostMesh hm;
    int nf = 0, nc = 0, levels = 0;
    bool bc_set = false;

    cgp::DevCsr F, C;            // fine and coarse P1 patterns
    cgp::DevElems EF, EC;
    int* cif_su = nullptr;       // coarse CSR columns mapped to fine node indices (ci[k] -> xi)
    double* xy_f = nullptr;
    double* xy_c = nullptr;

    // fine operators (values in the fine pattern)
    double* M = nullptr;         // consistent mass
    double* A0 = nullptr;        // rho M + dt mu K
    double* A = nullptr;         // per-step momentum matrix
    float* A32 = nullptr;        // FP32 copy (CGP_MIXED)
    double* Gxy = nullptr;       // [nnz][2] gradient (G = D on the fine mesh)
    double* dinvM = nullptr;     // [nf]
    float* M32 = nullptr;        // FP32 copies of M and its inverse diagonal (CGP_MIXED)
    float* dinvM32 = nullptr;
    double* dinvA = nullptr;     // [nf][2]
    float* dinvA32 = nullptr;    // [nf][2]
    double* b_mom = nullptr;     // [nf][2]

    // coarse operators
    double* Kc_raw = nullptr;    // stiffness before boundary elimination
    double* Kc = nullptr;        // after symmetric elimination
    float* Kc32 = nullptr;
    double* Dc_xy = nullptr;     // [nnz_c][2]
    double* dinvK = nullptr;
    float* dinvK32 = nullptr;

    // mapping tables and boundary data
    std::vector<int2*> sp;       // per level [N_{k+1}] (beta, gamma)
    std::vector<int> lv_n;       // node count per level
    std::vector<double*> pl;     // prolongation buffers per level 1..L (level L may be caller's)
    unsigned char* vel_mask = nullptr;   // [nf]
    unsigned char* p_mask = nullptr;     // [nc]
    double* g = nullptr;                 // [nf][2]

    // correction
    double* grad = nullptr;      // [nf][2] G p_f
    double* w = nullptr;         // [nf][2] M^{-1} G p_f (kept as the next warm start)
    double* pf = nullptr;        // [nf]
    double* ut = nullptr;        // [nf][2] intermediate velocity for cgp_step
    double* bc = nullptr;        // [nc] coarse right-hand side for cgp_step
    double* pc_prev = nullptr;   // [nc] pressure seen by the previous predictor call
    int* pc_flag = nullptr;      // 1 once pc_prev holds a pressure
    double* w_prev = nullptr;    // [nf][2] previous mass-solve solution (warm_start >= 1)
    double* w_prev2 = nullptr;   // [nf][2] the two before (warm_start >= 2, 3)
    double* w_prev3 = nullptr;
    double* pc_prev2 = nullptr;  // [nc] the two pressures before pc_prev
    double* pc_prev3 = nullptr;
    double* mom_dx2 = nullptr;   // [nf][2] the momentum increment before mom_dx (warm_start = 3)
    int* asm_ip = nullptr;       // [nnz_f + 1] per CSR entry: offsets into asm_idx
    int* asm_idx = nullptr;      // [9 t_f] element contributions of each entry, element order
    double* asm_ev = nullptr;    // [9 t_f] the step's element contributions
    int* w_flag = nullptr;
    double* mom_dx = nullptr;    // [nf][2] last momentum increment u~^n - u^(n-1) (warm_start = 1)
    int* mom_flag = nullptr;     // number of increments recorded, 0 .. 2
    unsigned int* mom_bound = nullptr;   // Gershgorin bound of the spectrum of D^-1 A (float bits)
    bool fp32_A = false;         // the assembly writes A32 / dinvA32 (mixed, or momentum polynomial)

    // Krylov workspace and reductions
    void* ws = nullptr;
    size_t ws_bytes = 0;
    double* part = nullptr;      // partial sums [CGP_PART_SLOTS][max_blocks]
    int max_blocks = 0;
    cgp::SyncWords* sync = nullptr;
    cgp::DevStats* stats = nullptr;

    // staging for cgp_step_host
    double* u_stage = nullptr;
    double* pc_stage = nullptr;

    // fine-node storage order (fine_order 0: a Hilbert curve, see host_mesh.h). Fine vectors
    // cross the interface in the refinement order; fperm[i] is the refinement-order index of
    // stored node i (nullptr: the two orders coincide). u_int: the velocity in the stored order.
    int* fperm = nullptr;
    double* u_int = nullptr;
    // u_asm: the stored-order u^n of the last assembly while some buffer still holds it (nullptr
    // once a correction wrote u^(n+1) over the caller's buffer in the identity order, or a
    // diagnostic reused u_int); assembled: A of Eq. 19 holds an assembly
    const double* u_asm = nullptr;
    bool assembled = false;

    // sliced-ELL (SELL-32-256) copy of the fine pattern for the stand-alone SpMV
    int sell_nslices = 0, sell_total = 0;
    int *sell_ptr = nullptr, *sell_col = nullptr, *sell_src = nullptr, *sell_perm = nullptr;
    double* sell_val = nullptr;  // A0 values in SELL slot order
    bool spmv_sell = false;      // cgp_spmv uses the SELL kernel (cgp_autotune decides)

    // sliced ELL of the fine pattern in the natural row order (32-row slices, slot k of a slice's
    // rows contiguous), the layout of the fine-mesh Krylov solvers' products when ell_on
    bool ell_on = false;
    int ell_nslices = 0, ell_total = 0;
    int *ell_ptr = nullptr, *ell_col = nullptr, *ell_pos = nullptr;   // ell_pos: CSR entry -> slot
    int* ell_src = nullptr;                                            // slot -> CSR entry or -1
    double *ell_A = nullptr, *ell_M = nullptr;
    float *ell_A32 = nullptr, *ell_M32 = nullptr;

    // Galerkin restriction (restrict_mode 1): per level k the inverse child lists of the s^p
    // table (for each level-k node the finer nodes whose (beta, gamma) pair contains it) and the
    // fine divergence D_f u~_f
    std::vector<int*> gal_ptr, gal_idx, gal_self;   // gal_self: the coinciding finer node
    double* gal_div = nullptr;   // [nf]
    // incremental / rotational pressure correction (projection 1, 2)
    double* grad_n = nullptr;    // [nf][2] G_f P p_c^n, the momentum right-hand side's pressure term
    double* phi = nullptr;       // [nc] the pressure increment of the latest step
    double* mlump_c = nullptr;   // [nc] lumped coarse mass (row sums of the coarse P1 mass matrix)

    // diagnostic surfaces (cgp_set_surface): 0 the body of cgp_body_force, 1 the wall of
    // cgp_reattachment; boundary edges (a, b, owning fine triangle) and the wall's shear scratch
    struct Surface {
        int n = 0;
        int4* e = nullptr;
        double* xs = nullptr;    // [2 n]: edge midpoints x, then shear
    } surf[2];

    cgp::Shape sh_f, sh_c;       // persistent shapes for fine and coarse problems
    int width_c = 0;             // longest coarse CSR row
    bool use_pipe = false;       // coarse Poisson on an on-chip CG kernel
    bool onchip_pipelined = false;   // ... in its pipelined form (else classical)
    cgp::Shape pipe_c;           // its launch shape
    size_t pipe_smem64 = 0, pipe_smem32 = 0;

    // two-level Schwarz preconditioned coarse CG (coarse_solver 3 and 4)
    bool use_schwarz = false;
    bool schwarz_fp32 = false;   // preconditioner applied in FP32
    int sz_degree = 0;
    double sz_ratio = 0.0, sz_lmin = 0.0, sz_lmax = 0.0;
    int *sz_perm = nullptr, *sz_rp = nullptr, *sz_ci = nullptr;
    double *sz_val64 = nullptr, *sz_dinv64 = nullptr, *sz_ainv64 = nullptr;
    float *sz_val32 = nullptr, *sz_dinv32 = nullptr, *sz_ainv32 = nullptr;
    double* sz_fxy64 = nullptr;  // [n][2] linear coarse functions, renumbered
    float* sz_fxy32 = nullptr;
    std::vector<int> sz_src;     // renumbered CSR entry -> caller CSR entry
    std::vector<int> sz_rp_h, sz_ci_h;
    std::vector<double> sz_fxy_h;
    size_t sz_smem = 0;
    cgp::TwoLevel tl;            // batched two-level coarse CG
    cgp::ManyRhs many;           // multi-right-hand-side coarse solve
    std::vector<void*> allocs;   // everything to free
};

// A batch of independent contexts advanced together: one cooperative launch per persistent stage
// covers every instance, each on its own group of blocks.
struct cgp_batch_s {
    std::vector<cgp_ctx_s*> ctx;
    std::vector<double*> u, pc;          // per-instance state (caller device buffers)
    int n = 0, threads = 512, precision = CGP_FP64;
    int blocks_f = 0, blocks_c = 0, max_group = 1;
    std::vector<int> b0_f, nb_f, b0_c, nb_c;
    cgp::BatchMap map_f{nullptr, nullptr, nullptr}, map_c{nullptr, nullptr, nullptr};
    cgp::SyncWords* sync = nullptr;      // [n][SYNC_COUNT]
    double* part = nullptr;              // [n][32 * max_group]
    void* tab_asm = nullptr;             // device tables of per-instance kernel arguments
    void* tab_mom = nullptr;
    void* tab_poi = nullptr;
    void* tab_mass = nullptr;
    void* tab_poi2 = nullptr;            // two-level coarse CG arguments (poisson_2l)
    void* tab_predict = nullptr;         // coarse-pressure predictor arguments (warm_start = 1)
    bool predict = false;
    int predict_nmax = 0, predict_count = 0;
    bool poisson_2l = false;
    size_t smem_poi2 = 0;
    bool gather = false;                 // batched inter-stage gathers (one launch per stage)
    void* tab_gather = nullptr;
    int gather_nc = 0, gather_nf = 0, gather_levels = 0, gather_nlv = 0;
    void* tab_perm = nullptr;            // velocities gathered into the instances' stored fine order
    int perm_nmax = 0, perm_count = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    std::vector<void*> allocs;
};

namespace cgp {

// batch stages (assemble.cu, krylov.cu)
cudaError_t batch_asm_build(cgp_batch_s* b);
cudaError_t batch_asm_launch(cgp_batch_s* b, cudaStream_t s);
cudaError_t batch_solvers_build(cgp_batch_s* b);
cudaError_t batch_momentum_launch(cgp_batch_s* b, cudaStream_t s);
cudaError_t batch_poisson_launch(cgp_batch_s* b, cudaStream_t s);
cudaError_t batch_mass_launch(cgp_batch_s* b, cudaStream_t s);
// krylov_2l.cu
int twolevel_build(cgp_ctx_s* c);
bool batch_poisson2l_build(cgp_batch_s* b);
cudaError_t batch_poisson2l_launch(cgp_batch_s* b, cudaStream_t s);
int persistent_blocks_per_sm(int threads, bool batch);
int many_prepare(cgp_ctx_s* c);
int many_solve(cgp_ctx_s* c, int nrhs, const double* b, double* x, int* iters, double* rel, int* status,
               cudaStream_t s);

// assemble.cu
cudaError_t launch_geometry(const double* xy, const int* tri, int t, double* geo, cudaStream_t s);
cudaError_t launch_conv_scale(const double* geo, int t, double dtrho, double* conv, cudaStream_t s);
cudaError_t launch_const_assembly(const DevElems& E, double* M, double* K, double* Dxy, cudaStream_t s);
cudaError_t launch_apply_pressure_bc(cgp_ctx_s* c, cudaStream_t s);
cudaError_t launch_make_A0(cgp_ctx_s* c, const double* K, cudaStream_t s);
cudaError_t launch_assemble_step(cgp_ctx_s* c, const double* u, cudaStream_t s, const double* gpn = nullptr);
cudaError_t launch_assemble_step_coloured(cgp_ctx_s* c, const double* u, cudaStream_t s);
int assemble_gather_build(cgp_ctx_s* c);

// krylov.cu
cudaError_t launch_poisson_cg(cgp_ctx_s* c, const double* b, double* x, cudaStream_t s);
cudaError_t launch_mass_cg(cgp_ctx_s* c, const double* b, double* x, cudaStream_t s);
cudaError_t launch_momentum_bicgstab(cgp_ctx_s* c, const double* u_in, double* x, cudaStream_t s);
cudaError_t time_spmv_lanes(cgp_ctx_s* c, bool fine, int lanes, cudaStream_t s, float* ms);
cudaError_t launch_spmv_fine(cgp_ctx_s* c, const double* x, double* y, cudaStream_t s);
cudaError_t launch_spmv_sell(cgp_ctx_s* c, const double* x, double* y, cudaStream_t s);
// y = A32 x, the fine solvers' FP32 product in their launch shape and layout (two RHS)
cudaError_t launch_solver_spmv(cgp_ctx_s* c, const float* x, float* y, cudaStream_t s);
cudaError_t sell_fill(cgp_ctx_s* c, const double* csr_val, cudaStream_t s);
cudaError_t ell_fill(int total, const int* src, const double* csr_val, double* val, float* val32, cudaStream_t s);

// krylov_pipe.cu
bool pipe_shape(int n, int width, int num_sms, size_t elem, int* blocks, int* threads, size_t* smem);
cudaError_t pipe_prepare(cgp_ctx_s* c);
cudaError_t launch_poisson_pipe(cgp_ctx_s* c, const double* b, double* x, cudaStream_t s);
int schwarz_values(cgp_ctx_s* c);

// mapping.cu
cudaError_t launch_restrict_rhs(cgp_ctx_s* c, const double* ut, double* bc, cudaStream_t s);
cudaError_t launch_prolong(cgp_ctx_s* c, const double* pc, double* pf, cudaStream_t s);
cudaError_t launch_gradient(cgp_ctx_s* c, const double* pf, double* grad, cudaStream_t s);
cudaError_t launch_correct(cgp_ctx_s* c, const double* ut, const double* w, double* u, double* gp_out,
                           cudaStream_t s, bool to_public = false);
// fine vectors between the refinement order (the interface) and the stored order (fperm);
// comps = values per node (1 or 2); copies when the two orders coincide
cudaError_t fine_to_stored(cgp_ctx_s* c, const double* pub, double* st, int comps, cudaStream_t s);
cudaError_t fine_to_public(cgp_ctx_s* c, const double* st, double* pub, int comps, cudaStream_t s);
cudaError_t launch_copy_pairs(const double* src, double* dst, int n, cudaStream_t s);
cudaError_t launch_pressure_term(cgp_ctx_s* c, const double* pc, cudaStream_t s);
cudaError_t launch_pressure_update(cgp_ctx_s* c, const double* bc, const double* phi, double* pc, cudaStream_t s);
cudaError_t launch_lumped_mass(cgp_ctx_s* c, double* tmp_nnzc, cudaStream_t s);
int galerkin_build(cgp_ctx_s* c);
cudaError_t launch_predict(cgp_ctx_s* c, double* pc, cudaStream_t s);
cudaError_t launch_predict_vec(const double* in, double* out, double* prev, double* prev2, double* prev3, int* flag,
                               int n, int order, cudaStream_t s);
cudaError_t batch_predict_launch(cgp_batch_s* b, cudaStream_t s);
cudaError_t batch_predict_build(cgp_batch_s* b);
bool batch_gather_build(cgp_batch_s* b);
cudaError_t batch_restrict_launch(cgp_batch_s* b, cudaStream_t s);
cudaError_t batch_prolong_gradient_launch(cgp_batch_s* b, cudaStream_t s);
cudaError_t batch_correct_launch(cgp_batch_s* b, cudaStream_t s);
cudaError_t batch_perm_build(cgp_batch_s* b);
// The velocity an instance's batched kernels read: its stored-order copy when it renumbers.
inline double* batch_u_work(const cgp_batch_s* b, int i) { return b->ctx[i]->fperm ? b->ctx[i]->u_int : b->u[i]; }
cudaError_t batch_perm_launch(cgp_batch_s* b, cudaStream_t s);

// Cooperative launch helper: launches `func` with the shape, `smem` bytes of dynamic shared
// memory and its single by-value argument (typed, so a kernel cannot be handed the wrong
// argument structure).
template <typename Args>
cudaError_t coop_launch(void (*func)(Args), int blocks, int threads, Args& args, cudaStream_t s, size_t smem = 0) {
    void* kargs[] = {(void*)&args};
    if (blocks == 1) return cudaLaunchKernel((const void*)func, dim3(1), dim3(threads), kargs, smem, s);
    return cudaLaunchCooperativeKernel((const void*)func, dim3(blocks), dim3(threads), kargs, smem, s);
}

}  // namespace cgp
