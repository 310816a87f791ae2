// Learned warm start for the coarse Poisson solve (a systems pattern around Eq. 21, not in the
// paper): a BF16 network n -> H -> H -> n with GELU, trained and run by the project's own
// kernels. The contractions are tcgen05 tensor-core GEMMs (sm_100-family): operands are moved by
// TMA into 128-byte-swizzled shared-memory tiles through a 4-stage mbarrier pipeline, one thread
// issues tcgen05.mma into a TMEM accumulator, and four warps read it back with tcgen05.ld for a
// fused epilogue (bias, GELU, GELU derivative, BF16 conversion).
//
// Network (per right-hand side b, n entries): s = ||b||, x = b/s, z1 = W1 x + b1, h1 = gelu(z1),
// z2 = W2 h1 + b2, h2 = gelu(z2), y = W3 h2 + b3, p = s y (pressure-held entries 0);
// gelu(z) = z/2 (1 + tanh(c (z + 0.044715 z^3))), c = sqrt(2/pi) (Hendrycks & Gimpel 2016).
// Loss 1/(B n) sum m (y - p_true/s)^2, Adam (Kingma & Ba 2015) on FP32 master weights.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "ctx.h"

namespace cgp {
namespace {

constexpr int GM = 128;                       // tile rows = MMA M
constexpr int GN = 128;                       // tile columns = MMA N = TMEM columns
constexpr int GK = 64;                        // K per stage: one 128-byte swizzle row of bf16
constexpr int STAGES = 4;
constexpr int A_BYTES = GM * GK * 2;
constexpr int B_BYTES = GN * GK * 2;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int GEMM_SMEM = STAGES * STAGE_BYTES + 1024;   // + slack for 1024-byte alignment
constexpr uint32_t WAIT_LIMIT = 1u << 20;    // try_wait may suspend per attempt: about a second

enum { EPI_F32 = 0, EPI_GELU = 1, EPI_GELU_BWD = 2, EPI_RAW = 3 /* split-K partial, no bias */ };

struct GemmArgs {
    int M, N, K;
    int epi;
    const float* bias;          // [N] or nullptr
    float* out_f32;             // [M][ldo]: result (EPI_F32), z (EPI_GELU), dz (EPI_GELU_BWD)
    __nv_bfloat16* out_bf16;    // [M][ldo]: gelu(z) (EPI_GELU), dz (EPI_GELU_BWD), optional
    const float* zin;           // [M][ldo] pre-activation for EPI_GELU_BWD
    int ldo;
    int* err;
    int splits;                 // K split across blockIdx.z (EPI_RAW: partial z at out_f32 + z M ldo)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Wait until the phase with the given parity of the mbarrier has completed; false after the limit.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t i = 0; i < WAIT_LIMIT; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred P;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, P;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile in the 128-byte-swizzled canonical layout:
// rows of 128 bytes, 8-row groups 1024 bytes apart (stride byte offset), version 1, swizzle 128B.
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;                   // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset
    d |= (uint64_t)1 << 46;                   // descriptor version
    d |= (uint64_t)2 << 61;                   // 128-byte swizzle
    return d;
}

// Instruction descriptor of kind::f16: D f32, A and B bf16, both K-major, M = GM, N = GN.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(GN >> 3) << 17) | ((uint32_t)(GM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ float gelu_f(float z) {
    const float c = 0.7978845608028654f, a = 0.044715f;
    return 0.5f * z * (1.0f + tanhf(c * (z + a * z * z * z)));
}

__device__ __forceinline__ float gelu_grad_f(float z) {
    const float c = 0.7978845608028654f, a = 0.044715f;
    const float t = tanhf(c * (z + a * z * z * z));
    return 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * c * (1.0f + 3.0f * a * z * z);
}

// C[M, N] = A[M, K] * B[N, K]^T, A and B bf16 row-major with K contiguous (K-major), fp32
// accumulation in TMEM. One CTA of 4 warps per 128 x 128 output tile and K range: with
// g.splits > 1, CTA z of a tile takes its share of the 64-wide K blocks and stores the raw
// partial tile (EPI_RAW); k_splitk_reduce adds the partials in order and applies the epilogue.
__global__ void __launch_bounds__(128, 1) k_gemm_tn(const __grid_constant__ CUtensorMap tmA,
                                                    const __grid_constant__ CUtensorMap tmB, GemmArgs g) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[STAGES];
    __shared__ __align__(8) uint64_t empty_bar[STAGES];
    __shared__ __align__(8) uint64_t done_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int s_fail, s_issued, s_consumed;
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * GM, n0 = blockIdx.x * GN;
    const int nk_all = g.K / GK, per = (nk_all + g.splits - 1) / g.splits;
    const int kb0 = min(nk_all, (int)blockIdx.z * per);
    const int nk = min(nk_all, kb0 + per) - kb0;     // >= 1: the host drops empty splits
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        mbar_init(smem_u32(&done_bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        s_fail = 0;
        s_issued = 0;
        s_consumed = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(GN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tmem_slot;

    // Warp 0 lane 0 produces (TMA), warp 1 lane 0 issues the MMAs; the other lanes of those two
    // warps wait converged at __syncwarp rather than polling the completion barrier, which would
    // share the warp's issue slots with the producer or issuer lane.
    if (warp == 0) {
        if (lane == 0) {
            // TMA producer
            for (int kb = 0; kb < nk; ++kb) {
                const int s = kb % STAGES;
                if (kb >= STAGES && !mbar_wait(smem_u32(&empty_bar[s]), ((kb / STAGES) & 1) ^ 1)) {
                    s_fail = 1;
                    break;
                }
                if (s_fail) break;
                const uint32_t fb = smem_u32(&full_bar[s]);
                mbar_expect_tx(fb, STAGE_BYTES);
                const uint32_t sa = smem_u32(smem + (size_t)s * STAGE_BYTES);
                tma_load_2d(sa, &tmA, (kb0 + kb) * GK, m0, fb);
                tma_load_2d(sa + A_BYTES, &tmB, (kb0 + kb) * GK, n0, fb);
                s_issued = kb + 1;
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer
            for (int kb = 0; kb < nk; ++kb) {
                const int s = kb % STAGES;
                if (!mbar_wait(smem_u32(&full_bar[s]), (kb / STAGES) & 1)) {
                    s_fail = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t sa = smem_u32(smem + (size_t)s * STAGE_BYTES);
#pragma unroll
                for (int k = 0; k < GK / 16; ++k)
                    mma_bf16(tbase, umma_desc(sa + 32 * k), umma_desc(sa + A_BYTES + 32 * k), (kb > 0 || k > 0) ? 1u : 0u);
                mma_commit(smem_u32(&empty_bar[s]));
                s_consumed = kb + 1;
            }
            mma_commit(smem_u32(&done_bar));
        }
        __syncwarp();
    }
    // epilogue: warp w owns TMEM lanes (rows) 32w .. 32w+31
    if (!mbar_wait(smem_u32(&done_bar), 0)) s_fail = 1;
    tc_fence_after();
    __syncthreads();
    if (!s_fail) {
        const int row = m0 + warp * 32 + lane;
        const uint32_t lane_base = tbase + ((uint32_t)(warp * 32) << 16);
        for (int c = 0; c < GN; c += 16) {
            uint32_t r[16];
            tmem_ld16(lane_base + c, r);
            const int col0 = n0 + c;
            const size_t o = (size_t)row * g.ldo + col0;
            float v[16];
            if (g.epi == EPI_RAW) {
                float* dst = g.out_f32 + (size_t)blockIdx.z * g.M * g.ldo + o;
#pragma unroll
                for (int j = 0; j < 16; j += 4)
                    *reinterpret_cast<float4*>(dst + j) = make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                                                                      __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]));
                continue;
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]) + (g.bias ? g.bias[col0 + j] : 0.0f);
            if (g.epi == EPI_F32) {
#pragma unroll
                for (int j = 0; j < 16; j += 4)
                    *reinterpret_cast<float4*>(g.out_f32 + o + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
            } else {
                __nv_bfloat16 hb[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    float outv;
                    if (g.epi == EPI_GELU) {
                        outv = gelu_f(v[j]);
                    } else {
                        v[j] = v[j] * gelu_grad_f(g.zin[o + j]);
                        outv = v[j];
                    }
                    hb[j] = __float2bfloat16_rn(outv);
                }
                if (g.out_f32) {
#pragma unroll
                    for (int j = 0; j < 16; j += 4)
                        *reinterpret_cast<float4*>(g.out_f32 + o + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                }
                if (g.out_bf16) {
                    *reinterpret_cast<uint4*>(g.out_bf16 + o) = *reinterpret_cast<const uint4*>(&hb[0]);
                    *reinterpret_cast<uint4*>(g.out_bf16 + o + 8) = *reinterpret_cast<const uint4*>(&hb[8]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (s_fail && threadIdx.x == 0) {
        atomicExch(g.err, CGP_ERR_TIMEOUT);
        // let every copy this CTA issued land before its shared memory goes away (bounded)
        for (int kb = s_consumed; kb < s_issued; ++kb) mbar_wait(smem_u32(&full_bar[kb % STAGES]), (kb / STAGES) & 1);
    }
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(GN) : "memory");
}

// Sum of the split-K partials W[z][M][N] (z in order, so the result does not depend on timing),
// then bias and the epilogue of g, four outputs per thread.
__global__ void k_splitk_reduce(const float* __restrict__ W, int splits, GemmArgs g) {
    const size_t i4 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t total = (size_t)g.M * g.N;
    if (i4 * 4 >= total) return;
    const size_t o = i4 * 4;
    const int col = (int)(o % g.N), row = (int)(o / g.N);
    float4 acc = *reinterpret_cast<const float4*>(W + o);
    for (int z = 1; z < splits; ++z) {
        const float4 q = *reinterpret_cast<const float4*>(W + (size_t)z * total + o);
        acc.x += q.x;
        acc.y += q.y;
        acc.z += q.z;
        acc.w += q.w;
    }
    float v[4] = {acc.x, acc.y, acc.z, acc.w};
    const size_t oo = (size_t)row * g.ldo + col;
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] += g.bias ? g.bias[col + j] : 0.0f;
    if (g.epi == EPI_F32) {
        *reinterpret_cast<float4*>(g.out_f32 + oo) = make_float4(v[0], v[1], v[2], v[3]);
        return;
    }
    __nv_bfloat16 hb[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float outv;
        if (g.epi == EPI_GELU) {
            outv = gelu_f(v[j]);
        } else {
            v[j] = v[j] * gelu_grad_f(g.zin[oo + j]);
            outv = v[j];
        }
        hb[j] = __float2bfloat16_rn(outv);
    }
    if (g.out_f32) *reinterpret_cast<float4*>(g.out_f32 + oo) = make_float4(v[0], v[1], v[2], v[3]);
    if (g.out_bf16) *reinterpret_cast<uint2*>(g.out_bf16 + oo) = *reinterpret_cast<const uint2*>(&hb[0]);
}

// ---- host side of the GEMM -----------------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::mutex g_encode_mu;

cudaError_t get_encoder() {
    std::lock_guard<std::mutex> lock(g_encode_mu);
    if (g_encode) return cudaSuccess;
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return e != cudaSuccess ? e : cudaErrorUnknown;
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    return cudaSuccess;
}

// 2-D bf16 tensor map over a row-major [rows][cols] matrix, box 64 x 128, 128-byte swizzle.
cudaError_t make_map(CUtensorMap* m, const void* ptr, int rows, int cols) {
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)GK, 128u};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

bool g_gemm_attr = false;

// Number of K splits for an M x N x K product: enough CTAs to cover the SMs when the output has
// few tiles, at least two 64-wide K blocks per split, and no more than the workspace holds.
int choose_splits(int M, int N, int K, int num_sms, size_t work_floats) {
    const int tiles = (M / GM) * (N / GN), nk = K / GK;
    int sp = std::max(1, std::min(num_sms / std::max(1, tiles), nk / 2));
    while (sp > 1 && (size_t)sp * M * N > work_floats) --sp;
    if (sp > 1) {
        const int per = (nk + sp - 1) / sp;
        sp = (nk + per - 1) / per;   // no empty split
    }
    return sp;
}

// C[M,N] = A[M,K] B[N,K]^T with the requirements M % 128 == 0, N % 128 == 0, K % 64 == 0,
// 16-byte aligned A, B, C. With a workspace (work, work_floats), a product with few output tiles
// is split along K across more CTAs and reduced by k_splitk_reduce.
cudaError_t gemm_tn(const __nv_bfloat16* A, const __nv_bfloat16* B, const GemmArgs& ga_in, cudaStream_t s,
                    float* work = nullptr, size_t work_floats = 0, int num_sms = 0) {
    GemmArgs ga = ga_in;
    ga.splits = 1;
    if (ga.M % GM || ga.N % GN || ga.K % GK || ga.M <= 0 || ga.N <= 0 || ga.K <= 0) return cudaErrorInvalidValue;
    if (((uintptr_t)A | (uintptr_t)B) & 15) return cudaErrorInvalidValue;
    cudaError_t e = get_encoder();
    if (e != cudaSuccess) return e;
    if (!g_gemm_attr) {
        e = cudaFuncSetAttribute((const void*)k_gemm_tn, cudaFuncAttributeMaxDynamicSharedMemorySize, GEMM_SMEM);
        if (e != cudaSuccess) return e;
        g_gemm_attr = true;
    }
    CUtensorMap ma, mb;
    if ((e = make_map(&ma, A, ga.M, ga.K)) != cudaSuccess) return e;
    if ((e = make_map(&mb, B, ga.N, ga.K)) != cudaSuccess) return e;
    const int sp = work ? choose_splits(ga.M, ga.N, ga.K, num_sms, work_floats) : 1;
    if (sp <= 1) {
        dim3 grid(ga.N / GN, ga.M / GM);
        k_gemm_tn<<<grid, 128, GEMM_SMEM, s>>>(ma, mb, ga);
        return cudaGetLastError();
    }
    GemmArgs gp = ga;
    gp.epi = EPI_RAW;
    gp.out_f32 = work;
    gp.out_bf16 = nullptr;
    gp.bias = nullptr;
    gp.ldo = ga.N;
    gp.splits = sp;
    dim3 grid(ga.N / GN, ga.M / GM, sp);
    k_gemm_tn<<<grid, 128, GEMM_SMEM, s>>>(ma, mb, gp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t quads = (size_t)ga.M * ga.N / 4;
    k_splitk_reduce<<<(unsigned)((quads + 255) / 256), 256, 0, s>>>(work, sp, ga);
    return cudaGetLastError();
}

// ---- network kernels ------------------------------------------------------------------------

// Per right-hand side row r < B: s = ||b_r||, X[r][j] = bf16(b_rj / s) (0 beyond n), and for
// training T[r][j] = p_rj / s. Rows r >= B are zero. One block per row of the padded batch.
__global__ void k_prep(int B, int n, int np, const double* __restrict__ b, const double* __restrict__ p,
                       __nv_bfloat16* X, float* T, float* S) {
    __shared__ double red[32];
    const int r = blockIdx.x;
    double acc = 0.0;
    if (r < B)
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const double v = b[(size_t)r * n + j];
            acc += v * v;
        }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) red[0] = t;
    }
    __syncthreads();
    const double nrm = sqrt(red[0]);
    const double inv = nrm > 0.0 ? 1.0 / nrm : 1.0;
    if (threadIdx.x == 0) S[r] = r < B ? (float)(nrm > 0.0 ? nrm : 1.0) : 0.0f;
    for (int j = threadIdx.x; j < np; j += blockDim.x) {
        const bool in = r < B && j < n;
        X[(size_t)r * np + j] = __float2bfloat16_rn(in ? (float)(b[(size_t)r * n + j] * inv) : 0.0f);
        if (T) T[(size_t)r * np + j] = (in && p) ? (float)(p[(size_t)r * n + j] * inv) : 0.0f;
    }
}

// out[c][r] = in[r][c] for a [R][C] bf16 matrix (32 x 32 tiles through shared memory).
__global__ void k_transpose_bf16(int R, int C, const __nv_bfloat16* __restrict__ in, __nv_bfloat16* __restrict__ out) {
    __shared__ __nv_bfloat16 t[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = r0 + k, c = c0 + threadIdx.x;
        if (r < R && c < C) t[k][threadIdx.x] = in[(size_t)r * C + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int c = c0 + k, r = r0 + threadIdx.x;
        if (r < R && c < C) out[(size_t)c * R + r] = t[threadIdx.x][k];
    }
}

// dY = 2/(B n_valid) (Y - T) on rows < B and unmasked columns, else 0; bf16 copy; loss partials.
__global__ void k_loss_grad(int B, int np, int n, const unsigned char* __restrict__ mask, float scale,
                            const float* __restrict__ Y, const float* __restrict__ T, float* dY,
                            __nv_bfloat16* dYb, double* loss_part) {
    __shared__ double red[32];
    const int r = blockIdx.x;
    double acc = 0.0;
    for (int j = threadIdx.x; j < np; j += blockDim.x) {
        const size_t o = (size_t)r * np + j;
        float d = 0.0f;
        if (r < B && j < n && !mask[j]) {
            const float diff = Y[o] - T[o];
            acc += (double)diff * diff;
            d = scale * diff;
        }
        dY[o] = d;
        dYb[o] = __float2bfloat16_rn(d);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        loss_part[r] = t;
    }
}

// loss = sum(parts) / (B n_valid), fixed order.
__global__ void k_loss_final(int rows, const double* parts, double denom, float* loss) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double t = 0.0;
        for (int r = 0; r < rows; ++r) t += parts[r];
        *loss = (float)(t / denom);
    }
}

// column sums over the first B rows of a [R][C] f32 matrix (bias gradients), fixed order.
__global__ void k_colsum(int B, int C, const float* __restrict__ in, float* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    float t = 0.0f;
    for (int r = 0; r < B; ++r) t += in[(size_t)r * C + c];
    out[c] = t;
}

// Adam on FP32 master weights (bias-corrected), entries with keep[i] == 0 held at zero; writes
// the bf16 copy used by the products (and its transpose when Wt != nullptr, rows x cols = R x C).
__global__ void k_adam(size_t count, int C, float* w, float* m, float* v, const float* __restrict__ gr,
                       const unsigned char* keep_col, const unsigned char* keep_row, float lr, float b1, float b2,
                       float bc1, float bc2, float eps, __nv_bfloat16* wb, __nv_bfloat16* wt, int R) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int r = (int)(i / C), c = (int)(i % C);
    const bool keep = (!keep_col || keep_col[c]) && (!keep_row || keep_row[r]);
    float wi = 0.0f;
    if (keep) {
        const float gi = gr[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        wi = w[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16_rn(wi);
    if (wt) wt[(size_t)c * R + r] = __float2bfloat16_rn(wi);
}

// bf16 copies (and transpose) of an FP32 master matrix.
__global__ void k_to_bf16(size_t count, int C, int R, const float* __restrict__ w, __nv_bfloat16* wb, __nv_bfloat16* wt) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int r = (int)(i / C), c = (int)(i % C);
    if (wb) wb[i] = __float2bfloat16_rn(w[i]);
    if (wt) wt[(size_t)c * R + r] = __float2bfloat16_rn(w[i]);
}

// Residual form: r[i] = b[i] - (K x_base)[i] for every right-hand side of the batch (row-major
// [B][n], one thread per entry, the coarse CSR matrix after the elimination of held rows), and with
// p the training target c[i] = p[i] - x_base[i].
__global__ void k_base_residual(int B, int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                const double* __restrict__ K, const double* __restrict__ b,
                                const double* __restrict__ base, const double* __restrict__ p, double* __restrict__ r,
                                double* __restrict__ c) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)B * n) return;
    const size_t r0 = i / n * n;
    const int row = (int)(i - r0);
    double kx = 0.0;
    for (int k = rp[row]; k < rp[row + 1]; ++k) kx += K[k] * base[r0 + ci[k]];
    r[i] = b[i] - kx;
    if (p) c[i] = p[i] - base[i];
}

// Residual form output: p = x_base + S[r] Y[r][j] (x_base alone at pressure-held entries).
__global__ void k_output_add(int B, int n, int np, const unsigned char* __restrict__ mask, const float* __restrict__ S,
                             const float* __restrict__ Y, const double* __restrict__ base, double* p) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)B * n) return;
    const int r = (int)(i / n), j = (int)(i % n);
    p[i] = base[i] + (mask[j] ? 0.0 : (double)S[r] * (double)Y[(size_t)r * np + j]);
}

// p[r][j] = S[r] * Y[r][j] (0 at pressure-held entries), r < B, j < n.
__global__ void k_output(int B, int n, int np, const unsigned char* __restrict__ mask, const float* __restrict__ S,
                         const float* __restrict__ Y, double* p) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)B * n) return;
    const int r = (int)(i / n), j = (int)(i % n);
    p[i] = mask[j] ? 0.0 : (double)S[r] * (double)Y[(size_t)r * np + j];
}

}  // namespace
}  // namespace cgp

using namespace cgp;

// ---- the network object -----------------------------------------------------------------------

struct cgp_ws_s {
    int n = 0, np = 0, H = 0, bmax = 0, bp = 0;
    int n_free = 0;                 // unmasked outputs counted by the loss
    long long step = 0;
    std::vector<void*> allocs;
    int* err = nullptr;
    // masters and Adam moments (f32), bf16 copies
    float *W1, *b1, *W2, *b2, *W3, *b3;
    float *mW1, *vW1, *mb1, *vb1, *mW2, *vW2, *mb2, *vb2, *mW3, *vW3, *mb3, *vb3;
    __nv_bfloat16 *W1b, *W2b, *W2t, *W3b, *W3t;
    // activations
    __nv_bfloat16 *X, *Xt, *H1, *H1t, *H2, *H2t, *dYb, *dYt, *dZ2b, *dZ2t, *dZ1b, *dZ1t;
    float *T, *S, *Z1, *Z2, *Y, *dY, *dZ2, *dZ1;
    // gradients
    float *gW1, *gb1, *gW2, *gb2, *gW3, *gb3;
    double* loss_part;
    float* loss;
    // residual form: r = b - K_c x_base and the correction target p - x_base, [bmax][n] (lazily)
    double *res = nullptr, *cor = nullptr;
    unsigned char *mask, *keep_n, *keep_all;
    // split-K workspace of the GEMMs with few output tiles
    float* work = nullptr;
    size_t work_floats = 0;
    int num_sms = 0;
};

namespace {

template <typename T>
int walloc(cgp_ws_s* w, T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? CGP_ERR_NOMEM : CGP_ERR_CUDA;
    w->allocs.push_back(q);
    cudaMemset(q, 0, std::max<size_t>(count, 1) * sizeof(T));
    *p = (T*)q;
    return CGP_OK;
}

int ws_create(cgp_ws_s* w, int n, int H, int bmax) {
    w->n = n;
    w->n_free = n;
    w->np = ((n + 127) / 128) * 128;
    w->H = H;
    w->bmax = bmax;
    w->bp = ((bmax + 127) / 128) * 128;
    const size_t np = w->np, h = H, bp = w->bp;
    int s = CGP_OK;
#define A(ptr, cnt) \
    if ((s = walloc(w, &(ptr), (cnt)))) return s
    A(w->err, 1);
    A(w->W1, h * np); A(w->b1, h); A(w->W2, h * h); A(w->b2, h); A(w->W3, np * h); A(w->b3, np);
    A(w->mW1, h * np); A(w->vW1, h * np); A(w->mb1, h); A(w->vb1, h);
    A(w->mW2, h * h); A(w->vW2, h * h); A(w->mb2, h); A(w->vb2, h);
    A(w->mW3, np * h); A(w->vW3, np * h); A(w->mb3, np); A(w->vb3, np);
    A(w->W1b, h * np); A(w->W2b, h * h); A(w->W2t, h * h); A(w->W3b, np * h); A(w->W3t, h * np);
    A(w->X, bp * np); A(w->Xt, np * bp); A(w->H1, bp * h); A(w->H1t, h * bp); A(w->H2, bp * h); A(w->H2t, h * bp);
    A(w->dYb, bp * np); A(w->dYt, np * bp); A(w->dZ2b, bp * h); A(w->dZ2t, h * bp); A(w->dZ1b, bp * h);
    A(w->dZ1t, h * bp);
    A(w->T, bp * np); A(w->S, bp); A(w->Z1, bp * h); A(w->Z2, bp * h); A(w->Y, bp * np); A(w->dY, bp * np);
    A(w->dZ2, bp * h); A(w->dZ1, bp * h);
    A(w->gW1, h * np); A(w->gb1, h); A(w->gW2, h * h); A(w->gb2, h); A(w->gW3, np * h); A(w->gb3, np);
    A(w->loss_part, bp); A(w->loss, 1);
    A(w->mask, np); A(w->keep_n, np); A(w->keep_all, np > h ? np : h);
    w->work_floats = 32 * std::max(bp * h, h * h);
    A(w->work, w->work_floats);
#undef A
    {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&w->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return CGP_ERR_CUDA;
    }
    std::vector<unsigned char> kn(np, 0), ka(std::max(np, h), 1);
    for (int j = 0; j < n; ++j) kn[j] = 1;
    std::vector<unsigned char> mk(np, 1);
    for (int j = 0; j < n; ++j) mk[j] = 0;
    if (cudaMemcpy(w->keep_n, kn.data(), np, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(w->keep_all, ka.data(), ka.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(w->mask, mk.data(), np, cudaMemcpyHostToDevice) != cudaSuccess)
        return CGP_ERR_CUDA;
    return CGP_OK;
}

GemmArgs gargs(int M, int N, int K, int epi, const float* bias, float* of, __nv_bfloat16* ob, const float* zin,
               int ldo, int* err) {
    GemmArgs g;
    g.M = M; g.N = N; g.K = K; g.epi = epi; g.bias = bias; g.out_f32 = of; g.out_bf16 = ob; g.zin = zin;
    g.ldo = ldo; g.err = err; g.splits = 1;
    return g;
}

cudaError_t transpose(int R, int C, const __nv_bfloat16* in, __nv_bfloat16* out, cudaStream_t s) {
    dim3 grid((C + 31) / 32, (R + 31) / 32), block(32, 8);
    k_transpose_bf16<<<grid, block, 0, s>>>(R, C, in, out);
    return cudaGetLastError();
}

cudaError_t refresh_bf16(cgp_ws_s* w, cudaStream_t s) {
    const size_t h = w->H, np = w->np;
    k_to_bf16<<<(unsigned)((h * np + 255) / 256), 256, 0, s>>>(h * np, (int)np, (int)h, w->W1, w->W1b, nullptr);
    k_to_bf16<<<(unsigned)((h * h + 255) / 256), 256, 0, s>>>(h * h, (int)h, (int)h, w->W2, w->W2b, w->W2t);
    k_to_bf16<<<(unsigned)((np * h + 255) / 256), 256, 0, s>>>(np * h, (int)h, (int)np, w->W3, w->W3b, w->W3t);
    return cudaGetLastError();
}

cudaError_t forward(cgp_ws_s* w, const double* b, const double* p, int B, cudaStream_t s) {
    const int np = w->np, H = w->H, bp = ((B + 127) / 128) * 128;
    k_prep<<<bp, 256, 0, s>>>(B, w->n, np, b, p, w->X, p ? w->T : nullptr, w->S);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = gemm_tn(w->X, w->W1b, gargs(bp, H, np, EPI_GELU, w->b1, w->Z1, w->H1, nullptr, H, w->err), s, w->work, w->work_floats, w->num_sms);
    if (e == cudaSuccess) e = gemm_tn(w->H1, w->W2b, gargs(bp, H, H, EPI_GELU, w->b2, w->Z2, w->H2, nullptr, H, w->err), s, w->work, w->work_floats, w->num_sms);
    if (e == cudaSuccess) e = gemm_tn(w->H2, w->W3b, gargs(bp, np, H, EPI_F32, w->b3, w->Y, nullptr, nullptr, np, w->err), s, w->work, w->work_floats, w->num_sms);
    return e;
}

cudaError_t adam(cgp_ws_s* w, size_t count, int C, int R, float* P, float* M, float* V, const float* G,
                 const unsigned char* kc, const unsigned char* kr, float lr, __nv_bfloat16* wb, __nv_bfloat16* wt,
                 cudaStream_t s) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float bc1 = 1.0f - powf(b1, (float)w->step), bc2 = 1.0f - powf(b2, (float)w->step);
    k_adam<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(count, C, P, M, V, G, kc, kr, lr, b1, b2, bc1, bc2, 1e-8f,
                                                            wb, wt, R);
    return cudaGetLastError();
}

cudaError_t train_step(cgp_ws_s* w, const double* b, const double* p, int B, float lr, cudaStream_t s) {
    const int np = w->np, H = w->H, bp = ((B + 127) / 128) * 128;
    cudaError_t e = forward(w, b, p, B, s);
    if (e != cudaSuccess) return e;
    // L = 1/(B n_free) sum (y - t)^2 over unmasked entries, dL/dy = 2 (y - t) / (B n_free)
    const double den = (double)B * (double)w->n_free;
    k_loss_grad<<<bp, 256, 0, s>>>(B, np, w->n, w->mask, (float)(2.0 / den), w->Y, w->T, w->dY, w->dYb, w->loss_part);
    k_loss_final<<<1, 32, 0, s>>>(bp, w->loss_part, den, w->loss);
    k_colsum<<<(np + 255) / 256, 256, 0, s>>>(B, np, w->dY, w->gb3);
    if ((e = transpose(bp, np, w->dYb, w->dYt, s)) != cudaSuccess) return e;
    if ((e = transpose(bp, H, w->H2, w->H2t, s)) != cudaSuccess) return e;
    if ((e = transpose(bp, H, w->H1, w->H1t, s)) != cudaSuccess) return e;
    if ((e = transpose(bp, np, w->X, w->Xt, s)) != cudaSuccess) return e;
    // dW3 = dY^T h2 ; dz2 = (dY W3) * gelu'(z2)
    if ((e = gemm_tn(w->dYt, w->H2t, gargs(np, H, bp, EPI_F32, nullptr, w->gW3, nullptr, nullptr, H, w->err), s, w->work, w->work_floats, w->num_sms))) return e;
    if ((e = gemm_tn(w->dYb, w->W3t, gargs(bp, H, np, EPI_GELU_BWD, nullptr, w->dZ2, w->dZ2b, w->Z2, H, w->err), s, w->work, w->work_floats, w->num_sms)))
        return e;
    k_colsum<<<(H + 255) / 256, 256, 0, s>>>(B, H, w->dZ2, w->gb2);
    if ((e = transpose(bp, H, w->dZ2b, w->dZ2t, s)) != cudaSuccess) return e;
    // dW2 = dz2^T h1 ; dz1 = (dz2 W2) * gelu'(z1)
    if ((e = gemm_tn(w->dZ2t, w->H1t, gargs(H, H, bp, EPI_F32, nullptr, w->gW2, nullptr, nullptr, H, w->err), s, w->work, w->work_floats, w->num_sms))) return e;
    if ((e = gemm_tn(w->dZ2b, w->W2t, gargs(bp, H, H, EPI_GELU_BWD, nullptr, w->dZ1, w->dZ1b, w->Z1, H, w->err), s, w->work, w->work_floats, w->num_sms)))
        return e;
    k_colsum<<<(H + 255) / 256, 256, 0, s>>>(B, H, w->dZ1, w->gb1);
    if ((e = transpose(bp, H, w->dZ1b, w->dZ1t, s)) != cudaSuccess) return e;
    // dW1 = dz1^T x
    if ((e = gemm_tn(w->dZ1t, w->Xt, gargs(H, np, bp, EPI_F32, nullptr, w->gW1, nullptr, nullptr, np, w->err), s, w->work, w->work_floats, w->num_sms)))
        return e;
    if (lr <= 0.0f) return cudaSuccess;     // gradients only
    w->step += 1;
    const size_t h = H;
    if ((e = adam(w, h * np, np, H, w->W1, w->mW1, w->vW1, w->gW1, w->keep_n, nullptr, lr, w->W1b, nullptr, s))) return e;
    if ((e = adam(w, h, H, 1, w->b1, w->mb1, w->vb1, w->gb1, nullptr, nullptr, lr, nullptr, nullptr, s))) return e;
    if ((e = adam(w, h * h, H, H, w->W2, w->mW2, w->vW2, w->gW2, nullptr, nullptr, lr, w->W2b, w->W2t, s))) return e;
    if ((e = adam(w, h, H, 1, w->b2, w->mb2, w->vb2, w->gb2, nullptr, nullptr, lr, nullptr, nullptr, s))) return e;
    if ((e = adam(w, (size_t)np * h, H, np, w->W3, w->mW3, w->vW3, w->gW3, nullptr, w->keep_n, lr, w->W3b, w->W3t, s)))
        return e;
    if ((e = adam(w, np, np, 1, w->b3, w->mb3, w->vb3, w->gb3, w->keep_n, nullptr, lr, nullptr, nullptr, s))) return e;
    return cudaSuccess;
}

}  // namespace

// ---- C ABI -------------------------------------------------------------------------------------

namespace {
__device__ int g_gemm_err;
int* gemm_err_ptr() {
    static std::mutex mu;
    static int* p[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!p[dev]) {
        void* q = nullptr;
        if (cudaGetSymbolAddress(&q, g_gemm_err) != cudaSuccess) return nullptr;
        p[dev] = (int*)q;
    }
    return p[dev];
}

int ws_upload_params(cgp_ws_s* w, const float* W1, const float* b1, const float* W2, const float* b2, const float* W3,
                     const float* b3) {
    const int n = w->n, np = w->np, H = w->H;
    std::vector<float> t1((size_t)H * np, 0.0f), t3((size_t)np * H, 0.0f), tb3(np, 0.0f);
    for (int r = 0; r < H; ++r) std::memcpy(&t1[(size_t)r * np], W1 + (size_t)r * n, sizeof(float) * n);
    std::memcpy(t3.data(), W3, sizeof(float) * (size_t)n * H);
    std::memcpy(tb3.data(), b3, sizeof(float) * n);
    if (cudaMemcpy(w->W1, t1.data(), sizeof(float) * t1.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(w->b1, b1, sizeof(float) * H, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(w->W2, W2, sizeof(float) * (size_t)H * H, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(w->b2, b2, sizeof(float) * H, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(w->W3, t3.data(), sizeof(float) * t3.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(w->b3, tb3.data(), sizeof(float) * np, cudaMemcpyHostToDevice) != cudaSuccess)
        return CGP_ERR_CUDA;
    float* moments[] = {w->mW1, w->vW1, w->mb1, w->vb1, w->mW2, w->vW2, w->mb2, w->vb2, w->mW3, w->vW3, w->mb3, w->vb3};
    size_t sizes[] = {(size_t)H * np, (size_t)H * np, (size_t)H, (size_t)H, (size_t)H * H, (size_t)H * H, (size_t)H,
                      (size_t)H, (size_t)np * H, (size_t)np * H, (size_t)np, (size_t)np};
    for (int k = 0; k < 12; ++k)
        if (cudaMemset(moments[k], 0, sizeof(float) * sizes[k]) != cudaSuccess) return CGP_ERR_CUDA;
    w->step = 0;
    if (refresh_bf16(w, 0) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return CGP_ERR_CUDA;
    return CGP_OK;
}

int ws_download(cgp_ws_s* w, const float* dW1, const float* db1, const float* dW2, const float* db2, const float* dW3,
                const float* db3, float* W1, float* b1, float* W2, float* b2, float* W3, float* b3) {
    const int n = w->n, np = w->np, H = w->H;
    if (cudaDeviceSynchronize() != cudaSuccess) return CGP_ERR_CUDA;
    std::vector<float> t1((size_t)H * np);
    if (W1) {
        if (cudaMemcpy(t1.data(), dW1, sizeof(float) * t1.size(), cudaMemcpyDeviceToHost) != cudaSuccess) return CGP_ERR_CUDA;
        for (int r = 0; r < H; ++r) std::memcpy(W1 + (size_t)r * n, &t1[(size_t)r * np], sizeof(float) * n);
    }
    if ((b1 && cudaMemcpy(b1, db1, sizeof(float) * H, cudaMemcpyDeviceToHost) != cudaSuccess) ||
        (W2 && cudaMemcpy(W2, dW2, sizeof(float) * (size_t)H * H, cudaMemcpyDeviceToHost) != cudaSuccess) ||
        (b2 && cudaMemcpy(b2, db2, sizeof(float) * H, cudaMemcpyDeviceToHost) != cudaSuccess) ||
        (W3 && cudaMemcpy(W3, dW3, sizeof(float) * (size_t)n * H, cudaMemcpyDeviceToHost) != cudaSuccess) ||
        (b3 && cudaMemcpy(b3, db3, sizeof(float) * n, cudaMemcpyDeviceToHost) != cudaSuccess))
        return CGP_ERR_CUDA;
    return CGP_OK;
}

void ws_free(cgp_ws_s* w) {
    for (void* p : w->allocs) cudaFree(p);
    w->allocs.clear();
}

}  // namespace

extern "C" {

int cgp_gemm_bf16(int M, int N, int K, const void* A_dev, const void* B_dev, float* C_dev, void* stream) {
    if (!A_dev || !B_dev || !C_dev || M <= 0 || N <= 0 || K <= 0 || M % 128 || N % 128 || K % 64) return CGP_ERR_ARG;
    int* err = gemm_err_ptr();
    if (!err) return CGP_ERR_CUDA;
    cudaError_t e = gemm_tn((const __nv_bfloat16*)A_dev, (const __nv_bfloat16*)B_dev,
                            gargs(M, N, K, EPI_F32, nullptr, C_dev, nullptr, nullptr, N, err), (cudaStream_t)stream);
    return e == cudaSuccess ? CGP_OK : CGP_ERR_CUDA;
}

int cgp_ws_create(int n, int hidden, int batch_max, cgp_ws* out) {
    if (!out || n <= 0 || hidden <= 0 || hidden % 128 || batch_max <= 0) return CGP_ERR_ARG;
    *out = nullptr;
    cgp_ws_s* w = new (std::nothrow) cgp_ws_s();
    if (!w) return CGP_ERR_NOMEM;
    int s = ws_create(w, n, hidden, batch_max);
    if (s != CGP_OK) {
        ws_free(w);
        delete w;
        return s;
    }
    *out = w;
    return CGP_OK;
}

int cgp_ws_set_params(cgp_ws w, const float* W1, const float* b1, const float* W2, const float* b2, const float* W3,
                      const float* b3) {
    if (!w || !W1 || !b1 || !W2 || !b2 || !W3 || !b3) return CGP_ERR_ARG;
    return ws_upload_params(w, W1, b1, W2, b2, W3, b3);
}

int cgp_ws_get_params(cgp_ws w, float* W1, float* b1, float* W2, float* b2, float* W3, float* b3) {
    if (!w) return CGP_ERR_ARG;
    return ws_download(w, w->W1, w->b1, w->W2, w->b2, w->W3, w->b3, W1, b1, W2, b2, W3, b3);
}

int cgp_ws_get_grads(cgp_ws w, float* dW1, float* db1, float* dW2, float* db2, float* dW3, float* db3) {
    if (!w) return CGP_ERR_ARG;
    return ws_download(w, w->gW1, w->gb1, w->gW2, w->gb2, w->gW3, w->gb3, dW1, db1, dW2, db2, dW3, db3);
}

int cgp_ws_set_mask(cgp_ws w, const unsigned char* held_host) {
    if (!w || !held_host) return CGP_ERR_ARG;
    std::vector<unsigned char> mk(w->np, 1);
    int free_cnt = 0;
    for (int j = 0; j < w->n; ++j) {
        mk[j] = held_host[j] ? 1 : 0;
        free_cnt += held_host[j] ? 0 : 1;
    }
    if (free_cnt <= 0) return CGP_ERR_ARG;
    if (cudaMemcpy(w->mask, mk.data(), w->np, cudaMemcpyHostToDevice) != cudaSuccess) return CGP_ERR_CUDA;
    w->n_free = free_cnt;
    return CGP_OK;
}

int cgp_ws_forward(cgp_ws w, const double* b_dev, int B, double* p_dev, void* stream) {
    if (!w || !b_dev || !p_dev || B <= 0 || B > w->bmax) return CGP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (forward(w, b_dev, nullptr, B, s) != cudaSuccess) return CGP_ERR_CUDA;
    const size_t cnt = (size_t)B * w->n;
    k_output<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(B, w->n, w->np, w->mask, w->S, w->Y, p_dev);
    return cudaGetLastError() == cudaSuccess ? CGP_OK : CGP_ERR_CUDA;
}

int cgp_ws_train_step(cgp_ws w, const double* b_dev, const double* p_dev, int B, float lr, float* loss_dev, void* stream) {
    if (!w || !b_dev || !p_dev || B <= 0 || B > w->bmax || !(lr >= 0.0f)) return CGP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (train_step(w, b_dev, p_dev, B, lr, s) != cudaSuccess) return CGP_ERR_CUDA;
    if (loss_dev && cudaMemcpyAsync(loss_dev, w->loss, sizeof(float), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return CGP_ERR_CUDA;
    return CGP_OK;
}

namespace {
int residual_prep(cgp_ws w, cgp_ctx c, const double* b, const double* base, const double* p, int B, cudaStream_t s) {
    if (c->nc != w->n) return CGP_ERR_ARG;
    if (!c->bc_set) return CGP_ERR_STATE;
    if (!w->res) {
        int st = CGP_OK;
        if ((st = walloc(w, &w->res, (size_t)w->bmax * w->n)) || (st = walloc(w, &w->cor, (size_t)w->bmax * w->n)))
            return st;
    }
    const size_t cnt = (size_t)B * w->n;
    k_base_residual<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(B, w->n, c->C.rp, c->C.ci, c->Kc, b, base, p, w->res,
                                                                  w->cor);
    return cudaGetLastError() == cudaSuccess ? CGP_OK : CGP_ERR_CUDA;
}
}  // namespace

int cgp_ws_forward_residual(cgp_ws w, cgp_ctx c, const double* b_dev, const double* base_dev, int B, double* p_dev,
                            void* stream) {
    if (!w || !c || !b_dev || !base_dev || !p_dev || B <= 0 || B > w->bmax) return CGP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int st = residual_prep(w, c, b_dev, base_dev, nullptr, B, s);
    if (st != CGP_OK) return st;
    if (forward(w, w->res, nullptr, B, s) != cudaSuccess) return CGP_ERR_CUDA;
    const size_t cnt = (size_t)B * w->n;
    k_output_add<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(B, w->n, w->np, w->mask, w->S, w->Y, base_dev, p_dev);
    return cudaGetLastError() == cudaSuccess ? CGP_OK : CGP_ERR_CUDA;
}

int cgp_ws_train_step_residual(cgp_ws w, cgp_ctx c, const double* b_dev, const double* p_dev, const double* base_dev,
                               int B, float lr, float* loss_dev, void* stream) {
    if (!w || !c || !b_dev || !p_dev || !base_dev || B <= 0 || B > w->bmax || !(lr >= 0.0f)) return CGP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int st = residual_prep(w, c, b_dev, base_dev, p_dev, B, s);
    if (st != CGP_OK) return st;
    if (train_step(w, w->res, w->cor, B, lr, s) != cudaSuccess) return CGP_ERR_CUDA;
    if (loss_dev && cudaMemcpyAsync(loss_dev, w->loss, sizeof(float), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return CGP_ERR_CUDA;
    return CGP_OK;
}

int cgp_ws_status(cgp_ws w, void* stream) {
    if (!w) return CGP_ERR_ARG;
    int e = 0;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return CGP_ERR_CUDA;
    if (cudaMemcpy(&e, w->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return CGP_ERR_CUDA;
    return e;
}

int cgp_ws_destroy(cgp_ws w) {
    if (!w) return CGP_OK;
    cudaDeviceSynchronize();
    ws_free(w);
    delete w;
    return CGP_OK;
}

}  // extern "C"
