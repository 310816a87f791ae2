// Device helpers shared by the CGP kernels: bounded grid barrier, deterministic reductions,
// CSR row products with a configurable number of lanes per row.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "cgp.h"

#ifndef CGP_BARRIER_TIMEOUT_NS
// Wall-clock bound of one grid-barrier wait before it gives up with CGP_ERR_TIMEOUT: 250 ms,
// read from the GPU's global nanosecond timer every 32 polls. A barrier of a healthy persistent
// launch completes within microseconds (every block is co-resident by the cooperative launch),
// so the bound only ends a wait that can never complete.
#define CGP_BARRIER_TIMEOUT_NS 250000000ull
#endif
#ifndef CGP_BARRIER_SPIN_LIMIT
// Backstop on the number of polls (one L2 round trip each, with a short sleep every 32 polls
// once the wait is long): the time bound above normally ends the wait long before this.
#define CGP_BARRIER_SPIN_LIMIT (1u << 24)
#endif

namespace cgp {

// Per-launch synchronisation words of a persistent kernel; zeroed by the host before launch.
struct SyncWords {
    unsigned int count;   // grid-barrier arrival counter
    int err;              // first error code raised by any block (0 = none)
};

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed_i32(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add_u32(unsigned int* p, unsigned int v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait of thread 0 until the arrival counter reaches `target`: polls with acquire loads
// and, every 32 polls, looks for an error raised by another block and checks the elapsed time
// against `limit_ns` (and the poll count against CGP_BARRIER_SPIN_LIMIT). Returns 0 on an error
// or when it gives up (then it records CGP_ERR_TIMEOUT), 1 once every block has arrived.
__device__ __forceinline__ int grid_poll(SyncWords* sw, unsigned int target,
                                         unsigned long long limit_ns = CGP_BARRIER_TIMEOUT_NS) {
    unsigned int spins = 0;
    unsigned long long t0 = 0;
    while (ld_acquire_u32(&sw->count) < target) {
        if ((++spins & 31u) == 0) {
            if (ld_relaxed_i32(&sw->err) != 0) return 0;
            const unsigned long long now = global_ns();
            if (t0 == 0) t0 = now;
            if (now - t0 > limit_ns || spins > CGP_BARRIER_SPIN_LIMIT) {
                atomicCAS(&sw->err, 0, CGP_ERR_TIMEOUT);
                return 0;
            }
            if (spins > 8192) __nanosleep(256);
        }
    }
    return 1;
}

// Grid-wide barrier for a cooperative launch. Every block calls it the same number of times.
// After a block barrier, thread 0 of each block arrives with a release-add (it orders the block's
// earlier writes, which the block barrier made visible to thread 0, before the arrival) and polls
// with acquire loads (they order the block's later reads after every arrival, again through the
// trailing block barrier); no further fence is needed. The poll is bounded: after
// CGP_BARRIER_TIMEOUT_NS of waiting, or as soon as another block has raised an error, it returns
// false (and records CGP_ERR_TIMEOUT if it was the one to give up). Callers must stop their work
// and return when it is false. `epoch` is thread 0's count of barriers passed.
__device__ __forceinline__ bool grid_sync(SyncWords* sw, unsigned int nblocks, unsigned int& epoch) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        epoch += 1;
        if (nblocks > 1) {
            red_release_add_u32(&sw->count, 1u);
            ok = grid_poll(sw, epoch * nblocks);
        } else {
            ok = ld_relaxed_i32(&sw->err) == 0;
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Split-phase form of grid_sync: grid_arrive publishes this block's arrival (after its earlier
// writes), grid_wait completes the barrier. Work placed between the two overlaps the wait.
__device__ __forceinline__ void grid_arrive(SyncWords* sw, unsigned int nblocks, unsigned int& epoch) {
    __syncthreads();
    if (threadIdx.x == 0) {
        epoch += 1;
        if (nblocks > 1) red_release_add_u32(&sw->count, 1u);
    }
}

__device__ __forceinline__ bool grid_wait(SyncWords* sw, unsigned int nblocks, unsigned int epoch) {
    __shared__ int s_okw;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        if (nblocks > 1) {
            ok = grid_poll(sw, epoch * nblocks);
        } else {
            ok = ld_relaxed_i32(&sw->err) == 0;
        }
        s_okw = ok;
    }
    __syncthreads();
    return s_okw != 0;
}

// Called by a block that leaves a persistent kernel because a barrier failed: thread 0 copies
// the launch's error code into the context's sticky barrier status.
__device__ __forceinline__ void record_failure(SyncWords* sw, int* status) {
    if (threadIdx.x == 0) {
        int e = ld_relaxed_i32(&sw->err);
        atomicCAS(status, 0, e != 0 ? e : CGP_ERR_TIMEOUT);
    }
}

// Sum K doubles over the block; the result is valid in thread 0 only. Fixed order, so the
// same inputs give the same bits.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* s_scratch /* [32*K] */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    }
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) s_scratch[k * 32 + warp] = v[k];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double t = lane < nwarps ? s_scratch[k * 32 + lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            v[k] = t;
        }
    }
}

// Write the block's K partial sums to part[k * nblocks + blockIdx.x].
template <int K>
__device__ __forceinline__ void block_partials(double (&v)[K], double* part, unsigned int nblocks,
                                               double* s_scratch) {
    block_sum<K>(v, s_scratch);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) part[k * nblocks + blockIdx.x] = v[k];
    }
}

// Same, for block `bid` of a block group of `nblocks` blocks.
template <int K>
__device__ __forceinline__ void block_partials(double (&v)[K], double* part, unsigned int nblocks, unsigned int bid,
                                               double* s_scratch) {
    block_sum<K>(v, s_scratch);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) part[k * nblocks + bid] = v[k];
    }
}

// Same result layout as block_partials, written for a GPU with a low FP64 rate: a shuffle tree in
// every warp costs about 5 x 32 FP64 additions per warp and value, so instead every thread stores
// its K values in shared memory and warp k adds up value k (blockDim.x additions in a fixed
// order, then one shuffle tree), about a quarter of the FP64 work; with fewer warps than values a
// warp takes values k, k + warps, ... Lane 0 of the summing warp writes part[k * nblocks + bid];
// a following grid barrier (which starts with __syncthreads) publishes it. Needs s_buf of
// K * blockDim.x doubles.
template <int K>
__device__ __forceinline__ void block_partials_lean(const double (&v)[K], double* part, unsigned int nblocks,
                                                    unsigned int bid, double* s_buf) {
    const int T = blockDim.x, t = threadIdx.x, lane = t & 31, warp = t >> 5, nwarps = T >> 5;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) s_buf[k * T + t] = v[k];
    __syncthreads();
    for (int k = warp; k < K; k += nwarps) {
        // four independent chains shorten the dependent FP64 latency; the order is fixed
        const double* b = s_buf + k * T;
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
        if (lane == 0) part[(size_t)k * nblocks + bid] = acc;
    }
}

// Sum K floats over the block in FP32 (shuffle tree in every warp, then warp k over the warp sums
// of value k) and store the block's totals as doubles at part[k * nblocks + bid]; needs s_scratch
// of 32 K floats.
template <int K>
__device__ __forceinline__ void block_partials_f32(const float (&v0)[K], double* part, unsigned int nblocks,
                                                   unsigned int bid, float* s_scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = (blockDim.x + 31) >> 5;
    float v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        v[k] = v0[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    }
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) s_scratch[k * 32 + warp] = v[k];
    }
    __syncthreads();
    // second level: warp k sums value k over the warps (the same order whichever warp does it)
    for (int k = warp; k < K; k += nwarps) {
        float s = lane < nwarps ? s_scratch[k * 32 + lane] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) part[(size_t)k * nblocks + bid] = (double)s;
    }
}

// Block partial sums of K values of the iteration type: FP32 shuffle trees for float, the lean
// shared-memory reduction for double.
template <int K, typename T>
__device__ __forceinline__ void block_partials_it(const T (&v)[K], double* part, unsigned int nblocks, unsigned int bid,
                                                  double* s_lean, float* s_f32) {
    if constexpr (sizeof(T) == sizeof(double)) {
        block_partials_lean<K>(v, part, nblocks, bid, s_lean);
    } else {
        block_partials_f32<K>(v, part, nblocks, bid, s_f32);
    }
}

// Block groups. A batched launch advances several independent problem instances at once: the
// grid is cut into contiguous block groups, one per instance, and every barrier and reduction
// runs within a group. map.inst_of_block == nullptr means one group spanning the whole grid.
struct BatchMap {
    const int* inst_of_block;   // [gridDim.x] instance of each block
    const int* inst_b0;         // [instances] first block of each group
    const int* inst_nb;         // [instances] blocks in each group
};

struct Grp {
    unsigned int nb, bid;       // blocks in this block's group, index of this block in it
    int inst;                   // instance handled by the group
};

// Kernel parameter of a persistent launch: the arguments of a single instance, or a device table
// of per-instance arguments plus the block-group map of a batched launch.
template <typename Args>
struct Launch {
    Args single;
    const Args* table;
    BatchMap map;
};

__device__ __forceinline__ Grp group_of(const BatchMap& m) {
    if (m.inst_of_block == nullptr) return {gridDim.x, blockIdx.x, 0};
    const int i = m.inst_of_block[blockIdx.x];
    return {(unsigned int)m.inst_nb[i], blockIdx.x - (unsigned int)m.inst_b0[i], i};
}

// Maximum number of blocks of a persistent launch (partials are read 32 x 8 at a time).
#define CGP_MAX_GRID 256
// Partial-sum slots (of nblocks doubles each) of a single-instance context.
#define CGP_PART_SLOTS 48

// After a grid barrier: every block sums the nblocks partials of each of the K slots in the same
// fixed order, so all blocks hold bit-identical totals. Slot k's partials start at
// part + slot[k] * nblocks. Warp k (mod the number of warps) handles slot k and issues all its
// loads at once, so the cost is about one L2 round trip. Needs nblocks <= CGP_MAX_GRID.
template <int K>
__device__ __forceinline__ void grid_totals_at(const double* part, const int (&slot)[K], unsigned int nblocks,
                                               double (&out)[K], double* s_bcast /* [K] */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (warp == k % nwarps) {
            const double* p = part + (size_t)slot[k] * nblocks;
            double v[CGP_MAX_GRID / 32];
#pragma unroll
            for (int q = 0; q < CGP_MAX_GRID / 32; ++q) {
                const unsigned int b = lane + 32u * q;
                v[q] = b < nblocks ? __ldcg(p + b) : 0.0;
            }
            double t = 0.0;
#pragma unroll
            for (int q = 0; q < CGP_MAX_GRID / 32; ++q) t += v[q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) s_bcast[k] = t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = s_bcast[k];
    __syncthreads();
}

// As grid_totals_at, but leaves the K totals in s_bcast (visible to the whole block after the
// trailing barrier) instead of copying them to every thread: for kernels where one thread does
// the scalar recurrences and broadcasts the results.
template <int K>
__device__ __forceinline__ void grid_totals_shared(const double* part, const int (&slot)[K], unsigned int nblocks,
                                                   double* s_bcast /* [K] */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (warp == k % nwarps) {
            const double* p = part + (size_t)slot[k] * nblocks;
            double v[CGP_MAX_GRID / 32];
#pragma unroll
            for (int q = 0; q < CGP_MAX_GRID / 32; ++q) {
                const unsigned int b = lane + 32u * q;
                v[q] = b < nblocks ? __ldcg(p + b) : 0.0;
            }
            double t = 0.0;
#pragma unroll
            for (int q = 0; q < CGP_MAX_GRID / 32; ++q) t += v[q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) s_bcast[k] = t;
        }
    }
    __syncthreads();
}

// Contiguous slots starting at region `base` (in units of nblocks).
template <int K>
__device__ __forceinline__ void grid_totals(const double* part, unsigned int nblocks, double (&out)[K],
                                            double* s_bcast /* [K] */) {
    int slot[K];
#pragma unroll
    for (int k = 0; k < K; ++k) slot[k] = k;
    grid_totals_at<K>(part, slot, nblocks, out, s_bcast);
}

// Rows owned by a block: a contiguous slice of [0, n).
struct RowRange {
    int r0, r1;
};
__device__ __forceinline__ RowRange block_rows(int n) {
    const long long per = ((long long)n + gridDim.x - 1) / gridDim.x;
    long long r0 = per * blockIdx.x, r1 = r0 + per;
    if (r0 > n) r0 = n;
    if (r1 > n) r1 = n;
    return {(int)r0, (int)r1};
}

// Rows owned by a block of a block group.
__device__ __forceinline__ RowRange group_rows(int n, const Grp& g) {
    const long long per = ((long long)n + g.nb - 1) / g.nb;
    long long r0 = per * g.bid, r1 = r0 + per;
    if (r0 > n) r0 = n;
    if (r1 > n) r1 = n;
    return {(int)r0, (int)r1};
}

// Rows owned by a block of a block group when rows go in 32-row slices (the sliced-ELL layout):
// whole slices per block, so every slice's rows belong to one block.
__device__ __forceinline__ RowRange group_rows_aligned(int n, const Grp& g) {
    const long long ns = ((long long)n + 31) >> 5;
    const long long per = (ns + g.nb - 1) / g.nb;
    long long r0 = per * g.bid * 32, r1 = r0 + per * 32;
    if (r0 > n) r0 = n;
    if (r1 > n) r1 = n;
    return {(int)r0, (int)r1};
}

// Two-wide loads/stores of interleaved pairs.
template <typename T> struct Pair;
template <> struct Pair<double> { typedef double2 type; };
template <> struct Pair<float> { typedef float2 type; };

template <typename T>
__device__ __forceinline__ void load2(const T* p, int i, T& a, T& b) {
    typename Pair<T>::type v = reinterpret_cast<const typename Pair<T>::type*>(p)[i];
    a = v.x;
    b = v.y;
}
template <typename T>
__device__ __forceinline__ void store2(T* p, int i, T a, T b) {
    typename Pair<T>::type v;
    v.x = a;
    v.y = b;
    reinterpret_cast<typename Pair<T>::type*>(p)[i] = v;
}

// Sum over the `lanes` (power of two <= 32) lanes of a row group.
template <typename T>
__device__ __forceinline__ T group_sum(T v, int lanes) {
    for (int o = lanes >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace cgp
