// common.cuh -- device helpers shared by the libafqmc kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/afqmc.h"

namespace afq {

// ---------------------------------------------------------------------------
// Device error word.  Kernels never trap: they record a code here and return.
// ---------------------------------------------------------------------------
enum DevErr : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_NUMERIC = 2, DEV_ARG = 3 };

__device__ __forceinline__ void set_err(int* err, int code) { atomicCAS(err, 0, code); }

__device__ __forceinline__ int read_err(const int* err) {
    return *((volatile const int*)err);
}

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC'11): a 10-round counter-based bijection.  Each round takes
// the two 64x64 -> 128-bit products of the multipliers with counter words 0
// and 2, and mixes the halves with words 1 and 3 and the key; the key is
// advanced by the two Weyl increments between rounds.
// ---------------------------------------------------------------------------
struct u64x4 { uint64_t v[4]; };

__device__ __forceinline__ u64x4 philox4x64_10(u64x4 c, uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t lo0 = M0 * c.v[0], hi0 = __umul64hi(M0, c.v[0]);
        uint64_t lo1 = M1 * c.v[2], hi1 = __umul64hi(M1, c.v[2]);
        u64x4 o;
        o.v[0] = hi1 ^ c.v[1] ^ k0;
        o.v[1] = lo1;
        o.v[2] = hi0 ^ c.v[3] ^ k1;
        o.v[3] = lo0;
        c = o;
    }
    return c;
}

// Uniform in [0,1) with 53 random bits: counter (j + 1, visit, 0, 0), key (seed, walker).
__device__ __forceinline__ double philox_uniform(uint64_t seed, uint64_t walker, uint64_t visit, uint64_t j) {
    u64x4 c;
    c.v[0] = j + 1; c.v[1] = visit; c.v[2] = 0; c.v[3] = 0;
    u64x4 o = philox4x64_10(c, seed, walker);
    return (double)(o.v[0] >> 11) * (1.0 / 9007199254740992.0);
}

// ---------------------------------------------------------------------------
// Grid-wide barrier for cooperative (co-resident) launches.  Sense is a
// generation counter; the wait is bounded: after ~2^24 polls (> 1 s) the
// barrier records DEV_TIMEOUT and returns false so the kernel can exit.
// ---------------------------------------------------------------------------
struct GridBar {
    unsigned int count;
    unsigned int gen;
};

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ bool grid_barrier(GridBar* b, unsigned int nblocks, int* err) {
    __syncthreads();
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned int g = ld_acquire_u32(&b->gen);
        __threadfence();
        unsigned int arrived = atomicAdd(&b->count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(&b->count, 0u);
            __threadfence();
            atomicAdd(&b->gen, 1u);
        } else {
            unsigned int polls = 0;
            while (ld_acquire_u32(&b->gen) == g) {
                if (read_err(err) != 0) { ok = 0; break; }
                if (++polls > (1u << 24)) { set_err(err, DEV_TIMEOUT); ok = 0; break; }
                if (polls > 64) __nanosleep(64);
            }
        }
        __threadfence();
        if (read_err(err) != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Grid-wide arrival counter for cooperative (co-resident) launches, for one thread per CTA: the
// k-th barrier adds one to *ctr with release semantics and completes when *ctr reaches k nblocks.
// The counter starts at zero for the launch and only grows, so a barrier costs one reduction and
// the polling, with no reset.  The caller synchronises its CTA before (so that every write of the
// CTA precedes the arrival) and after.  The wait is bounded: after about two seconds of
// %globaltimer, or once another CTA has recorded an error, it records DEV_TIMEOUT (or keeps the
// error) and returns false.
__device__ __forceinline__ bool grid_arrive_wait(unsigned int* ctr, unsigned int target, int* err) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(ctr) : "memory");
    unsigned long long t0 = 0;
    unsigned int polls = 0;
    while (ld_acquire_u32(ctr) < target) {
        if ((++polls & 255u) == 0u) {
            if (read_err(err) != 0) return false;
            unsigned long long t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            if (t0 == 0) t0 = t;
            else if (t - t0 > 2000000000ULL) {
                set_err(err, DEV_TIMEOUT);
                return false;
            }
        }
    }
    return true;
}

// Barrier `id` (1..15) over the first `nthreads` threads of the block (whole warps).
__device__ __forceinline__ void named_barrier_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Field-change factor Delta = exp(c (x' - x)) - 1 for one site and spin (Sec. II.C).
__device__ __forceinline__ double field_delta(double c, int x, int xp) {
    return exp(c * (double)(xp - x)) - 1.0;
}

}  // namespace afq
