// tc_gemm.cu -- 5th-generation tensor-core GEMM for sm_103a (tcgen05 + TMA + TMEM).
//
//   C[z] = alpha * diag(rs[z]) * A[z] * Bt[z]^T * diag(cs[z]) + beta * C[z]      (FP32 in / out)
//
// A is M x K and Bt is N x K, both row-major (K contiguous: the "K-major" operand layout), so
// every product of the wrap and of the rank-m flush is fed without a transpose pass.  C may be
// written row-major or transposed.  Tiles of 128 x BN are accumulated in TMEM by tcgen05.mma
// (kind::tf32, issued by one thread), operands arrive in 128-byte-swizzled shared memory by
// cp.async.bulk.tensor (TMA) through a multi-stage mbarrier pipeline, and the epilogue reads the
// accumulator back with tcgen05.ld.
//
// FP32 accuracy (split3): each operand x is split into hi = x with the low 13 mantissa bits
// cleared (exactly representable in TF32) and lo = x - hi, and the tile product is accumulated
// as hi*hi + lo*hi + hi*lo in FP32 (the three-term TF32 split of Ootomo and Yokota, 2022).  The
// split is done in shared memory after each stage lands.
//
// FP64 accuracy (the OZ instantiation, driven by ozaki.cu): the operands are stacks of integer
// digit planes of FP64 matrices, stored as bf16 (digits of at most 8 bits are exact) and
// multiplied by tcgen05.mma kind::f16 with FP32 accumulation.  A 128-byte swizzle row holds 64
// bf16, so a stage has the same bytes and the same 32-byte MMA steps as the TF32 path.  One
// launch runs the K loop over a list of (A plane, B plane) pairs into one FP32 accumulator --
// every partial sum is an integer below 2^24, so the tensor cores compute it exactly -- and the
// epilogue adds 2^(e_row + e_col - b d) times it into an FP64 C.
//
// Every wait is bounded (about two seconds of %globaltimer); on expiry the kernel records
// DEV_TIMEOUT, stops issuing work, waits (again bounded) for its copies in flight, frees its
// TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>
#include <utility>
#include <vector>

#include "internal.h"

namespace afq {

namespace {

constexpr int TC_BM = 128;
constexpr int TC_BK = 32;  // 32 FP32 = 128 bytes = one swizzle atom row
constexpr int TC_BK16 = 64;  // the same row in bf16
constexpr int TC_NT = 256;  // 8 warps: all split the stages; warps w and w + 4 share TMEM lane quarter w % 4 in the epilogue
constexpr unsigned long long WAIT_NS = 2000000000ULL;

// Digit-plane products (OZ) take three stages, so two CTAs (three at BN = 64) share an SM: their
// K loops are bound by operand latency, not by the MMA rate.
template <int BN, bool SPLIT, bool OZ = false>
struct TcCfg {
    static constexpr int A_BYTES = TC_BM * TC_BK * 4;
    static constexpr int B_BYTES = BN * TC_BK * 4;
    static constexpr int STAGE_BYTES = (A_BYTES + B_BYTES) * (SPLIT ? 2 : 1);
    static constexpr int STAGES = (SPLIT || OZ) ? 3 : 4;
    static constexpr int SMEM = STAGES * STAGE_BYTES + 1024;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on phase `parity`; false on timeout (DEV_TIMEOUT recorded) or a recorded error.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > WAIT_NS) {
            set_err(err, DEV_TIMEOUT);
            return false;
        }
    }
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(smem_u32(dst)),
        "l"((const void*)tm), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor: K-major tile, rows of 128 bytes, 128-byte swizzle, 8-row
// groups 1024 bytes apart (stride byte offset); the leading byte offset is unused for this layout.
__device__ __forceinline__ uint64_t desc_sw128(const void* tile) {
    const uint64_t addr = smem_u32(tile);
    uint64_t d = (addr & 0x3FFFFull) >> 4;
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor, kind::tf32: D = F32, A = B = TF32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
        "[%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

struct TcArgs {
    int M, N, K;
    float* C;
    long ldc, sC;
    int c_trans;
    const float* rs;
    long srs;
    const float* cs;
    long scs;
    float alpha, beta;
    int a_batched, b_batched;
    int* err;
    // digit-plane products (OZ): pairs of this launch, k-tiles per pair, planes per batch entry,
    // the plane of A and of B of every pair, and the FP64 output with its power-of-two scales
    int oz_np, oz_kt, oz_ns;
    signed char oz_pa[TC_OZ_MAXP], oz_pb[TC_OZ_MAXP];
    double* C64;
    long ldc64, sC64;
    const double* rsc;
    long srsc;
    const double* csc;
    long scsc;
    double gscale;
    int first;
};

template <int BN, bool SPLIT, bool OZ>
__global__ void __launch_bounds__(TC_NT, 1) tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                                                         const __grid_constant__ CUtensorMap tmB, TcArgs a) {
    static_assert(!(SPLIT && OZ), "digit-plane products are single TF32 passes");
    using Cfg = TcCfg<BN, SPLIT, OZ>;
    constexpr int S = Cfg::STAGES;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[S], empty[S], done;
    __shared__ uint32_t tmem_holder;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n0 = blockIdx.x * BN, m0 = blockIdx.y * TC_BM, z = blockIdx.z;
    const int KT = OZ ? a.oz_np * a.oz_kt : (a.K + TC_BK - 1) / TC_BK;
    const int za = a.a_batched ? z : 0, zb = a.b_batched ? z : 0;
    // k-tile t: its K offset and the batch coordinates of its A and B tiles
    auto tile_of = [&](int t, int& kx, int& ya, int& yb) {
        if (OZ) {
            const int pr = t / a.oz_kt, kk = t - pr * a.oz_kt;
            kx = kk * TC_BK16;
            ya = z * a.oz_ns + a.oz_pa[pr];
            yb = z * a.oz_ns + a.oz_pb[pr];
        } else {
            kx = t * TC_BK;
            ya = za;
            yb = zb;
        }
    };
    const uint32_t idesc = OZ ? idesc_bf16(TC_BM, BN) : idesc_tf32(TC_BM, BN);
    const uint32_t stage_tx = Cfg::A_BYTES + Cfg::B_BYTES;

    auto Ahi = [&](int s) { return base + (size_t)s * Cfg::STAGE_BYTES; };
    auto Bhi = [&](int s) { return base + (size_t)s * Cfg::STAGE_BYTES + Cfg::A_BYTES; };
    auto Alo = [&](int s) { return base + (size_t)s * Cfg::STAGE_BYTES + Cfg::A_BYTES + Cfg::B_BYTES; };
    auto Blo = [&](int s) { return base + (size_t)s * Cfg::STAGE_BYTES + 2 * Cfg::A_BYTES + Cfg::B_BYTES; };

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // The split product rotates k-tiles over NACC accumulators (summed in FP32 by the epilogue):
    // a shorter chain of in-pipe accumulations per accumulator keeps the result at FP32 accuracy.
    // Four accumulators of 128 columns fill the 512 TMEM columns; wider tiles use three.
    constexpr int NACC = SPLIT ? (BN <= 128 ? 4 : 3) : 1;
    constexpr uint32_t TMEM_COLS = (BN * NACC <= 128) ? 128u : (BN * NACC <= 256 ? 256u : 512u);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_holder;

    int issued = 0;  // k-tiles whose TMA was issued (thread 0 only)
    if (tid == 0) {
        for (int s = 0; s < S && s < KT; ++s) {
            int kx, ya, yb;
            tile_of(s, kx, ya, yb);
            mbar_expect_tx(&full[s], stage_tx);
            tma_load_3d(Ahi(s), &tmA, kx, m0, ya, &full[s]);
            tma_load_3d(Bhi(s), &tmB, kx, n0, yb, &full[s]);
            ++issued;
        }
    }
    int consumed = 0;   // k-tiles whose data every thread has waited for
    int committed = 0;  // k-tiles whose MMAs were issued and committed (thread 0 only)
    for (int kt = 0; kt < KT; ++kt) {
        const int s = kt % S;
        const uint32_t ph = (uint32_t)(kt / S) & 1u;
        if (!mbar_wait(&full[s], ph, a.err)) s_abort = 1;
        __syncthreads();
        if (s_abort) break;
        ++consumed;
        if (SPLIT) {
            // hi = x with the low 13 mantissa bits cleared, lo = x - hi, for both tiles of the stage
            // (16-byte accesses: consecutive threads touch consecutive 16-byte chunks, and hi / lo
            // tiles share the swizzled layout, so the split is position by position)
            auto split = [&](unsigned char* hp, unsigned char* lp, int n4) {
                uint4* h4 = (uint4*)hp;
                uint4* l4 = (uint4*)lp;
#pragma unroll 4
                for (int e = tid; e < n4; e += TC_NT) {
                    const uint4 x = h4[e];
                    uint4 h, l;
                    h.x = x.x & 0xFFFFE000u;
                    h.y = x.y & 0xFFFFE000u;
                    h.z = x.z & 0xFFFFE000u;
                    h.w = x.w & 0xFFFFE000u;
                    l.x = __float_as_uint(__uint_as_float(x.x) - __uint_as_float(h.x));
                    l.y = __float_as_uint(__uint_as_float(x.y) - __uint_as_float(h.y));
                    l.z = __float_as_uint(__uint_as_float(x.z) - __uint_as_float(h.z));
                    l.w = __float_as_uint(__uint_as_float(x.w) - __uint_as_float(h.w));
                    h4[e] = h;
                    l4[e] = l;
                }
            };
            split(Ahi(s), Alo(s), TC_BM * TC_BK / 4);
            split(Bhi(s), Blo(s), BN * TC_BK / 4);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
        }
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t dah = desc_sw128(Ahi(s)), dbh = desc_sw128(Bhi(s));
            const uint64_t dal = SPLIT ? desc_sw128(Alo(s)) : 0, dbl = SPLIT ? desc_sw128(Blo(s)) : 0;
            const uint32_t dacc = tmem + (uint32_t)((kt % NACC) * BN);
#pragma unroll
            for (int j = 0; j < TC_BK / 8; ++j) {
                const uint64_t kofs = (uint64_t)(j * 32) >> 4;  // 8 TF32 (16 bf16) = 32 bytes along K
                if (OZ) mma_bf16(dacc, dah + kofs, dbh + kofs, idesc, (kt >= NACC || j > 0) ? 1u : 0u);
                else mma_tf32(dacc, dah + kofs, dbh + kofs, idesc, (kt >= NACC || j > 0) ? 1u : 0u);
                if (SPLIT) {
                    mma_tf32(dacc, dal + kofs, dbh + kofs, idesc, 1u);
                    mma_tf32(dacc, dah + kofs, dbl + kofs, idesc, 1u);
                }
            }
            mma_commit(&empty[s]);
            ++committed;
            if (kt == KT - 1) mma_commit(&done);
            // refill the stage consumed one iteration ago (its MMAs are queued ahead of these)
            const int kr = kt - 1 + S;
            if (kt >= 1 && kr < KT) {
                const int sr = (kt - 1) % S;
                const uint32_t phr = (uint32_t)((kt - 1) / S) & 1u;
                if (mbar_wait(&empty[sr], phr, a.err)) {
                    int kx, ya, yb;
                    tile_of(kr, kx, ya, yb);
                    mbar_expect_tx(&full[sr], stage_tx);
                    tma_load_3d(Ahi(sr), &tmA, kx, m0, ya, &full[sr]);
                    tma_load_3d(Bhi(sr), &tmB, kx, n0, yb, &full[sr]);
                    ++issued;
                } else {
                    s_abort = 1;
                }
            }
        }
    }
    __syncthreads();
    if (!s_abort) {
        if (!mbar_wait(&done, 0, a.err)) s_abort = 1;
    }
    __syncthreads();
    if (!s_abort && OZ) {
        // FP64 epilogue: C64 (+)= (acc * 2^(-b d) * 2^e_row) * 2^e_col.  acc is an exact integer
        // and the scales are powers of two, so the only rounding is the FP64 addition.  The warp's
        // 32 x 16 chunk goes through shared memory so that every access covers 16 consecutive
        // columns of two rows.
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int quarter = warp & 3, half = warp >> 2;
        const int m = m0 + quarter * 32 + lane;
        double* C = a.C64 + (size_t)z * a.sC64;
        const double* csc = a.csc + (size_t)z * a.scsc;
        float* stg = (float*)base + warp * (32 * 17);
        double* srow = (double*)((float*)base + 8 * 32 * 17) + warp * 32;
        srow[lane] = (m < a.M) ? a.rsc[(size_t)z * a.srsc + m] * a.gscale : 0.0;
#pragma unroll 1
        for (int cb = half; cb < BN / 16; cb += 2) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(cb * 16), v);
#pragma unroll
            for (int j = 0; j < 16; ++j) stg[lane * 17 + j] = v[j];
            __syncwarp();
#pragma unroll 4
            for (int i = 0; i < 16; ++i) {
                const int row = 2 * i + (lane >> 4), col = lane & 15;
                const int mm = m0 + quarter * 32 + row, n = n0 + cb * 16 + col;
                if (mm < a.M && n < a.N) {
                    const double val = ((double)stg[row * 17 + col] * srow[row]) * csc[n];
                    const size_t o = (size_t)mm * a.ldc64 + n;
                    C[o] = a.first ? val : C[o] + val;
                }
            }
            __syncwarp();
        }
    } else if (!s_abort) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int quarter = warp & 3, half = warp >> 2;  // TMEM lanes 32 quarter .. + 31; column chunks by parity
        const int m = m0 + quarter * 32 + lane;
        float* C = a.C + (size_t)z * a.sC;
        const float* rs = a.rs ? a.rs + (size_t)z * a.srs : nullptr;
        const float* cs = a.cs ? a.cs + (size_t)z * a.scs : nullptr;
        const float rsm = (rs && m < a.M) ? rs[m] : 1.0f;
#pragma unroll 1
        for (int cb = half; cb < BN / 16; cb += 2) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(cb * 16), v);
            const int nacc = KT < NACC ? KT : NACC;
            for (int q = 1; q < nacc; ++q) {
                float v2[16];
                tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(q * BN + cb * 16), v2);
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] += v2[j];
            }
            if (a.c_trans) {  // lanes are consecutive rows m: consecutive addresses of C^T
                if (m < a.M) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int n = n0 + cb * 16 + j;
                        if (n >= a.N) continue;
                        float val = a.alpha * rsm * v[j];
                        if (cs) val *= cs[n];
                        const size_t o = (size_t)n * a.ldc + m;
                        C[o] = (a.beta == 0.0f) ? val : val + a.beta * C[o];
                    }
                }
            } else {
                // row-major C: the warp's 32 x 16 chunk goes through shared memory (the pipeline's
                // stage buffers, idle once every MMA has completed) so that each store instruction
                // writes two rows of 16 consecutive columns
                float* stg = (float*)base + warp * (32 * 17);
#pragma unroll
                for (int j = 0; j < 16; ++j) stg[lane * 17 + j] = v[j];
                __syncwarp();
#pragma unroll 4
                for (int i = 0; i < 16; ++i) {
                    const int row = 2 * i + (lane >> 4), col = lane & 15;
                    const int mm = m0 + quarter * 32 + row, n = n0 + cb * 16 + col;
                    if (mm < a.M && n < a.N) {
                        float val = a.alpha * (rs ? rs[mm] : 1.0f) * stg[row * 17 + col];
                        if (cs) val *= cs[n];
                        const size_t o = (size_t)mm * a.ldc + n;
                        C[o] = (a.beta == 0.0f) ? val : val + a.beta * C[o];
                    }
                }
                __syncwarp();
            }
        }
    } else if (tid == 0) {
        // drain (bounded): every issued copy must land and the last committed MMAs must finish
        // before the CTA frees its TMEM and exits
        for (int t = consumed; t < issued; ++t) mbar_wait(&full[t % S], (uint32_t)(t / S) & 1u, a.err);
        if (committed > 0) {
            const int t = committed - 1;
            mbar_wait(&empty[t % S], (uint32_t)(t / S) & 1u, a.err);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 3D map over a row-major (rows x cols) matrix of FP32 (es = 4) or bf16 (es = 2) elements with
// leading dimension ld, batch stride sb (elements), box = 128 bytes of columns x box_rows rows,
// 128-byte swizzle, zero fill out of bounds.
bool make_tmap(CUtensorMap* tm, const void* ptr, int es, int rows, int cols, long ld, int batch, long sb,
               int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    if (((uintptr_t)ptr & 15) || ((ld * es) & 15) || ((sb * es) & 15)) return false;
    cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)batch};
    cuuint64_t strides[2] = {(cuuint64_t)ld * es, (cuuint64_t)sb * es};
    cuuint32_t box[3] = {(cuuint32_t)(128 / es), (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(tm, es == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)ptr,
                    dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Encoded tensor maps are cached by their full description: the sweep reuses the same
// buffers every slice, and encoding on every launch would starve the GPU of work.
struct TmapKey {
    const void* ptr;
    int es, rows, cols, batch, box;
    long ld, sb;
    bool operator==(const TmapKey& o) const {
        return ptr == o.ptr && es == o.es && rows == o.rows && cols == o.cols && batch == o.batch && box == o.box &&
               ld == o.ld && sb == o.sb;
    }
};

bool cached_tmap(CUtensorMap* tm, const void* ptr, int es, int rows, int cols, long ld, int batch, long sb,
                 int box_rows) {
    static std::vector<std::pair<TmapKey, CUtensorMap>> cache;
    static std::mutex mu;
    const TmapKey k{ptr, es, rows, cols, batch, box_rows, ld, sb};
    std::lock_guard<std::mutex> lk(mu);
    for (auto& e : cache)
        if (e.first == k) {
            *tm = e.second;
            return true;
        }
    if (!make_tmap(tm, ptr, es, rows, cols, ld, batch, sb, box_rows)) return false;
    if (cache.size() >= 4096) cache.clear();
    cache.emplace_back(k, *tm);
    return true;
}

template <int BN, bool SPLIT>
cudaError_t tc_launch(cudaStream_t st, const TcGemmArgs& g) {
    using Cfg = TcCfg<BN, SPLIT>;
    {
        cudaError_t e = ensure_smem_attr((const void*)tc_gemm_kernel<BN, SPLIT, false>, Cfg::SMEM);
        if (e != cudaSuccess) return e;
    }
    CUtensorMap tmA, tmB;
    const int ba = g.sA ? g.batch : 1, bb = g.sB ? g.batch : 1;
    const long sA = g.sA ? g.sA : (long)g.M * g.lda, sB = g.sB ? g.sB : (long)g.N * g.ldb;
    if (!cached_tmap(&tmA, g.A, 4, g.M, g.K, g.lda, ba, sA, TC_BM)) return cudaErrorInvalidValue;
    if (!cached_tmap(&tmB, g.Bt, 4, g.N, g.K, g.ldb, bb, sB, BN)) return cudaErrorInvalidValue;
    TcArgs a;
    a.M = g.M; a.N = g.N; a.K = g.K;
    a.C = g.C; a.ldc = g.ldc; a.sC = g.sC; a.c_trans = g.c_trans;
    a.rs = g.rs; a.srs = g.srs; a.cs = g.cs; a.scs = g.scs;
    a.alpha = g.alpha; a.beta = g.beta;
    a.a_batched = g.sA != 0; a.b_batched = g.sB != 0;
    a.err = g.err;
    a.oz_np = a.oz_kt = a.oz_ns = 0;
    a.C64 = nullptr;
    a.rsc = a.csc = nullptr;
    dim3 grid((g.N + BN - 1) / BN, (g.M + TC_BM - 1) / TC_BM, g.batch);
    count_launch();
    tc_gemm_kernel<BN, SPLIT, false><<<grid, TC_NT, Cfg::SMEM, st>>>(tmA, tmB, a);
    return cudaGetLastError();
}

template <int BN>
cudaError_t tc_oz_launch(cudaStream_t st, const TcOzArgs& g) {
    using Cfg = TcCfg<BN, false, true>;
    {
        cudaError_t e = ensure_smem_attr((const void*)tc_gemm_kernel<BN, false, true>, Cfg::SMEM);
        if (e != cudaSuccess) return e;
    }
    CUtensorMap tmA, tmB;
    const long sa = (long)g.M * g.Kp, sb = (long)g.N * g.Kp;
    if (!cached_tmap(&tmA, g.Ad, 2, g.M, g.Kp, g.Kp, g.batch * g.ns, sa, TC_BM)) return cudaErrorInvalidValue;
    if (!cached_tmap(&tmB, g.Bd, 2, g.N, g.Kp, g.Kp, g.batch * g.ns, sb, BN)) return cudaErrorInvalidValue;
    TcArgs a = {};
    a.M = g.M; a.N = g.N; a.K = g.K;
    a.err = g.err;
    a.oz_np = g.np;
    a.oz_kt = (g.K + TC_BK16 - 1) / TC_BK16;
    a.oz_ns = g.ns;
    for (int i = 0; i < g.np; ++i) {
        a.oz_pa[i] = (signed char)g.pa[i];
        a.oz_pb[i] = (signed char)g.pb[i];
    }
    a.C64 = g.C; a.ldc64 = g.ldc; a.sC64 = g.sC;
    a.rsc = g.rsc; a.srsc = g.M;
    a.csc = g.csc; a.scsc = g.N;
    a.gscale = g.gscale;
    a.first = g.first;
    dim3 grid((g.N + BN - 1) / BN, (g.M + TC_BM - 1) / TC_BM, g.batch);
    count_launch();
    tc_gemm_kernel<BN, false, true><<<grid, TC_NT, Cfg::SMEM, st>>>(tmA, tmB, a);
    return cudaGetLastError();
}

}  // namespace

// Tile width: the BN in {128, 144, 160} that minimises (waves of 128 x BN tiles on the SMs) x BN,
// i.e. the time of the last wave; e.g. 1600 x 1600 x 2 takes BN = 160 (260 tiles, 2 waves on 152
// SMs, against 338 tiles and 3 waves at 128) and 1152 x 2304 takes BN = 144 (one wave of 144).
static int pick_bn(const TcGemmArgs& g) {
    static int nsm = 0;
    if (!nsm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (nsm <= 0) nsm = 148;
    }
    const long mt = (g.M + TC_BM - 1) / TC_BM;
    int best = 128;
    long best_cost = -1;
    for (int bn : {128, 144, 160}) {
        const long tiles = mt * ((g.N + bn - 1) / bn) * g.batch;
        const long cost = ((tiles + nsm - 1) / nsm) * bn;
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = bn;
        }
    }
    return best;
}

// Tile width of a digit-plane product: the BN in {64, 128, 144, 160} that minimises (tiles per
// SM, rounded up) x (128 + BN), the operand bytes an SM streams per K step -- the launches are
// bound by operand traffic.  Small products (U_L U_R: 700 x 700 x 2) take 64 and spread over
// every SM; U_R Z (1600 x 1600 x 2) keeps 160 (260 tiles, all resident at two per SM).
static int pick_bn_oz(const TcOzArgs& g) {
    static int nsm = 0;
    if (!nsm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (nsm <= 0) nsm = 148;
    }
    const long mt = (g.M + TC_BM - 1) / TC_BM;
    int best = 160;
    long best_cost = -1;
    for (int bn : {160, 144, 128, 64}) {
        const long tiles = mt * ((g.N + bn - 1) / bn) * g.batch;
        const long cost = ((tiles + nsm - 1) / nsm) * (TC_BM + bn);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = bn;
        }
    }
    return best;
}

cudaError_t tc_gemm_oz(cudaStream_t st, const TcOzArgs& g) {
    if (g.M <= 0 || g.N <= 0 || g.K <= 0 || g.batch <= 0) return cudaSuccess;
    if (g.np < 1 || g.np > TC_OZ_MAXP || g.K > g.Kp || (g.Kp & 7)) return cudaErrorInvalidValue;
    for (int i = 0; i < g.np; ++i)
        if (g.pa[i] < 0 || g.pa[i] >= g.ns || g.pb[i] < 0 || g.pb[i] >= g.ns) return cudaErrorInvalidValue;
    const int bn = pick_bn_oz(g);
    if (bn == 160) return tc_oz_launch<160>(st, g);
    if (bn == 144) return tc_oz_launch<144>(st, g);
    if (bn == 128) return tc_oz_launch<128>(st, g);
    return tc_oz_launch<64>(st, g);
}

cudaError_t tc_gemm(cudaStream_t st, const TcGemmArgs& g) {
    if (g.M <= 0 || g.N <= 0 || g.K <= 0 || g.batch <= 0) return cudaSuccess;
    const int bn = pick_bn(g);
    if (g.split3) {
        if (bn == 160) return tc_launch<160, true>(st, g);
        if (bn == 144) return tc_launch<144, true>(st, g);
        return tc_launch<128, true>(st, g);
    }
    if (bn == 160) return tc_launch<160, false>(st, g);
    if (bn == 144) return tc_launch<144, false>(st, g);
    return tc_launch<128, false>(st, g);
}

}  // namespace afq
