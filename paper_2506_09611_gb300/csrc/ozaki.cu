// ozaki.cu -- FP64 matrix products on the bf16 tensor cores by error-free digit splitting.
//
// GB300 runs FP64 at 1/64 of its FP32 rate, and the recompute of G (Sec. II.C, Eq. GrFMatNew)
// spends most of its time in two FP64 products: U_L U_R and U_R (U_L U_R)^{-1} U_L.  Both are
// formed here without FP64 multiplies, following the splitting of Ozaki, Ogita, Oishi and Rump
// (Numer. Algorithms 59, 2012):
//
//   * every row i of A gets the exponent E_i with max_k |A_ik| < 2^E_i, and every element becomes
//     A_ik = 2^E_i sum_{p=1..s} a_ik^(p) 2^(-b p) + (a remainder below 2^(E_i - b s)),
//     with signed integer digits |a^(p)| < 2^b taken from the bits of the FP64 significand
//     (integer shifts and masks only: no rounding anywhere).  B is split the same way by columns.
//   * a digit plane holds small integers, exact in bf16, so the tensor cores multiply two planes
//     exactly, and a sum of products stays exact in the FP32 accumulator as long as its terms
//     add up to less than 2^24 in magnitude: the pairs (p, q) of one digit level d = p + q are
//     accumulated together in groups of at most G = floor((2^24 - 1) / (K (2^b - 1)^2)).
//   * C_ij = 2^(E_i + F_j) sum_{p + q <= s + 1} 2^(-b (p + q)) (a^(p) b^(q))_ij is summed in FP64
//     in the epilogue of every group (tc_gemm.cu); the dropped levels and the remainders lie below
//     (s + 1) K 2^(-b s) 2^(E_i + F_j), with b s >= 54.
//
// b (bits per digit) is chosen per shape from {7, 6, 5} by a small cost model: fewer bits mean
// more pairs but larger groups, i.e. fewer FP64 epilogues.
#include <math.h>

#include <vector>

#include "internal.h"

namespace afq {

namespace {

constexpr int OZ_SMAX = 11;  // digits per element at b = 5

struct OzSplitArgs {
    const double* src;
    long ld, sb;  // leading dimension and batch stride of the source
    int R, K, Kp, b, s;
    uint16_t* out;  // [batch][s][R][Kp] bf16 bit patterns
    double* scale;  // [batch][R]: 2^E of every output row
    int* err;
};

__device__ __forceinline__ int biased_exp(double v) {
    return (int)(((unsigned long long)__double_as_longlong(v) >> 52) & 0x7ffull);
}

// v / 2^E * 2^F truncated toward zero, as an unsigned magnitude (< 2^F) and a sign, where
// E = ebmax - 1022 for the largest biased exponent ebmax of the row: v = +-m 2^(eb - 1075) with
// m the 53-bit significand (eb >= 1), so the fixed-point value is m 2^(eb - ebmax - 53 + F).
__device__ __forceinline__ unsigned long long oz_fixed(double v, int ebmax, int F, bool& neg) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    neg = (u >> 63) != 0ull;
    const int eb = (int)((u >> 52) & 0x7ffull);
    const unsigned long long m = (u & 0xFFFFFFFFFFFFFull) | (eb ? (1ull << 52) : 0ull);
    const int sh = (eb > 0 ? eb : 1) - ebmax - 53 + F;
    if (sh >= 0) return m << sh;
    if (sh <= -64) return 0ull;
    return m >> (-sh);
}

// Digit p as a bf16 bit pattern: an integer below 2^8 converts to FP32 exactly and its FP32
// pattern has 16 zero low bits, so the upper half is the exact bf16.  The digit is narrowed to 32
// bits before the conversion (a 64-bit integer conversion would run on the FP64 pipe).
__device__ __forceinline__ uint16_t oz_digit(unsigned long long X, int F, int b, int p, bool neg) {
    const float d = (float)(unsigned)((X >> (F - b * p)) & ((1ull << b) - 1ull));
    return (uint16_t)(__float_as_uint(neg ? -d : d) >> 16);
}

// Digit planes of the rows of a matrix (TRANS = false: output row r is source row r) or of its
// columns (TRANS = true: output row r is source column r, i.e. the source is K x R).  One CTA of
// 256 threads per 32 output rows; pass 1 finds each row's largest exponent, pass 2 writes the
// s planes (column-major sources go through a shared-memory tile so that both the reads and the
// writes are coalesced).
template <bool TRANS>
__global__ void __launch_bounds__(256) oz_split_kernel(OzSplitArgs a) {
    const int z = blockIdx.y, r0 = blockIdx.x * 32;
    const int tid = threadIdx.x, lane = tid & 31, wy = tid >> 5;
    const double* src = a.src + (size_t)z * a.sb;
    uint16_t* out = a.out + (size_t)z * a.s * a.R * a.Kp;
    __shared__ int s_emax[32];
    __shared__ uint16_t tile[32][34];
    if (tid < 32) s_emax[tid] = 1;
    __syncthreads();
    if (!TRANS) {
        for (int rr = wy; rr < 32; rr += 8) {
            const int r = r0 + rr;
            int e = 1;
            if (r < a.R)
                for (int k = lane; k < a.K; k += 32) e = max(e, biased_exp(src[(size_t)r * a.ld + k]));
            e = __reduce_max_sync(0xffffffffu, e);
            if (lane == 0) s_emax[rr] = e;
        }
    } else {
        const int r = r0 + lane;
        int e = 1;
        if (r < a.R)
            for (int k = wy; k < a.K; k += 8) e = max(e, biased_exp(src[(size_t)k * a.ld + r]));
        atomicMax(&s_emax[lane], e);
    }
    __syncthreads();
    if (tid < 32 && r0 + tid < a.R) {
        const int eb = s_emax[tid];
        if (eb >= 2046) set_err(a.err, DEV_NUMERIC);  // |v| >= 2^1023, inf or nan
        a.scale[(size_t)z * a.R + r0 + tid] = __longlong_as_double((long long)(min(eb, 2045) + 1) << 52);
    }
    const int F = a.b * a.s;
    if (!TRANS) {
        for (int rr = wy; rr < 32; rr += 8) {
            const int r = r0 + rr;
            if (r >= a.R) break;
            const int eb = s_emax[rr];
            for (int k = lane; k < a.Kp; k += 32) {
                bool neg = false;
                const unsigned long long X = (k < a.K) ? oz_fixed(src[(size_t)r * a.ld + k], eb, F, neg) : 0ull;
                for (int p = 1; p <= a.s; ++p) out[((size_t)(p - 1) * a.R + r) * a.Kp + k] = oz_digit(X, F, a.b, p, neg);
            }
        }
    } else {
        const int r = r0 + lane;
        const int eb = s_emax[lane];
        for (int k0 = 0; k0 < a.Kp; k0 += 32) {
            unsigned long long X[4];
            bool ng[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int k = k0 + wy + 8 * j;
                ng[j] = false;
                X[j] = (r < a.R && k < a.K) ? oz_fixed(src[(size_t)k * a.ld + r], eb, F, ng[j]) : 0ull;
            }
            for (int p = 1; p <= a.s; ++p) {
                __syncthreads();  // the previous plane's tile has been written out
#pragma unroll
                for (int j = 0; j < 4; ++j) tile[wy + 8 * j][lane] = oz_digit(X[j], F, a.b, p, ng[j]);
                __syncthreads();
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int ro = r0 + wy + 8 * j, k = k0 + lane;
                    if (ro < a.R && k < a.Kp) out[((size_t)(p - 1) * a.R + ro) * a.Kp + k] = tile[lane][wy + 8 * j];
                }
            }
        }
    }
}

struct OzPlan {
    int b = 0, s = 0;
    std::vector<std::vector<std::pair<int, int>>> groups;  // (p, q), 1-based digit indices
    long pairs = 0;
    double cost = 0.0;
};

// Estimated seconds: tensor passes bound by their operand traffic (a 128 x BN tile reads
// (128 + BN) x 2 bytes per K step: ~16 MACs per byte at ~6 TB/s), per group an FP64 epilogue
// (four FP64 operations and 16 bytes per output) and a launch.
static OzPlan oz_plan(int M, int N, int K, int batch) {
    OzPlan best;
    for (int b : {7, 6, 5}) {
        const double mx = (double)((1 << b) - 1) * (double)((1 << b) - 1);
        const long G = (long)floor(16777215.0 / ((double)K * mx));
        if (G < 1) continue;
        OzPlan p;
        p.b = b;
        p.s = (54 + b - 1) / b;
        const int gmax = (int)(G < TC_OZ_MAXP ? G : TC_OZ_MAXP);
        for (int d = 2; d <= p.s + 1; ++d) {
            std::vector<std::pair<int, int>> cur;
            for (int q = 1; q < d; ++q) {
                cur.emplace_back(d - q, q);
                ++p.pairs;
                if ((int)cur.size() == gmax) {
                    p.groups.push_back(cur);
                    cur.clear();
                }
            }
            if (!cur.empty()) p.groups.push_back(cur);
        }
        const double mn = (double)M * N * batch;
        p.cost = p.pairs * mn * K / 100e12 + (double)p.groups.size() * (mn * (4.0 / 600e9 + 16.0 / 4e12) + 4e-6);
        if (best.b == 0 || p.cost < best.cost) best = p;
    }
    return best;
}

// plane row length: K rounded up to 16 bytes (8 bf16), and at least one 64-wide TMA box
static int kpad(int K) { return K < 64 ? 64 : (K + 7) & ~7; }

}  // namespace

size_t ozaki_ws_bytes(int M, int N, int K, int batch) {
    return (size_t)OZ_SMAX * batch * ((size_t)M + N) * kpad(K) * sizeof(uint16_t);
}

size_t ozaki_sc_doubles(int M, int N, int batch) { return (size_t)batch * ((size_t)M + N); }

bool ozaki_pays(int M, int N, int K, int batch) {
    if (M < 64 || N < 64 || K < 1) return false;
    const OzPlan p = oz_plan(M, N, K, batch);
    if (p.b == 0) return false;
    const double split = ((double)M + N) * K * batch * (16.0 + 2.0 * p.s) / 4e12 + 8e-6;
    const double simt = 2.0 * M * N * (double)K * batch / 0.95e12;
    return p.cost + split < 0.8 * simt;
}

int ozaki_plan_info(int M, int N, int K, int batch, int* b, int* s, int* ngroups, int cap, int* np, int* pa,
                    int* pb) {
    if (M < 1 || N < 1 || K < 1 || batch < 1) return -1;
    const OzPlan plan = oz_plan(M, N, K, batch);
    if (plan.b == 0) return -1;
    *b = plan.b;
    *s = plan.s;
    *ngroups = (int)plan.groups.size();
    for (int g = 0; g < (int)plan.groups.size() && g < cap; ++g) {
        np[g] = (int)plan.groups[g].size();
        for (int i = 0; i < np[g]; ++i) {
            pa[g * TC_OZ_MAXP + i] = plan.groups[g][i].first;
            pb[g * TC_OZ_MAXP + i] = plan.groups[g][i].second;
        }
    }
    return 0;
}

cudaError_t ozaki_gemm(cudaStream_t st, const OzGemmArgs& g, void* ws, double* sc) {
    if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
    if (g.K <= 0) return cudaErrorInvalidValue;
    const OzPlan plan = oz_plan(g.M, g.N, g.K, g.batch);
    if (plan.b == 0) return cudaErrorInvalidValue;
    const int Kp = kpad(g.K);
    uint16_t* Ad = (uint16_t*)ws;
    uint16_t* Bd = Ad + (size_t)g.batch * plan.s * g.M * Kp;
    double* rsc = sc;
    double* csc = sc + (size_t)g.batch * g.M;
    OzSplitArgs sa;
    sa.src = g.A; sa.ld = g.lda; sa.sb = g.sA;
    sa.R = g.M; sa.K = g.K; sa.Kp = Kp; sa.b = plan.b; sa.s = plan.s;
    sa.out = Ad; sa.scale = rsc; sa.err = g.err;
    count_launch();
    oz_split_kernel<false><<<dim3((g.M + 31) / 32, g.batch), 256, 0, st>>>(sa);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    OzSplitArgs sb = sa;
    sb.src = g.B; sb.ld = g.ldb; sb.sb = g.sB;
    sb.R = g.N;
    sb.out = Bd; sb.scale = csc;
    count_launch();
    oz_split_kernel<true><<<dim3((g.N + 31) / 32, g.batch), 256, 0, st>>>(sb);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (size_t gi = 0; gi < plan.groups.size(); ++gi) {
        const auto& grp = plan.groups[gi];
        TcOzArgs t;
        t.M = g.M; t.N = g.N; t.K = g.K; t.Kp = Kp; t.batch = g.batch; t.ns = plan.s;
        t.Ad = Ad; t.Bd = Bd;
        t.np = (int)grp.size();
        for (int i = 0; i < t.np; ++i) {
            t.pa[i] = grp[i].first - 1;
            t.pb[i] = grp[i].second - 1;
        }
        const int d = grp[0].first + grp[0].second;
        t.C = g.C; t.ldc = g.ldc; t.sC = g.sC;
        t.rsc = rsc; t.csc = csc;
        t.gscale = ldexp(1.0, -plan.b * d);
        t.first = (gi == 0) ? 1 : 0;
        t.err = g.err;
        if ((e = tc_gemm_oz(st, t)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace afq
