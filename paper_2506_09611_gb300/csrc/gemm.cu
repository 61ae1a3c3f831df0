// gemm.cu -- SIMT tiled GEMM with diagonal scalings (FP64 / FP32), row-major.
//
// Used by the wrap G <- D E G E^{-1} D^{-1} (Eqs. BlMat, GrFMat), the rank-m
// flush of the delayed and block force-bias updates (Eqs. FinalDelay,
// BlkFrcBsTnew2 in G form) and the FP64 recompute (Eq. GrFMatNew).  An FP32
// update C += alpha A B with a small inner dimension (K <= 64: a window's flush)
// takes rankm_kernel, written for that shape; everything else the general tile.
#include "internal.h"

namespace afq {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <typename T>
__global__ void __launch_bounds__(NT) gemm_kernel(GemmArgs<T> g) {
    const int z = blockIdx.z;
    const T* A = g.A + z * g.sA;
    const T* B = g.B + z * g.sB;
    T* C = g.C + z * g.sC;
    const T* rs = g.rs ? g.rs + z * g.srs : nullptr;
    const T* cs = g.cs ? g.cs + z * g.scs : nullptr;
    const T* bs = g.bs ? g.bs + z * g.sbs : nullptr;
    const int K = g.Kdev ? min(g.Kdev[g.kdiv > 0 ? z / g.kdiv : 0], g.K) : g.K;
    if (K <= 0 && g.beta == T(1) && g.cs == nullptr && g.rs == nullptr) return;  // C unchanged

    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

    for (int k0 = 0; k0 < K; k0 += BK) {
        // A tile: BM x BK, 4 elements per thread, k fastest for coalescing
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int e = tid + q * NT;
            int r = e / BK, kk = e % BK;
            int gm = m0 + r, gk = k0 + kk;
            As[kk][r] = (gm < g.M && gk < K) ? A[(long)gm * g.lda + gk] : T(0);
        }
        // B tile: BK x BN, n fastest
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int e = tid + q * NT;
            int kk = e / BN, c = e % BN;
            int gk = k0 + kk, gn = n0 + c;
            T v = (gk < K && gn < g.N) ? B[(long)gk * g.ldb + gn] : T(0);
            if (bs && gk < K) v *= bs[gk];
            Bs[kk][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int gm = m0 + ty + 16 * i;
        if (gm >= g.M) continue;
        T r = rs ? rs[gm] : T(1);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int gn = n0 + tx + 16 * j;
            if (gn >= g.N) continue;
            T v = g.alpha * r * acc[i][j];
            if (cs) v *= cs[gn];
            long o = (long)gm * g.ldc + gn;
            C[o] = (g.beta == T(0)) ? v : v + g.beta * C[o];
        }
    }
}

// C += alpha A B for a small inner dimension (K <= RM_KMAX, FP32): the rank-m flush of a window,
// a read-modify-write of C with a short product per element.  128 x 64 output tiles, 256 threads
// of 8 x 4 outputs (rows ty*4 + i and 64 + ty*4 + i, columns tx*4 .. tx*4 + 3): the whole K of
// both panels is staged in shared memory at once (A transposed), so there is one barrier per tile,
// every shared-memory read is a 16-byte vector (32 multiply-adds per three reads) and C moves in
// 16-byte vectors.  Requires N, the leading dimensions and batch strides to be multiples of 4
// and 16-byte aligned bases (checked by the dispatcher).
constexpr int RM_BM = 128, RM_BN = 64, RM_KMAX = 64, RM_NT = 256;
constexpr int RM_PA = RM_BM + 4, RM_PB = RM_BN + 4;
constexpr size_t RM_SMEM = (size_t)RM_KMAX * (RM_PA + RM_PB) * sizeof(float);

__global__ void __launch_bounds__(RM_NT, 4) rankm_kernel(GemmArgs<float> g) {
    const int z = blockIdx.z;
    const float* A = g.A + z * g.sA;
    const float* B = g.B + z * g.sB;
    float* C = g.C + z * g.sC;
    const int K = g.Kdev ? min(g.Kdev[g.kdiv > 0 ? z / g.kdiv : 0], g.K) : g.K;
    if (K <= 0) return;  // beta = 1: C unchanged
    extern __shared__ __align__(16) float rm_smem[];
    float* As = rm_smem;                  // [RM_KMAX][RM_PA]: As[k][r] = A[m0 + r][k]
    float* Bs = As + RM_KMAX * RM_PA;     // [RM_KMAX][RM_PB]: Bs[k][c] = B[k][n0 + c]
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * RM_BM, n0 = blockIdx.x * RM_BN;
    const int M = g.M, N = g.N, K4 = (K + 3) >> 2;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    // A panel: thread item e -> row r = e % RM_BM, k = 4 (e / RM_BM) .. + 3 (entries k >= K land in
    // rows of As that the product never reads; the row has lda >= 4 K4 entries)
    for (int e = tid; e < RM_BM * K4; e += RM_NT) {
        const int r = e % RM_BM, k4 = e / RM_BM, row = m0 + r;
        const float4 v = (row < M) ? *(const float4*)(A + (long)row * g.lda + 4 * k4) : zero;
        As[(4 * k4 + 0) * RM_PA + r] = v.x;
        As[(4 * k4 + 1) * RM_PA + r] = v.y;
        As[(4 * k4 + 2) * RM_PA + r] = v.z;
        As[(4 * k4 + 3) * RM_PA + r] = v.w;
    }
    // B panel: K rows of RM_BN columns in 16-byte vectors
    for (int e = tid; e < K * (RM_BN / 4); e += RM_NT) {
        const int c4 = e % (RM_BN / 4), k = e / (RM_BN / 4), col = n0 + 4 * c4;
        const float4 v = (col < N) ? *(const float4*)(B + (long)k * g.ldb + col) : zero;
        *(float4*)(Bs + k * RM_PB + 4 * c4) = v;
    }
    __syncthreads();
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
#pragma unroll 4
    for (int kk = 0; kk < K; ++kk) {
        const float4 a0 = *(const float4*)(As + kk * RM_PA + ty * 4);
        const float4 a1 = *(const float4*)(As + kk * RM_PA + 64 + ty * 4);
        const float4 b = *(const float4*)(Bs + kk * RM_PB + tx * 4);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    const int col = n0 + tx * 4;
    if (col >= N) return;
    const float al = g.alpha;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int row = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        if (row >= M) continue;
        float4* p = (float4*)(C + (long)row * g.ldc + col);
        float4 o = *p;
        o.x = fmaf(al, acc[i][0], o.x);
        o.y = fmaf(al, acc[i][1], o.y);
        o.z = fmaf(al, acc[i][2], o.z);
        o.w = fmaf(al, acc[i][3], o.w);
        *p = o;
    }
}

template <typename T>
bool rankm_ok(const GemmArgs<T>& g) {
    if constexpr (sizeof(T) != 4) {
        return false;
    } else {
        auto al = [](const void* p) { return ((size_t)p & 15) == 0; };
        return g.beta == T(1) && !g.rs && !g.cs && !g.bs && g.K >= 1 && g.K <= RM_KMAX && g.N % 4 == 0 &&
               g.lda % 4 == 0 && g.ldb % 4 == 0 && g.ldc % 4 == 0 && g.sA % 4 == 0 && g.sB % 4 == 0 &&
               g.sC % 4 == 0 && g.lda >= 4 * ((g.K + 3) / 4) && g.ldb >= g.N && g.ldc >= g.N && al(g.A) &&
               al(g.B) && al(g.C);
    }
}

}  // namespace

template <typename T>
cudaError_t gemm(cudaStream_t st, const GemmArgs<T>& g) {
    if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
    if constexpr (sizeof(T) == 4) {
        if (rankm_ok(g)) {
            cudaError_t e = ensure_smem_attr((const void*)rankm_kernel, RM_SMEM);
            if (e != cudaSuccess) return e;
            dim3 grid((g.N + RM_BN - 1) / RM_BN, (g.M + RM_BM - 1) / RM_BM, g.batch);
            count_launch();
            rankm_kernel<<<grid, RM_NT, RM_SMEM, st>>>(g);
            return cudaGetLastError();
        }
    }
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, g.batch);
    count_launch();
    gemm_kernel<T><<<grid, NT, 0, st>>>(g);
    return cudaGetLastError();
}

template cudaError_t gemm<float>(cudaStream_t, const GemmArgs<float>&);
template cudaError_t gemm<double>(cudaStream_t, const GemmArgs<double>&);

}  // namespace afq
