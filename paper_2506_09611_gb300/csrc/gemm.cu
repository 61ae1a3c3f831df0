// gemm.cu -- SIMT tiled GEMM with diagonal scalings (FP64 / FP32), row-major.
//
// Used by the wrap G <- D E G E^{-1} D^{-1} (Eqs. BlMat, GrFMat), the rank-m
// flush of the delayed and block force-bias updates (Eqs. FinalDelay,
// BlkFrcBsTnew2 in G form) and the FP64 recompute (Eq. GrFMatNew).
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

}  // namespace

template <typename T>
cudaError_t gemm(cudaStream_t st, const GemmArgs<T>& g) {
    if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, g.batch);
    count_launch();
    gemm_kernel<T><<<grid, NT, 0, st>>>(g);
    return cudaGetLastError();
}

template cudaError_t gemm<float>(cudaStream_t, const GemmArgs<float>&);
template cudaError_t gemm<double>(cudaStream_t, const GemmArgs<double>&);

}  // namespace afq
