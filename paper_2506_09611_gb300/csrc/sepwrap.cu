// sepwrap.cu -- the device kernels and launcher of the separable wrap (code in sepwrap.cuh): by
// default the line passes (a grid-stride loop of 256-thread blocks, four resident per SM, one line
// per thread per step); with an explicit tile width, one block per tile and matrix, 256 threads,
// the tile's two buffers in dynamic shared memory.
#include <algorithm>

#include "internal.h"
#include "sepwrap.cuh"

namespace afq {

namespace {

struct BlockSync {
    SEP_HD void operator()() const {
#ifdef __CUDA_ARCH__
        __syncthreads();
#endif
    }
};

template <typename T>
__global__ void __launch_bounds__(256) sep_kernel(SepArgs a) {
    extern __shared__ __align__(16) unsigned char sep_smem[];
    sep_tile<T>(a, blockIdx.x, blockIdx.y, threadIdx.x, blockDim.x, sep_smem, BlockSync());
}

constexpr size_t SEP_SMEM_CAP = 220 * 1024;

// Line passes: a grid-stride loop over the lines of the batch, A staged once per block.
constexpr int SEP_LINE_THREADS = 256;
constexpr int SEP_LINE_BLOCKS_PER_SM = 8;  // grid cap; three or four blocks are resident per SM

template <typename T, int LM>
__global__ void __launch_bounds__(SEP_LINE_THREADS) sep_line_kernel(SepLineArgs a, const double* A) {
    __shared__ __align__(16) T As[LM * LM];
    sep_line_load_A<T>(A, a.L, LM, As, threadIdx.x, blockDim.x);
    __syncthreads();
    const long total = sep_line_count(a) * a.batch;
    for (long line = (long)blockIdx.x * blockDim.x + threadIdx.x; line < total; line += (long)gridDim.x * blockDim.x)
        sep_line<T, LM>(a, line, As);
}

// Circulant A (SepArgs::circ) with a compile-time lattice side: its first row converted to T once
// per block into shared memory (the inner loop reads it as register operands or broadcast shared
// loads, never as FP64 loads with a conversion); two blocks per SM (128 registers: the line and a
// chunk of outputs).
template <typename T, int L>
__global__ void __launch_bounds__(SEP_LINE_THREADS, 2) sep_line_circ_kernel(SepLineArgs a, const double* A) {
    __shared__ T c[L];
    for (int d = threadIdx.x; d < L; d += blockDim.x) c[d] = (T)A[d];
    __syncthreads();
    const long total = sep_line_count(a) * a.batch;
    for (long line = (long)blockIdx.x * blockDim.x + threadIdx.x; line < total; line += (long)gridDim.x * blockDim.x)
        sep_line_circ<T, L>(a, line, c);
}

int device_sms() {
    static int nsm[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (nsm[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
        nsm[dev] = v;
    }
    return nsm[dev];
}

template <typename T>
cudaError_t launch_line(cudaStream_t st, const SepLineArgs& a, const double* A) {
    const long total = sep_line_count(a) * a.batch;
    if (total <= 0) return cudaSuccess;
    const long want = (total + SEP_LINE_THREADS - 1) / SEP_LINE_THREADS;
    const int grid = (int)std::min<long>(want, (long)device_sms() * SEP_LINE_BLOCKS_PER_SM);
    count_launch();
    if (a.circ && sep_circ_side<T>(a.L)) {
        switch (a.L) {
#define SEP_CIRC_CASE(LV) \
    case LV: sep_line_circ_kernel<T, (sizeof(T) == 4 || LV <= 16) ? LV : 4><<<grid, SEP_LINE_THREADS, 0, st>>>(a, A); break;
            SEP_CIRC_CASE(4)
            SEP_CIRC_CASE(6)
            SEP_CIRC_CASE(8)
            SEP_CIRC_CASE(12)
            SEP_CIRC_CASE(16)
            SEP_CIRC_CASE(20)
            SEP_CIRC_CASE(24)
            SEP_CIRC_CASE(32)
            SEP_CIRC_CASE(40)
#undef SEP_CIRC_CASE
            default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    switch (sep_line_lm(a.L)) {
#define SEP_LINE_CASE(LMV) \
    case LMV: sep_line_kernel<T, LMV><<<grid, SEP_LINE_THREADS, 0, st>>>(a, A); break;
        SEP_LINE_CASE(8)
        SEP_LINE_CASE(12)
        SEP_LINE_CASE(16)
        SEP_LINE_CASE(20)
        SEP_LINE_CASE(24)
        SEP_LINE_CASE(32)
        SEP_LINE_CASE(40)
        SEP_LINE_CASE(48)
        SEP_LINE_CASE(64)
#undef SEP_LINE_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

// The default tile: 4 columns (rows), the narrowest the register-blocked passes take.  Narrow
// tiles give more blocks and more of them resident per SM (at 40 x 40 in FP32: 3 blocks of 58 KB
// per SM against 1 of 211 KB at 16 columns), which the passes' shared-memory latency needs.
template <typename T>
int sep_width(int L, int N) {
    return sep_smem_bytes<T>(L, N, 4) <= SEP_SMEM_CAP ? 4 : 0;
}

template <typename T>
bool sep_available(int L, int N) {
    return L >= 2 && N == L * L && (sep_line_lm(L) > 0 || sep_width<T>(L, N) > 0);
}

template <typename T>
bool sep_width_fits(int L, int N, int w) {
    return w >= 4 && w % 4 == 0 && sep_smem_bytes<T>(L, N, w) <= SEP_SMEM_CAP;
}

template <typename T>
cudaError_t launch_sep(cudaStream_t st, const SepArgs& a0) {
    SepArgs a = a0;
    const int ext = a.C > 0 ? a.C : a.N;  // the untransformed extent
    if (a.L < 2 || a.N != a.L * a.L || a.batch < 1 || a.C < 0 || (a.side != 0 && a.side != 1) || !a.G || !a.A)
        return cudaErrorInvalidValue;
    if (a.ld < (a.side == 0 ? ext : a.N)) return cudaErrorInvalidValue;
    // a.w == 0: the line passes (two launches) where L <= 64; a.w > 0 asks for tiles of that width
    // (a multiple of 4 whose tile fits on chip)
    if (a.w == 0 && sep_line_lm(a.L) > 0) {
        SepLineArgs p1, p2;
        sep_line_passes(a, &p1, &p2);
        cudaError_t e = launch_line<T>(st, p1, a.A);
        if (e != cudaSuccess) return e;
        return launch_line<T>(st, p2, a.A);
    }
    if (a.w > 0) {
        if (!sep_width_fits<T>(a.L, a.N, a.w)) return cudaErrorInvalidValue;
    } else {
        a.w = sep_width<T>(a.L, a.N);
    }
    if (a.w == 0) return cudaErrorInvalidValue;  // the lattice is too large for an on-chip tile
    {
        cudaError_t e = ensure_smem_attr((const void*)sep_kernel<T>, SEP_SMEM_CAP);
        if (e != cudaSuccess) return e;
    }
    count_launch();
    sep_kernel<T><<<dim3((ext + a.w - 1) / a.w, a.batch), 256, sep_smem_bytes<T>(a.L, a.N, a.w), st>>>(a);
    return cudaGetLastError();
}

template int sep_width<float>(int, int);
template int sep_width<double>(int, int);
template bool sep_available<float>(int, int);
template bool sep_available<double>(int, int);
template bool sep_width_fits<float>(int, int, int);
template bool sep_width_fits<double>(int, int, int);
template cudaError_t launch_sep<float>(cudaStream_t, const SepArgs&);
template cudaError_t launch_sep<double>(cudaStream_t, const SepArgs&);

}  // namespace afq
