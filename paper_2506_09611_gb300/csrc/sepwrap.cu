// sepwrap.cu -- the device kernel and launcher of the separable wrap (tile code in sepwrap.cuh):
// one block per tile and matrix, 256 threads, the tile's two buffers in dynamic shared memory.
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

}  // namespace

// The default tile: 4 columns (rows), the narrowest the register-blocked passes take.  Narrow
// tiles give more blocks and more of them resident per SM (at 40 x 40 in FP32: 3 blocks of 58 KB
// per SM against 1 of 211 KB at 16 columns), which the passes' shared-memory latency needs.
template <typename T>
int sep_width(int L, int N) {
    return sep_smem_bytes<T>(L, N, 4) <= SEP_SMEM_CAP ? 4 : 0;
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
    // a.w > 0 asks for that tile width (a multiple of 4 whose tile fits on chip); 0 takes the default
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
template bool sep_width_fits<float>(int, int, int);
template bool sep_width_fits<double>(int, int, int);
template cudaError_t launch_sep<float>(cudaStream_t, const SepArgs&);
template cudaError_t launch_sep<double>(cudaStream_t, const SepArgs&);

}  // namespace afq
