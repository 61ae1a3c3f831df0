// flips.cu -- stateless application of accepted field changes to G in one
// rank-m product (the G form of Eqs. FinalDelay and BlkFrcBsTnew2):
//     G_s <- G_s - G_s[:, I] W_s (E_I^T - G_s[I, :]),
//     W_s  = D_s (1 + (1 - G_s[I, I]) D_s)^{-1},   (D_s)_aa = exp(c_s (x'_a - x_a)) - 1.
#include <math.h>

#include "internal.h"

namespace afq {

// Scratch layout (bytes), pitch NW = window_max<T>() as in the sweep's flush:
//   [0, 256)      int m, int err, ...
//   [256, ...)    idx[NW] (validated copy of the sites)
//   Wm            2 * NW * NW * T
//   X             2 * N * NW * T
//   Y             4 * NW * N * T
template <typename T>
size_t flips_scratch_bytes(int N) {
    const size_t NW = (size_t)window_max<T>();
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    return 256 + al(NW * sizeof(int)) + al(2 * NW * NW * sizeof(T)) + al(2 * (size_t)N * NW * sizeof(T)) +
           al(4 * NW * (size_t)N * sizeof(T));
}

template <typename T>
static WindowBufs flips_layout(unsigned char* scratch, int N) {
    const size_t NW = (size_t)window_max<T>();
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    WindowBufs wb;
    wb.m = (int*)scratch;
    size_t off = 256;
    wb.idx = (int*)(scratch + off);
    off += al(NW * sizeof(int));
    wb.Wm = scratch + off;
    wb.Wx = nullptr;
    off += al(2 * NW * NW * sizeof(T));
    wb.X = scratch + off;
    off += al(2 * (size_t)N * NW * sizeof(T));
    wb.Y = scratch + off;
    wb.dtot = nullptr;
    return wb;
}

// One CTA: validate the sites, then W_s for both spins by Gauss-Jordan with partial pivoting
// on [M | 1] in shared memory, M = 1 + (1 - G_II) D.  The status word wb.m[1] is rewritten by every
// call: 0, DEV_ARG (a site outside [0, N)) or DEV_NUMERIC (a zero pivot); on either error wb.m[0]
// (the product's inner dimension) is 0, so G is left unchanged.
template <typename T>
__global__ void __launch_bounds__(1024) flips_W_kernel(const T* __restrict__ Gu, const T* __restrict__ Gd, long ld,
                                                       int N, const int* sites, const double* delta, int m,
                                                       WindowBufs wb, int NWC) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int AP = 2 * m + 1;
    T* Aug = (T*)smem_raw;
    T* colk = Aug + (size_t)m * AP;
    __shared__ int s_piv, s_bad, s_num;
    if (tid == 0) {
        s_bad = 0;
        s_num = 0;
    }
    __syncthreads();
    for (int a = tid; a < m; a += nt) {
        int v = sites[a];
        if (v < 0 || v >= N) s_bad = 1;
        wb.idx[a] = (v < 0 || v >= N) ? 0 : v;
    }
    __syncthreads();
    if (s_bad) {  // nothing is applied: the product below sees m = 0
        if (tid == 0) {
            wb.m[0] = 0;
            wb.m[1] = DEV_ARG;
        }
        return;
    }
    if (tid == 0) {
        wb.m[0] = m;
        wb.m[1] = 0;
    }
    const T* G[2] = {Gu, Gd};
    for (int s = 0; s < 2; ++s) {
        for (int e = tid; e < m * m; e += nt) {
            int a = e / m, c = e % m;
            double A0 = (a == c ? 1.0 : 0.0) - (double)G[s][(long)wb.idx[a] * ld + wb.idx[c]];
            Aug[a * AP + c] = (T)((a == c ? 1.0 : 0.0) + A0 * delta[s * m + c]);
            Aug[a * AP + m + c] = (a == c) ? T(1) : T(0);
        }
        __syncthreads();
        for (int k = 0; k < m; ++k) {
            if (tid < 32) {
                T best = T(-1);
                int br = k;
                for (int r = k + tid; r < m; r += 32) {
                    T v = fabs(Aug[r * AP + k]);
                    if (v > best) { best = v; br = r; }
                }
                for (int o = 16; o > 0; o >>= 1) {
                    T ob = __shfl_down_sync(0xffffffffu, best, o);
                    int orr = __shfl_down_sync(0xffffffffu, br, o);
                    if (ob > best || (ob == best && orr < br)) { best = ob; br = orr; }
                }
                if (tid == 0) {
                    s_piv = br;
                    if (!(best > T(0))) s_num = 1;
                }
            }
            __syncthreads();
            const int pr = s_piv;
            if (pr != k)
                for (int c = tid; c < 2 * m; c += nt) {
                    T t0 = Aug[k * AP + c];
                    Aug[k * AP + c] = Aug[pr * AP + c];
                    Aug[pr * AP + c] = t0;
                }
            __syncthreads();
            const T inv = T(1) / Aug[k * AP + k];
            for (int r = tid; r < m; r += nt) colk[r] = Aug[r * AP + k];
            __syncthreads();
            for (int c = tid; c < 2 * m; c += nt) Aug[k * AP + c] *= inv;
            __syncthreads();
            for (int e = tid; e < m * 2 * m; e += nt) {
                int r = e / (2 * m), c = e % (2 * m);
                if (r == k) continue;
                Aug[r * AP + c] -= colk[r] * Aug[k * AP + c];
            }
            __syncthreads();
        }
        T* Wm = (T*)wb.Wm + (size_t)s * NWC * NWC;
        for (int e = tid; e < m * m; e += nt) {
            int a = e / m, c = e % m;
            Wm[a * NWC + c] = (T)(delta[s * m + a] * (double)Aug[a * AP + m + c]);
        }
        __syncthreads();
    }
    if (tid == 0 && s_num) {  // singular: apply nothing
        wb.m[0] = 0;
        wb.m[1] = DEV_NUMERIC;
    }
}

template <typename T>
static cudaError_t apply_flips_impl(cudaStream_t st, int N, long ld, T* Gu, T* Gd, const int* sites,
                                    const double* delta, int m, unsigned char* scratch) {
    const int NWC = window_max<T>();
    WindowBufs wb = flips_layout<T>(scratch, N);
    size_t shm = (size_t)m * (2 * (size_t)m + 1) * sizeof(T) + (size_t)m * sizeof(T);
    const size_t mx = (size_t)NWC * (2 * (size_t)NWC + 1) * sizeof(T) + (size_t)NWC * sizeof(T);
    cudaError_t e = ensure_smem_attr((const void*)flips_W_kernel<T>, mx);
    if (e != cudaSuccess) return e;
    count_launch();
    flips_W_kernel<T><<<1, 1024, shm, st>>>(Gu, Gd, ld, N, sites, delta, m, wb, NWC);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    SiteParams sp{};
    sp.N = N;
    sp.ld = ld;
    return launch_flush<T>(st, Gu, Gd, sp, wb, m);
}

// Copy the call's device status word (wb.m[1], at byte 4 of the scratch) to the host on the call's
// stream, wait for the stream, and map it to an ABI code.
static int flips_status(cudaStream_t st, const unsigned char* scratch) {
    int h = 0;
    if (cudaMemcpyAsync(&h, scratch + sizeof(int), sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return AFQMC_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return AFQMC_ERR_CUDA;
    if (h == DEV_ARG) return AFQMC_ERR_ARG;
    if (h == DEV_NUMERIC) return AFQMC_ERR_NUMERIC;
    return h == 0 ? AFQMC_OK : AFQMC_ERR_CUDA;
}

static int flips_check(int precision, int N, long long ld, void* G_up, void* G_dn, const int* sites,
                       const double* delta, int m) {
    if (precision != AFQMC_PREC_FP64 && precision != AFQMC_PREC_FP32) return AFQMC_ERR_ARG;
    const int NW = precision == AFQMC_PREC_FP64 ? window_max<double>() : window_max<float>();
    if (N < 1 || ld < N || m < 0 || m > NW || !G_up || !G_dn) return AFQMC_ERR_ARG;
    if (m > 0 && (!sites || !delta)) return AFQMC_ERR_ARG;
    return AFQMC_OK;
}

}  // namespace afq

using namespace afq;

extern "C" int afqmc_apply_flips(int precision, int N, long long ld, void* G_up, void* G_dn, const int* sites,
                                 const double* delta, int m, void* stream) {
    int rc = flips_check(precision, N, ld, G_up, G_dn, sites, delta, m);
    if (rc) return rc;
    if (m == 0) return AFQMC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = precision == AFQMC_PREC_FP64 ? flips_scratch_bytes<double>(N) : flips_scratch_bytes<float>(N);
    void* scratch = nullptr;
    if (cudaMallocAsync(&scratch, bytes, st) != cudaSuccess) return AFQMC_ERR_OOM;
    cudaError_t e = precision == AFQMC_PREC_FP64
                        ? apply_flips_impl<double>(st, N, (long)ld, (double*)G_up, (double*)G_dn, sites, delta, m,
                                                   (unsigned char*)scratch)
                        : apply_flips_impl<float>(st, N, (long)ld, (float*)G_up, (float*)G_dn, sites, delta, m,
                                                  (unsigned char*)scratch);
    const int rs = (e == cudaSuccess) ? flips_status(st, (const unsigned char*)scratch) : AFQMC_ERR_CUDA;
    cudaError_t e2 = cudaFreeAsync(scratch, st);
    if (rs != AFQMC_OK) return rs;
    return e2 == cudaSuccess ? AFQMC_OK : AFQMC_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// No-allocation variant.
//
// Some callers cannot allocate device memory at the point where they apply an
// update: code that runs under a fixed device-memory budget owned by a host
// framework, code inside a real-time loop where an allocation (and the
// synchronisation cudaMalloc may imply) is not allowed, or a plugin whose host
// process gives it no allocator.  afqmc_apply_flips_noalloc does exactly the
// work of afqmc_apply_flips, with its scratch in the file-scope device array
// below instead of cudaMallocAsync.
//
// The array is sized for lattices up to NOALLOC_MAX_N sites in either
// precision; every GPU that loads this library holds it until the process
// exits.  Host code cannot use the array's name as a device address, so the
// first call on each device looks the address up with cudaGetSymbolAddress
// while that device is current and caches it.
// ---------------------------------------------------------------------------
namespace afq {

constexpr int NOALLOC_MAX_N = 4096;

constexpr size_t noalloc_align(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t noalloc_bytes_for(size_t NW, size_t esz, size_t N) {
    return 256 + noalloc_align(NW * sizeof(int)) + noalloc_align(2 * NW * NW * esz) + noalloc_align(2 * N * NW * esz) +
           noalloc_align(4 * NW * N * esz);
}
constexpr size_t NOALLOC_BYTES_F32 = noalloc_bytes_for(128, 4, NOALLOC_MAX_N);
constexpr size_t NOALLOC_BYTES_F64 = noalloc_bytes_for(64, 8, NOALLOC_MAX_N);
constexpr size_t NOALLOC_BYTES = NOALLOC_BYTES_F32 > NOALLOC_BYTES_F64 ? NOALLOC_BYTES_F32 : NOALLOC_BYTES_F64;

static __device__ __align__(256) unsigned char g_flips_scratch[NOALLOC_BYTES];

}  // namespace afq

#include <mutex>

namespace {
constexpr int NOALLOC_MAXDEV = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[NOALLOC_MAXDEV] = {};
}  // namespace

extern "C" int afqmc_apply_flips_noalloc(int precision, int N, long long ld, void* G_up, void* G_dn,
                                         const int* sites, const double* delta, int m, void* stream) {
    int rc = afq::flips_check(precision, N, ld, G_up, G_dn, sites, delta, m);
    if (rc) return rc;
    if (N > afq::NOALLOC_MAX_N) return AFQMC_ERR_ARG;
    const size_t need = precision == AFQMC_PREC_FP64 ? afq::flips_scratch_bytes<double>(N)
                                                     : afq::flips_scratch_bytes<float>(N);
    if (need > afq::NOALLOC_BYTES) return AFQMC_ERR_ARG;
    if (m == 0) return AFQMC_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAXDEV) return AFQMC_ERR_CUDA;
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, afq::g_flips_scratch) != cudaSuccess || !p) return AFQMC_ERR_CUDA;
            g_noalloc_addr[dev] = p;
        }
        scratch = g_noalloc_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = precision == AFQMC_PREC_FP64
                        ? afq::apply_flips_impl<double>(st, N, (long)ld, (double*)G_up, (double*)G_dn, sites, delta,
                                                        m, (unsigned char*)scratch)
                        : afq::apply_flips_impl<float>(st, N, (long)ld, (float*)G_up, (float*)G_dn, sites, delta, m,
                                                       (unsigned char*)scratch);
    if (e != cudaSuccess) return AFQMC_ERR_CUDA;
    return afq::flips_status(st, (const unsigned char*)scratch);
}
