// setup.cu -- model matrices, FP64 re-orthonormalisation / solve, measurements.
//
//   exp(-tau K) for the periodic square lattice (Eq. 2DHubbard): the dispersion
//   eps_k = -2t(cos kx + cos ky) separates, so E = Ex (x) Ey with
//   Ex_{x,x'} = L^{-1} sum_k exp(2 tau t cos k) cos(k (x - x')).
#include <math.h>

#include "internal.h"

namespace afq {

// ---------------------------------------------------------------------------
// exp(-tau K)
// ---------------------------------------------------------------------------
__global__ void expK_kernel(int L, double t, double tau, double* E, long ld) {
    extern __shared__ double f1[];  // 1D factor by displacement
    for (int d = threadIdx.x; d < L; d += blockDim.x) {
        double acc = 0.0;
        for (int q = 0; q < L; ++q) {
            double k = 2.0 * M_PI * q / L;
            acc += exp(2.0 * tau * t * cos(k)) * cos(k * d);
        }
        f1[d] = acc / L;
    }
    __syncthreads();
    const int N = L * L;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < (long)N * N; e += (long)gridDim.x * blockDim.x) {
        int i = (int)(e / N), j = (int)(e % N);
        int dx = ((i % L) - (j % L) + L) % L, dy = ((i / L) - (j / L) + L) % L;
        E[(long)i * ld + j] = f1[dx] * f1[dy];
    }
}

cudaError_t launch_expK(cudaStream_t st, int L, double t, double tau, double* E, long ld) {
    count_launch();
    expK_kernel<<<256, 256, L * sizeof(double), st>>>(L, t, tau, E, ld);
    return cudaGetLastError();
}

__global__ void expK1d_kernel(int L, double t, double tau, double* Ex) {
    // Ex[x][x'] = L^{-1} sum_k exp(2 tau t cos k) cos(k (x - x')), k = 2 pi q / L
    for (int e = threadIdx.x; e < L * L; e += blockDim.x) {
        int x = e / L, xp = e % L;
        int d = ((x - xp) % L + L) % L;
        double acc = 0.0;
        for (int q = 0; q < L; ++q) {
            double k = 2.0 * M_PI * q / L;
            acc += exp(2.0 * tau * t * cos(k)) * cos(k * d);
        }
        Ex[e] = acc / L;
    }
}

cudaError_t launch_expK1d(cudaStream_t st, int L, double t, double tau, double* Ex) {
    count_launch();
    expK1d_kernel<<<1, 256, 0, st>>>(L, t, tau, Ex);
    return cudaGetLastError();
}

__global__ void scale_rows_kernel(double* U, int rows, int cols, const double* d) {
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < (long)rows * cols; e += (long)gridDim.x * blockDim.x)
        U[e] *= d[e / cols];
}
__global__ void scale_cols_kernel(double* U, int rows, int cols, const double* d) {
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < (long)rows * cols; e += (long)gridDim.x * blockDim.x)
        U[e] *= d[e % cols];
}
cudaError_t launch_scale_rows(cudaStream_t st, double* U, int rows, int cols, const double* d) {
    count_launch();
    scale_rows_kernel<<<512, 256, 0, st>>>(U, rows, cols, d);
    return cudaGetLastError();
}
cudaError_t launch_scale_cols(cudaStream_t st, double* U, int rows, int cols, const double* d) {
    count_launch();
    scale_cols_kernel<<<512, 256, 0, st>>>(U, rows, cols, d);
    return cudaGetLastError();
}

template <typename T>
__global__ void scale2_kernel(T* G, long ld, int N, long sG, const T* a, const T* b) {
    const int s = blockIdx.y;  // batch entry (walker, spin)
    T* g = G + s * sG;
    const T* as = a + (size_t)s * N;
    const T* bs = b + (size_t)s * N;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < (long)N * N; e += (long)gridDim.x * blockDim.x) {
        int i = (int)(e / N), j = (int)(e % N);
        g[(long)i * ld + j] *= as[i] * bs[j];
    }
}
template <typename T>
cudaError_t launch_scale2(cudaStream_t st, T* G, long ld, int N, long sG, const T* a, const T* b, int nbatch) {
    count_launch();
    scale2_kernel<T><<<dim3(512, nbatch), 256, 0, st>>>(G, ld, N, sG, a, b);
    return cudaGetLastError();
}
template cudaError_t launch_scale2<float>(cudaStream_t, float*, long, int, long, const float*, const float*, int);
template cudaError_t launch_scale2<double>(cudaStream_t, double*, long, int, long, const double*, const double*, int);

template <typename T>
__global__ void cast_kernel(const double* src, long lds, T* dst, long ldd, int rows, int cols, long ssrc, long sdst) {
    src += blockIdx.y * ssrc;
    dst += blockIdx.y * sdst;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < (long)rows * cols; e += (long)gridDim.x * blockDim.x) {
        int r = (int)(e / cols), c = (int)(e % cols);
        dst[(long)r * ldd + c] = (T)src[(long)r * lds + c];
    }
}
template <typename T>
cudaError_t launch_cast(cudaStream_t st, const double* src, long lds, T* dst, long ldd, int rows, int cols, int nbatch,
                        long ssrc, long sdst) {
    count_launch();
    cast_kernel<T><<<dim3(512, nbatch), 256, 0, st>>>(src, lds, dst, ldd, rows, cols, ssrc, sdst);
    return cudaGetLastError();
}
template cudaError_t launch_cast<float>(cudaStream_t, const double*, long, float*, long, int, int, int, long, long);
template cudaError_t launch_cast<double>(cudaStream_t, const double*, long, double*, long, int, int, int, long, long);

template <typename T>
__global__ void to_double_kernel(const T* src, long lds, double* dst, long ldd, int rows, int cols) {
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < (long)rows * cols; e += (long)gridDim.x * blockDim.x) {
        int r = (int)(e / cols), c = (int)(e % cols);
        dst[(long)r * ldd + c] = (double)src[(long)r * lds + c];
    }
}
template <typename T>
cudaError_t launch_to_double(cudaStream_t st, const T* src, long lds, double* dst, long ldd, int rows, int cols) {
    count_launch();
    to_double_kernel<T><<<512, 256, 0, st>>>(src, lds, dst, ldd, rows, cols);
    return cudaGetLastError();
}
template cudaError_t launch_to_double<float>(cudaStream_t, const float*, long, double*, long, int, int);
template cudaError_t launch_to_double<double>(cudaStream_t, const double*, long, double*, long, int, int);

// d_i = exp(c x_i), dinv_i = exp(-c x_i) for both spins; c2 = {c_up, c_dn}; outputs [2][N] with stride sd
template <typename T>
__global__ void field_scales_kernel(const int8_t* x, int N, double c0, double c1, T* d, T* dinv, long sd, long xstride) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    x += blockIdx.y * xstride;  // walker blockIdx.y of a group: outputs [walker][2][N]
    d += (size_t)blockIdx.y * 2 * sd;
    dinv += (size_t)blockIdx.y * 2 * sd;
    double xv = (double)x[i];
    d[i] = (T)exp(c0 * xv);
    dinv[i] = (T)exp(-c0 * xv);
    d[sd + i] = (T)exp(c1 * xv);
    dinv[sd + i] = (T)exp(-c1 * xv);
}
template <typename T>
cudaError_t launch_field_scales_T(cudaStream_t st, const int8_t* x, int N, const double* c2, T* d, T* dinv, long sd,
                                  int nwk, long xstride) {
    count_launch();
    field_scales_kernel<T><<<dim3((N + 255) / 256, nwk), 256, 0, st>>>(x, N, c2[0], c2[1], d, dinv, sd, xstride);
    return cudaGetLastError();
}
template cudaError_t launch_field_scales_T<float>(cudaStream_t, const int8_t*, int, const double*, float*, float*, long,
                                                  int, long);
template cudaError_t launch_field_scales_T<double>(cudaStream_t, const int8_t*, int, const double*, double*, double*,
                                                   long, int, long);

// ---------------------------------------------------------------------------
// FP64 propagation of the walker factors over several slices (Sec. II.C), fused.
// A factor is a set of vectors of length N = L*L (columns of U_R, rows of U_L), vector v element
// i = x + L*y at U[v * vs + i * es].  E = exp(-dtau K) = Ex (x) Ex on the periodic square lattice,
// so E v is Ex M Ex for the L x L matrix M[y][x] = v[x + L*y].  Per slice l (in the given order):
//   right factor (B_l U):  v <- D_l (E v);      left factor (U B_l): v <- E (D_l v),
// with D_l = diag(exp(c x_{l,i})) (x = +-1, so D_l picks exp(+c) or exp(-c)).  Each CTA keeps
// PV_VEC vectors in shared memory for all slices.  Grid (vector blocks, spin).
// ---------------------------------------------------------------------------
constexpr int PV_VEC = 10;
__global__ void __launch_bounds__(256) prop_kernel(PropArgs a, int vpc) {
    const int s = blockIdx.y & 1, wk = blockIdx.y >> 1;  // factor (walker, spin)
    double* U = a.U0 + wk * a.wstride + s * a.sstride;
    const int L = a.L, N = L * L, nvec = a.nvec[s];
    const long vs = a.vs[s], es = a.es[s];
    const int8_t* xw = a.x + wk * a.xstride;
    const int v0 = blockIdx.x * vpc;
    if (v0 >= nvec) return;
    const int nv = min(vpc, nvec - v0);
    const double dp = a.dplus[s], dm = a.dminus[s];
    extern __shared__ __align__(16) double pv_smem[];
    double* Ex = pv_smem;            // [L][L]
    double* T = Ex + L * L;          // [L][L]
    double* V = T + L * L;           // [nv][N]
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < L * L; e += nt) Ex[e] = a.Ex[e];
    for (int e = tid; e < nv * N; e += nt) {
        const int v = e / N, i = e - v * N;
        V[e] = U[(long)(v0 + v) * vs + (long)i * es];
    }
    __syncthreads();
    for (int t = 0; t < a.nsl; ++t) {
        const int ell = a.l_first + t * a.l_step;
        const int8_t* xl = xw + (size_t)(ell - 1) * N;
        if (a.left)
            for (int e = tid; e < nv * N; e += nt) V[e] *= (xl[e % N] > 0) ? dp : dm;
        __syncthreads();
        for (int v = 0; v < nv; ++v) {
            double* M = V + (size_t)v * N;
            // (four independent accumulators: FP64 multiply-add latency is long on this part)
            for (int e = tid; e < N; e += nt) {  // T = Ex M  (along y)
                const int y = e / L, x = e - y * L;
                double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
                int yp = 0;
                for (; yp + 3 < L; yp += 4) {
                    a0 += Ex[y * L + yp] * M[yp * L + x];
                    a1 += Ex[y * L + yp + 1] * M[(yp + 1) * L + x];
                    a2 += Ex[y * L + yp + 2] * M[(yp + 2) * L + x];
                    a3 += Ex[y * L + yp + 3] * M[(yp + 3) * L + x];
                }
                for (; yp < L; ++yp) a0 += Ex[y * L + yp] * M[yp * L + x];
                T[e] = (a0 + a1) + (a2 + a3);
            }
            __syncthreads();
            for (int e = tid; e < N; e += nt) {  // M = T Ex  (along x)
                const int y = e / L, x = e - y * L;
                double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
                int xp = 0;
                for (; xp + 3 < L; xp += 4) {
                    a0 += T[y * L + xp] * Ex[xp * L + x];
                    a1 += T[y * L + xp + 1] * Ex[(xp + 1) * L + x];
                    a2 += T[y * L + xp + 2] * Ex[(xp + 2) * L + x];
                    a3 += T[y * L + xp + 3] * Ex[(xp + 3) * L + x];
                }
                for (; xp < L; ++xp) a0 += T[y * L + xp] * Ex[xp * L + x];
                M[e] = (a0 + a1) + (a2 + a3);
            }
            __syncthreads();
        }
        if (!a.left) {
            for (int e = tid; e < nv * N; e += nt) V[e] *= (xl[e % N] > 0) ? dp : dm;
            __syncthreads();
        }
    }
    for (int e = tid; e < nv * N; e += nt) {
        const int v = e / N, i = e - v * N;
        U[(long)(v0 + v) * vs + (long)i * es] = V[e];
    }
}

cudaError_t launch_prop(cudaStream_t st, const PropArgs& a) {
    const int N = a.L * a.L;
    const long room = 220 * 1024 / 8 - 2L * a.L * a.L;  // doubles left for the vectors
    const int vpc = (int)((room / N < PV_VEC) ? room / N : PV_VEC);
    if (vpc < 1) return cudaErrorInvalidValue;  // lattice too large to keep one vector on chip
    const size_t shm = ((size_t)2 * a.L * a.L + (size_t)vpc * N) * sizeof(double);
    {
        cudaError_t e = ensure_smem_attr((const void*)prop_kernel, 220 * 1024);
        if (e != cudaSuccess) return e;
    }
    const int nv = a.nvec[0] > a.nvec[1] ? a.nvec[0] : a.nvec[1];
    count_launch();
    prop_kernel<<<dim3((nv + vpc - 1) / vpc, a.nmat), 256, shm, st>>>(a, vpc);
    return cudaGetLastError();
}

template <typename T>
__global__ void identity_minus_kernel(T* G, long ld, int N, long sG) {
    G += blockIdx.y * sG;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < (long)N * N; e += (long)gridDim.x * blockDim.x) {
        int i = (int)(e / N), j = (int)(e % N);
        G[(long)i * ld + j] = (i == j ? T(1) : T(0)) - G[(long)i * ld + j];
    }
}
template <typename T>
cudaError_t launch_identity_minus(cudaStream_t st, T* G, long ld, int N, int nbatch, long sG) {
    count_launch();
    identity_minus_kernel<T><<<dim3(512, nbatch), 256, 0, st>>>(G, ld, N, sG);
    return cudaGetLastError();
}
template cudaError_t launch_identity_minus<float>(cudaStream_t, float*, long, int, int, long);
template cudaError_t launch_identity_minus<double>(cudaStream_t, double*, long, int, int, long);

// acc2[0] += sum (Gold - Gnew)^2, acc2[1] += sum Gnew^2; Gnew is FP64 with the same ld
template <typename T>
__global__ void drift_kernel(const T* Gold, const double* Gnew, long ld, int N, double* acc2, long sold, long snew,
                             int adiv) {
    Gold += blockIdx.y * sold;
    Gnew += blockIdx.y * snew;
    acc2 += 2 * (blockIdx.y / adiv);
    double a = 0.0, bsum = 0.0;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < (long)N * N; e += (long)gridDim.x * blockDim.x) {
        int i = (int)(e / N), j = (int)(e % N);
        double gn = Gnew[(long)i * ld + j];
        double d = (double)Gold[(long)i * ld + j] - gn;
        a += d * d;
        bsum += gn * gn;
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        bsum += __shfl_down_sync(0xffffffffu, bsum, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(acc2, a);
        atomicAdd(acc2 + 1, bsum);
    }
}
template <typename T>
cudaError_t launch_drift(cudaStream_t st, const T* Gold, const T* Gnew, long ld, int N, double* acc2, int nbatch,
                         long sold, long snew, int adiv) {
    count_launch();
    drift_kernel<T><<<dim3(256, nbatch), 256, 0, st>>>(Gold, (const double*)Gnew, ld, N, acc2, sold, snew, adiv);
    return cudaGetLastError();
}
template cudaError_t launch_drift<float>(cudaStream_t, const float*, const float*, long, int, double*, int, long, long,
                                         int);
template cudaError_t launch_drift<double>(cudaStream_t, const double*, const double*, long, int, double*, int, long,
                                          long, int);

// E = sum_s tr(K A^s) + U sum_i (n_up n_dn - (n_up + n_dn)/2), A = 1 - G, K_ij = -t per bond
template <typename T>
__global__ void energy_kernel(const T* Gu0, long ld, int L, double t, double U, double* out, long gstride) {
    const int N = L * L;
    const T* Gu = Gu0 + blockIdx.y * gstride;  // walker blockIdx.y of a group
    const T* Gd = Gu + (size_t)N * ld;
    out += blockIdx.y;
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        int x = i % L, y = i / L;
        int nbr[4] = {((x + 1) % L) + L * y, ((x - 1 + L) % L) + L * y, x + L * ((y + 1) % L), x + L * ((y - 1 + L) % L)};
        for (int q = 0; q < 4; ++q) {
            int j = nbr[q];
            double aju = (j == i ? 1.0 : 0.0) - (double)Gu[(long)j * ld + i];
            double ajd = (j == i ? 1.0 : 0.0) - (double)Gd[(long)j * ld + i];
            acc += -t * (aju + ajd);
        }
        double nu = 1.0 - (double)Gu[(long)i * ld + i], nd = 1.0 - (double)Gd[(long)i * ld + i];
        acc += U * (nu * nd - 0.5 * (nu + nd));
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}
template <typename T>
cudaError_t launch_energy(cudaStream_t st, const T* Gu, long ld, int L, double t, double U, double* out, int nwk,
                          long gstride) {
    count_launch();
    energy_kernel<T><<<dim3(64, nwk), 256, 0, st>>>(Gu, ld, L, t, U, out, gstride);
    return cudaGetLastError();
}
template cudaError_t launch_energy<float>(cudaStream_t, const float*, long, int, double, double, double*, int, long);
template cudaError_t launch_energy<double>(cudaStream_t, const double*, long, int, double, double, double*, int, long);

}  // namespace afq
