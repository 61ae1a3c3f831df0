// soc.cu -- the spin-orbit-coupled sweep (Appendix A): the complex Green's function of the 2N
// orbitals (i spin up, N + i spin down), auxiliary fields acting as 2 x 2 matrices on the pairs
// (i, N + i) -- real rotations (the spin-y channel) or the phases diag(e^{i gamma x}, e^{-i gamma x})
// of the imaginary spin-z channel (Eqs. HSspinDecomp, BIOpForHubbard; with lam = 0 the paper's
// attractive Hubbard model) -- and rank-2 updates per site.
//
// Layout.  A complex matrix with C columns is stored "row-split": row r holds the real parts of
// its C entries, padded to ldz, then the imaginary parts, padded to ldz (2 ldz elements per row).
// The bulk G of walker j is 2N rows of 2 ldz elements in the bulk precision T.  With that layout
// a product X C by a constant complex C is one real product with the realified
//   C~ = [[Re C, Im C], [-Im C, Re C]]   (2 ldz x 2 ldz),
// and a product E S is the real product [Re E | Im E] . [[Re S, Im S], [-Im S, Re S]], whose
// right operand is filled from S by one copy pass.  The wrap is therefore two real GEMMs of
// 2N x 2ldz x 2ldz (the four real products of a complex GEMM) plus the rotation pass D G D^{-1}.
//
// Updates.  A window of n sites works on the 2n x 2n block of the current G on its orbitals
// (ordered site by site: up, down).  Delayed / local: warp 0 tests the sites on that block (ratio
// R = det(1 + delta A_SS), Eqs. DetRatioSOC, LocalSOC; 32 at a time with a ballot) and an
// accepted site updates the trailing rows and columns of the block by the rank-2 formula.  Block
// force bias: the stripped spin-flip expectations come from (1 + Delta_s)(1 + A_bb Delta_s)^{-1}
// A_bb of the block, the flipped set F is proposed jointly and tested with det(1 + A_FF Delta_F).
// Either way the window ends with
//   W = Delta_F (1 + A_FF Delta_F)^{-1}   (in-place Gauss-Jordan with 2 x 2 pivot blocks; the pivot
// determinants are the successive ratios, non-zero for accepted moves) and the full G takes the
// rank-2m update  G <- G - (G[:, F] W)(E_F^T - G[F, :]) out of place (soc_xw_kernel, then
// soc_flush_kernel into the second G buffer).  Windows of up to 32 sites are pipelined: window
// w + 1 reads the G before window w's update and applies that update to its own block, while
// window w's X' and flush run on a second stream.
//
// FP64 recompute.  The factors U_R (2N x n_e) and U_L^+ are carried realified, as 4N x 2n_e real
// matrices (rows: real parts, then imaginary parts); the column space of the realified factor
// determines G exactly, so the realified factor is re-orthonormalised by the blocked pivoted LU
// of lu.cu like the spin-decoupled factors.  Propagation applies B_l = D(x_l) exp(-dtau H0) to
// each column in shared memory through the lattice Fourier transform (exp(-dtau H0) is the 2 x 2
// block e^{-dtau h_k} per momentum), in FP64.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/afqmc_soc.h"
#include "internal.h"

namespace afq {
namespace {

// ---------------------------------------------------------------------------
// complex helpers
// ---------------------------------------------------------------------------
template <typename T>
struct cx {
    T r, i;
};
template <typename T>
__host__ __device__ __forceinline__ cx<T> cmk(T r, T i) {
    cx<T> z;
    z.r = r;
    z.i = i;
    return z;
}
template <typename T>
__host__ __device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) { return cmk(a.r + b.r, a.i + b.i); }
template <typename T>
__host__ __device__ __forceinline__ cx<T> csub(cx<T> a, cx<T> b) { return cmk(a.r - b.r, a.i - b.i); }
template <typename T>
__host__ __device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
    return cmk(a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r);
}
template <typename T>
__host__ __device__ __forceinline__ cx<T> cscale(cx<T> a, T s) { return cmk(a.r * s, a.i * s); }
// a += b c
template <typename T>
__host__ __device__ __forceinline__ void cfma(cx<T>& a, cx<T> b, cx<T> c) {
    a.r = fma(b.r, c.r, fma(-b.i, c.i, a.r));
    a.i = fma(b.r, c.i, fma(b.i, c.r, a.i));
}
template <typename T>
__host__ __device__ __forceinline__ cx<T> cinv(cx<T> a) {
    const T d = a.r * a.r + a.i * a.i;
    return cmk(a.r / d, -a.i / d);
}

// 2 x 2 complex block, row-major
template <typename T>
struct c22 {
    cx<T> a[2][2];
};

// The field's 2 x 2 matrix is A(t) = exp(t g), t = gamma x: the spin-y channel (hs = 0,
// g = [[0, 1], [-1, 0]]) gives the rotation [[cos t, sin t], [-sin t, cos t]], the spin-z channel
// (hs = 1, g = diag(i, -i)) the phases diag(e^{it}, e^{-it}).
// The flip of site field x (-> -x): delta = A(-2 gamma x) - 1; stripping the field (x -> 0):
// A(-gamma x) - 1.  With (cm1, s) = (cos 2gamma - 1, sin 2gamma) or (cos gamma - 1, sin gamma):
//   spin-y: [[cm1, -x s], [x s, cm1]];   spin-z: diag(cm1 - i x s, cm1 + i x s).
struct SocConsts {
    double c2m1, s2;  // cos(2 gamma) - 1, sin(2 gamma)
    double c1m1, s1;  // cos(gamma) - 1, sin(gamma)
    double gamma;
    int hs;           // AFQMC_SOC_HS_SY or AFQMC_SOC_HS_SZ
};

template <typename T>
__device__ __forceinline__ void site_delta(int hs, double cm1, double s, int x, cx<T> d[2][2]) {
    if (hs == AFQMC_SOC_HS_SZ) {
        d[0][0] = cmk((T)cm1, (T)(-x * s));
        d[1][1] = cmk((T)cm1, (T)(x * s));
        d[0][1] = cmk((T)0, (T)0);
        d[1][0] = cmk((T)0, (T)0);
        return;
    }
    d[0][0] = cmk((T)cm1, (T)0);
    d[1][1] = cmk((T)cm1, (T)0);
    d[0][1] = cmk((T)(-x * s), (T)0);
    d[1][0] = cmk((T)(x * s), (T)0);
}

// ---------------------------------------------------------------------------
// wrap kernels
// ---------------------------------------------------------------------------

// G <- A_r G A_c on every pair block {i, N+i} x {j, N+j}, both parts: rows by A(rs gamma x_i),
// columns by right multiplication with A(cs gamma x_j).  Forward wrap: rs = +1, cs = -1
// (D G D^{-1}); backward: rs = -1, cs = +1.  Spin-y: a real rotation of each part; spin-z: the
// entry (s i, s' j) times e^{i gamma (f_s rs x_i + f_s' cs x_j)}, f_up = 1, f_dn = -1.
template <typename T>
__global__ void soc_rot_kernel(T* G0, long ldz, int N, long gstride, const int8_t* x0, long xstride, T cg, T sg,
                               int rs, int cs, int hs) {
    const int j = blockIdx.x * 32 + threadIdx.x;
    const int i = blockIdx.y * 8 + threadIdx.y;
    if (i >= N || j >= N) return;
    T* G = G0 + (long)blockIdx.z * gstride;
    const int8_t* x = x0 + (long)blockIdx.z * xstride;
    const T sr = (T)(rs * x[i]) * sg, sc = (T)(cs * x[j]) * sg;
    const long ld2 = 2 * ldz;
    if (hs == AFQMC_SOC_HS_SZ) {
        // row phase e^{i f_s t_r} = cg + i f_s sr, column phase cg + i f_s' sc
        const cx<T> pr[2] = {cmk(cg, sr), cmk(cg, -sr)}, pc[2] = {cmk(cg, sc), cmk(cg, -sc)};
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const long o = (long)(s * N + i) * ld2 + t * N + j;
                const cx<T> v = cmul(cmul(cmk(G[o], G[o + ldz]), pr[s]), pc[t]);
                G[o] = v.r;
                G[o + ldz] = v.i;
            }
        return;
    }
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        T* g = G + p * ldz;
        const T a = g[(long)i * ld2 + j], b = g[(long)i * ld2 + N + j];
        const T c = g[(long)(N + i) * ld2 + j], d = g[(long)(N + i) * ld2 + N + j];
        const T a1 = cg * a + sr * c, b1 = cg * b + sr * d;
        const T c1 = cg * c - sr * a, d1 = cg * d - sr * b;
        g[(long)i * ld2 + j] = a1 * cg - b1 * sc;
        g[(long)i * ld2 + N + j] = a1 * sc + b1 * cg;
        g[(long)(N + i) * ld2 + j] = c1 * cg - d1 * sc;
        g[(long)(N + i) * ld2 + N + j] = c1 * sc + d1 * cg;
    }
}

// Fill the second half of the realified right operand of E S.
//   rows == 1 (row-major S~, 2 ldz x 2 ldz, rows [0, n) hold [Re S | Im S]):
//       row ldz + r = [-Im S[r] | Re S[r]]
//   rows == 0 (its transpose, the K-major operand of the tensor-core product, columns [0, n)
//       hold [[Re S^T], [Im S^T]]): column ldz + m = [[-Im S^T], [Re S^T]] column m.
template <typename T>
__global__ void soc_realify_kernel(T* S0, long ldz, int n, long sstride, int rows) {
    T* S = S0 + (long)blockIdx.z * sstride;
    const long ld2 = 2 * ldz;
    if (rows) {
        const int r = blockIdx.y;
        for (long c = blockIdx.x * blockDim.x + threadIdx.x; c < ld2; c += (long)gridDim.x * blockDim.x)
            S[(ldz + r) * ld2 + c] = (c < ldz) ? -S[(long)r * ld2 + ldz + c] : S[(long)r * ld2 + c - ldz];
    } else {
        const long nrow = blockIdx.y;  // rows of the K-major operand: 2 ldz of them
        for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x)
            S[nrow * ld2 + ldz + m] = (nrow < ldz) ? -S[(nrow + ldz) * ld2 + m] : S[(nrow - ldz) * ld2 + m];
    }
}

// ---------------------------------------------------------------------------
// the window chain
// ---------------------------------------------------------------------------
struct SocWinArgs {
    const void* G0;
    long gstride, ldz;
    int N;
    int8_t* x0;
    long xstride;        // fields of the slice, walker j at x0 + j xstride
    const double* u0;    // uniforms, 2N per walker
    const uint8_t* rep;  // nullable, 2N per walker
    int mode;            // 0: site chain (local / delayed), 1: block force bias
    int s0, n, blk;      // window sites [s0, s0 + n), block index (mode 1)
    SocConsts k;
    uint8_t* dec0;       // 2N per walker
    double* ratio0;      // 2N complex per walker
    double* lam0;        // N per walker
    int* sites0;         // kmax per walker: accepted (flipped) sites in order
    int kmax;
    void* W0;            // W (2m x 2m complex, leading dimension 2 kmax) per walker
    int* Kdev;           // per walker: 2m (complex orbitals of the update), 0 = no update
    int* err;
    // pipelined windows: G0 is the G before the previous window's update, which is applied to the
    // window's block here from the previous window's W (pW), flipped sites (psites) and size
    // (pKdev); corr = 0 reads G0 as the current G
    int corr;
    const void* pW;
    const int* psites;
    const int* pKdev;
    void* Gw0;           // per walker (2 kmax)^2 complex: the window's block of the current G
};

constexpr int SOC_PIPE_N = 32;  // windows of up to 32 sites run pipelined (the correction's staging buffer)

template <typename T>
__device__ __forceinline__ cx<T> g_at(const T* G, long ldz, int r, int c) {
    return cmk(G[(long)r * 2 * ldz + c], G[(long)r * 2 * ldz + ldz + c]);
}

// In-place inverse of the 2m x 2m complex matrix M (row stride ldm) by Gauss-Jordan with the
// 2 x 2 diagonal blocks as pivots (every thread inverts the pivot block itself, so a step costs
// two barriers).  det (thread 0 only, nullable) receives the product of the pivot block
// determinants, i.e. det M.  colF: 2 * 2m complex scratch.  Returns false (on every thread) if a
// pivot block is singular or not finite.
template <typename T>
__device__ bool gj_inverse_2x2(cx<T>* M, int m2, int ldm, cx<T>* colF, cx<T>* det) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int per = nt / m2, jj = tid % m2, i0 = tid / m2;  // 2D map of the trailing update
    cx<T> dacc = cmk((T)1, (T)0);
    for (int t = 0; t < m2 / 2; ++t) {
        const int q0 = 2 * t;
        __syncthreads();
        const cx<T> a = M[q0 * ldm + q0], b = M[q0 * ldm + q0 + 1];
        const cx<T> c = M[(q0 + 1) * ldm + q0], d = M[(q0 + 1) * ldm + q0 + 1];
        const cx<T> dt = csub(cmul(a, d), cmul(b, c));
        const T mag = dt.r * dt.r + dt.i * dt.i;
        if (!(mag > (T)0) || !isfinite(mag)) return false;  // uniform: every thread read the same block
        const cx<T> di = cinv(dt);
        c22<T> P;
        P.a[0][0] = cmul(d, di);
        P.a[0][1] = cmul(cmk(-b.r, -b.i), di);
        P.a[1][0] = cmul(cmk(-c.r, -c.i), di);
        P.a[1][1] = cmul(a, di);
        dacc = cmul(dacc, dt);
        __syncthreads();  // every thread has read the pivot block
        for (int j = tid; j < m2; j += nt) {
            if (j == q0 || j == q0 + 1) {
                colF[2 * j] = cmk((T)0, (T)0);
                colF[2 * j + 1] = cmk((T)0, (T)0);
                continue;
            }
            const cx<T> u = M[q0 * ldm + j], v = M[(q0 + 1) * ldm + j];
            cx<T> nu = cmul(P.a[0][0], u), nv = cmul(P.a[1][0], u);
            cfma(nu, P.a[0][1], v);
            cfma(nv, P.a[1][1], v);
            M[q0 * ldm + j] = nu;
            M[(q0 + 1) * ldm + j] = nv;
            colF[2 * j] = M[j * ldm + q0];
            colF[2 * j + 1] = M[j * ldm + q0 + 1];
        }
        __syncthreads();
        if (i0 < per) {
            const int j = jj;
            const bool jp = (j == q0 || j == q0 + 1);
            const cx<T> p0 = M[q0 * ldm + j], p1 = M[(q0 + 1) * ldm + j];
            for (int i = i0; i < m2; i += per) {
                if (i == q0 || i == q0 + 1) {
                    if (jp) M[i * ldm + j] = P.a[i - q0][j - q0];
                    continue;
                }
                const cx<T> f0 = colF[2 * i], f1 = colF[2 * i + 1];
                if (jp) {
                    const int p = j - q0;
                    cx<T> w = cmul(f0, P.a[0][p]);
                    cfma(w, f1, P.a[1][p]);
                    M[i * ldm + j] = cmk(-w.r, -w.i);
                } else {
                    cx<T> w = M[i * ldm + j];
                    cfma(w, cmk(-f0.r, -f0.i), p0);
                    cfma(w, cmk(-f1.r, -f1.i), p1);
                    M[i * ldm + j] = w;
                }
            }
        }
    }
    __syncthreads();
    if (det && threadIdx.x == 0) *det = dacc;
    return true;
}

// W = Delta_F Minv (2m x 2m complex, leading dimension ldw).  Delta_F is block diagonal: the
// 2 x 2 block dl[t] of flipped site t.
template <typename T>
__device__ void write_W(const cx<T>* Minv, int m2, int ldm, const cx<T> (*dl)[2][2], cx<T>* W, int ldw) {
    for (int e = threadIdx.x; e < m2 * m2; e += blockDim.x) {
        const int q = e / m2, qq = e - q * m2;
        const int t = q >> 1, p = q & 1;
        cx<T> w = cmul(dl[t][p][0], Minv[(2 * t) * ldm + qq]);
        cfma(w, dl[t][p][1], Minv[(2 * t + 1) * ldm + qq]);
        W[(long)q * ldw + qq] = w;
    }
}

// The flip delta of site field x and the 2 x 2 test of the site block g (all in registers):
// R = det(1 + delta A), W2 = delta (1 + A delta)^{-1}, A = 1 - g.
template <typename T>
__device__ __forceinline__ cx<T> site_test(const cx<T> g[2][2], const cx<T> dl[2][2], c22<T>& w2) {
    cx<T> A[2][2], m1[2][2], m2[2][2];
    for (int p = 0; p < 2; ++p)
        for (int q = 0; q < 2; ++q) A[p][q] = cmk((p == q ? (T)1 : (T)0) - g[p][q].r, -g[p][q].i);
    for (int p = 0; p < 2; ++p)
        for (int q = 0; q < 2; ++q) {
            m1[p][q] = cmk(p == q ? (T)1 : (T)0, (T)0);
            m2[p][q] = m1[p][q];
            for (int r = 0; r < 2; ++r) {
                cfma(m1[p][q], dl[p][r], A[r][q]);
                cfma(m2[p][q], A[p][r], dl[r][q]);
            }
        }
    const cx<T> R = csub(cmul(m1[0][0], m1[1][1]), cmul(m1[0][1], m1[1][0]));
    const cx<T> d2 = csub(cmul(m2[0][0], m2[1][1]), cmul(m2[0][1], m2[1][0]));
    const cx<T> di = cinv(d2);
    const cx<T> inv[2][2] = {{cmul(m2[1][1], di), cmul(cmk(-m2[0][1].r, -m2[0][1].i), di)},
                             {cmul(cmk(-m2[1][0].r, -m2[1][0].i), di), cmul(m2[0][0], di)}};
    for (int p = 0; p < 2; ++p)
        for (int q = 0; q < 2; ++q) {
            w2.a[p][q] = cmul(dl[p][0], inv[0][q]);
            cfma(w2.a[p][q], dl[p][1], inv[1][q]);
        }
    return R;
}

template <typename T>
__global__ void __launch_bounds__(512) soc_window_kernel(SocWinArgs a) {
    extern __shared__ __align__(16) unsigned char soc_smem[];
    const int z = blockIdx.x;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int N = a.N, n = a.n, s0 = a.s0, n2 = 2 * n;
    const long ldz = a.ldz;
    const T* G = (const T*)a.G0 + (long)z * a.gstride;
    int8_t* x = a.x0 + (long)z * a.xstride;
    const double* u = a.u0 + (long)z * 2 * N;
    const uint8_t* rep = a.rep ? a.rep + (long)z * 2 * N : nullptr;
    uint8_t* dec = a.dec0 + (long)z * 2 * N;
    double* ratio = a.ratio0 + (long)z * 4 * N;
    double* lam = a.lam0 + (long)z * N;
    int* sites = a.sites0 + (long)z * a.kmax;
    cx<T>* W = (cx<T>*)a.W0 + (long)z * 4 * a.kmax * a.kmax;
    const int ldw = 2 * a.kmax;

    cx<T>* Mw = (cx<T>*)soc_smem;               // (2 kmax)^2: the window block / the LU matrix
    cx<T>* aux = Mw + 4 * a.kmax * a.kmax;      // 8 kmax: column / row snapshots, GJ scratch
    cx<T>* Ys = aux + 8 * a.kmax;               // (2 SOC_PIPE_N)^2: staging of the correction
    cx<T>* Gw = (cx<T>*)a.Gw0 + (long)z * 4 * a.kmax * a.kmax;  // n2 x n2: the block of the current G
    __shared__ cx<T> s_dl[64][2][2];            // flip deltas of the flipped sites
    __shared__ int s_site[64];
    __shared__ T s_uT[64];
    __shared__ int s_x[64], s_rep[64];
    __shared__ int s_m, s_acc;
    __shared__ T s_logq;
    __shared__ c22<T> s_w2;
    __shared__ cx<T> s_det;
    auto orb = [&](int q) { return (q & 1) ? N + s0 + (q >> 1) : s0 + (q >> 1); };

    for (int t = tid; t < n; t += nt) {
        s_uT[t] = (T)u[s0 + t];
        s_x[t] = x[s0 + t];
        s_rep[t] = rep ? (int)rep[s0 + t] : -1;
    }
    // ---- the window's block of the current G, into Gw ----
    {
        const int m2p = a.corr ? a.pKdev[z] : 0;
        if (m2p == 0) {
            for (int e = tid; e < n2 * n2; e += nt) {
                const int r = e / n2, c = e - r * n2;
                Gw[e] = g_at(G, ldz, orb(r), orb(c));
            }
        } else {
            // G = G0 - (G0[:, Fp] Wp) (E_Fp^T - G0[Fp, :]) on the block (the previous window's update)
            const int* ps = a.psites + (long)z * a.kmax;
            const cx<T>* pW = (const cx<T>*)a.pW + (long)z * 4 * a.kmax * a.kmax;
            auto porb = [&](int q) { return (q & 1) ? N + ps[q >> 1] : ps[q >> 1]; };
            // Wp staged after T1 in the block buffer when it fits (the FP32 window buffer does)
            const bool wsh = n2 * m2p + m2p * m2p <= 4 * a.kmax * a.kmax;
            cx<T>* Wsh = Mw + n2 * m2p;
            for (int e = tid; e < n2 * m2p; e += nt) {  // G0[block, Fp]
                const int r = e / m2p, q = e - r * m2p;
                Ys[e] = g_at(G, ldz, orb(r), porb(q));
            }
            if (wsh)
                for (int e = tid; e < m2p * m2p; e += nt) Wsh[e] = pW[(long)(e / m2p) * ldw + e % m2p];
            __syncthreads();
            for (int e = tid; e < n2 * m2p; e += nt) {  // T1 = G0[block, Fp] Wp
                const int r = e / m2p, q = e - r * m2p;
                cx<T> v0 = cmk((T)0, (T)0), v1 = cmk((T)0, (T)0);
                int p = 0;
                if (wsh) {
                    for (; p + 1 < m2p; p += 2) {
                        cfma(v0, Ys[r * m2p + p], Wsh[p * m2p + q]);
                        cfma(v1, Ys[r * m2p + p + 1], Wsh[(p + 1) * m2p + q]);
                    }
                    if (p < m2p) cfma(v0, Ys[r * m2p + p], Wsh[p * m2p + q]);
                } else {
                    for (; p < m2p; ++p) cfma(v0, Ys[r * m2p + p], pW[(long)p * ldw + q]);
                }
                Mw[e] = cadd(v0, v1);
            }
            __syncthreads();
            for (int e = tid; e < m2p * n2; e += nt) {  // E_Fp^T - G0[Fp, block]
                const int q = e / n2, c = e - q * n2;
                const int o = porb(q), oc = orb(c);
                const cx<T> g = g_at(G, ldz, o, oc);
                Ys[e] = cmk((o == oc ? (T)1 : (T)0) - g.r, -g.i);
            }
            __syncthreads();
            for (int e = tid; e < n2 * n2; e += nt) {
                const int r = e / n2, c = e - r * n2;
                cx<T> v = g_at(G, ldz, orb(r), orb(c)), v1 = cmk((T)0, (T)0);
                int q = 0;
                for (; q + 1 < m2p; q += 2) {
                    const cx<T> t0 = Mw[r * m2p + q], t1 = Mw[r * m2p + q + 1];
                    cfma(v, cmk(-t0.r, -t0.i), Ys[q * n2 + c]);
                    cfma(v1, cmk(-t1.r, -t1.i), Ys[(q + 1) * n2 + c]);
                }
                if (q < m2p) {
                    const cx<T> t0 = Mw[r * m2p + q];
                    cfma(v, cmk(-t0.r, -t0.i), Ys[q * n2 + c]);
                }
                Gw[e] = cadd(v, v1);
            }
        }
        __syncthreads();
    }
    auto gl = [&](int r, int c) { return Gw[r * n2 + c]; };  // local orbitals 2t + p
    int m2 = 0;  // complex orbitals of the window's update (uniform)
    if (a.mode == 0) {
        // ---- sites one after another on the 2n x 2n block ----
        for (int e = tid; e < n2 * n2; e += nt) Mw[e] = Gw[e];
        __syncthreads();
        int m = 0;
        cx<T>* colW = aux;           // [n2][2]
        cx<T>* rowY = aux + 2 * n2;  // [2][n2]
        __shared__ int s_next, s_apos;
        int t = 0;
        while (t < n) {
            if (warp == 0) {
                // warp 0 tests the next 32 sites at once on the current block (a rejection leaves G
                // unchanged) and a ballot finds the first acceptance; all lanes of a site agree
                const int q = t + lane;
                bool acc = false, fin = true;
                cx<T> R = cmk((T)0, (T)0);
                c22<T> w2;
                cx<T> dl[2][2];
                int xi = 0;
                if (q < n) {
                    xi = s_x[q];
                    site_delta<T>(a.k.hs, a.k.c2m1, a.k.s2, xi, dl);
                    cx<T> g[2][2];
                    for (int p = 0; p < 2; ++p)
                        for (int qq = 0; qq < 2; ++qq) g[p][qq] = Mw[(2 * q + p) * n2 + 2 * q + qq];
                    R = site_test<T>(g, dl, w2);
                    // the test in the bulk precision (the FP32 bulk rounds u to float: a bias below
                    // 2^-25 in the acceptance probability)
                    const T absR = sqrt(R.r * R.r + R.i * R.i);
                    fin = isfinite(absR);
                    acc = (s_rep[q] >= 0 ? (s_rep[q] != 0) : (s_uT[q] < absR)) && fin && absR > (T)0;
                    if (!fin) set_err(a.err, DEV_NUMERIC);
                }
                const unsigned ball = __ballot_sync(0xffffffffu, acc);
                const int first = ball ? __ffs(ball) - 1 : 32;
                if (q < n && lane <= first) {
                    const int i = s0 + q;
                    ratio[2 * i] = (double)R.r;
                    ratio[2 * i + 1] = (double)R.i;
                    dec[i] = (uint8_t)(lane == first);
                }
                if (first < 32) {
                    // snapshot of the accepted site's rank-2 factors on the trailing rows / columns
                    c22<T> wv;
#pragma unroll
                    for (int p = 0; p < 2; ++p)
#pragma unroll
                        for (int qq = 0; qq < 2; ++qq) {
                            wv.a[p][qq].r = __shfl_sync(0xffffffffu, w2.a[p][qq].r, first);
                            wv.a[p][qq].i = __shfl_sync(0xffffffffu, w2.a[p][qq].i, first);
                        }
                    const int at = t + first, c0 = 2 * at + 2;
                    for (int r = c0 + lane; r < n2; r += 32) {
                        const cx<T> g0 = Mw[r * n2 + 2 * at], g1 = Mw[r * n2 + 2 * at + 1];
                        for (int qq = 0; qq < 2; ++qq) {
                            cx<T> v = cmul(g0, wv.a[0][qq]);
                            cfma(v, g1, wv.a[1][qq]);
                            colW[2 * r + qq] = v;
                        }
                        for (int p = 0; p < 2; ++p) {
                            const cx<T> gg = Mw[(2 * at + p) * n2 + r];
                            rowY[p * n2 + r] = cmk(-gg.r, -gg.i);  // E_S^T - G[S, :] beyond the site
                        }
                    }
                    if (lane == first) {
                        for (int p = 0; p < 2; ++p)
                            for (int qq = 0; qq < 2; ++qq) s_dl[m][p][qq] = dl[p][qq];
                        s_site[m] = s0 + q;
                        sites[m] = s0 + q;
                        x[s0 + q] = (int8_t)(-xi);
                    }
                }
                if (lane == 0) {
                    s_apos = first < 32 ? t + first : -1;
                    s_next = first < 32 ? t + first + 1 : min(n, t + 32);
                }
            }
            __syncthreads();
            const int at = s_apos;
            t = s_next;
            if (at < 0) continue;
            ++m;
            // trailing rank-2 update: rows and columns after the accepted site (earlier ones are
            // never read again; W comes from the window's starting G)
            const int c0 = 2 * at + 2, w = n2 - c0;
            if (w > 0) {
                const int per = nt / w, cc = tid % w, r0 = tid / w;
                if (r0 < per) {
                    const int c = c0 + cc;
                    const cx<T> y0 = rowY[c], y1 = rowY[n2 + c];
                    for (int r = c0 + r0; r < n2; r += per) {
                        cx<T> v = Mw[r * n2 + c];
                        const cx<T> q0 = colW[2 * r], q1 = colW[2 * r + 1];
                        cfma(v, cmk(-q0.r, -q0.i), y0);
                        cfma(v, cmk(-q1.r, -q1.i), y1);
                        Mw[r * n2 + c] = v;
                    }
                }
            }
            __syncthreads();
        }
        if (m == 0) {
            if (tid == 0) a.Kdev[z] = 0;
            return;
        }
        // M = 1 + A_FF Delta_F from the window's starting block
        m2 = 2 * m;
        for (int e = tid; e < m2 * m2; e += nt) {
            const int q = e / m2, qq = e - q * m2;
            const int t2 = qq >> 1, p2 = qq & 1;
            const int lq = 2 * (s_site[q >> 1] - s0) + (q & 1);
            cx<T> v = cmk((q == qq) ? (T)1 : (T)0, (T)0);
            for (int p = 0; p < 2; ++p) {
                const int lc = 2 * (s_site[t2] - s0) + p;
                const cx<T> gg = gl(lq, lc);
                const cx<T> Aq = cmk((lq == lc ? (T)1 : (T)0) - gg.r, -gg.i);
                cfma(v, Aq, s_dl[t2][p][p2]);
            }
            Mw[e] = v;
        }
        if (!gj_inverse_2x2<T>(Mw, m2, m2, aux, nullptr)) {
            if (tid == 0) {
                set_err(a.err, DEV_NUMERIC);
                a.Kdev[z] = 0;
            }
            return;
        }
    } else {
        // ---- block force bias over the block [s0, s0 + n) ----
        __syncthreads();
        // stripped matrix Mb = 1 + A_bb Delta_s, Delta_s = A(-gamma x) - 1 per site
        for (int e = tid; e < n2 * n2; e += nt) {
            const int q = e / n2, qq = e - q * n2;
            const int t2 = qq >> 1, p2 = qq & 1;
            cx<T> ds[2][2];
            site_delta<T>(a.k.hs, a.k.c1m1, a.k.s1, s_x[t2], ds);
            cx<T> v = cmk((q == qq) ? (T)1 : (T)0, (T)0);
            for (int p = 0; p < 2; ++p) {
                const int cq = 2 * t2 + p;
                const cx<T> g = gl(q, cq);
                const cx<T> Aq = cmk((q == cq ? (T)1 : (T)0) - g.r, -g.i);
                cfma(v, Aq, ds[p][p2]);
            }
            Mw[e] = v;
        }
        if (!gj_inverse_2x2<T>(Mw, n2, n2, aux, nullptr)) {
            if (tid == 0) {
                set_err(a.err, DEV_NUMERIC);
                a.Kdev[z] = 0;
            }
            return;
        }
        // (Minv A)[2t + p][2t + q] for the four entries of every site: one warp per (t, p, q)
        {
            const int nw = nt >> 5;
            for (int e = warp; e < 4 * n; e += nw) {
                const int t = e >> 2, p = (e >> 1) & 1, q = e & 1;
                const int row = 2 * t + p, col = 2 * t + q;
                cx<T> acc = cmk((T)0, (T)0);
                for (int r = lane; r < n2; r += 32) {
                    const cx<T> g = gl(r, col);
                    const cx<T> Ar = cmk((r == col ? (T)1 : (T)0) - g.r, -g.i);
                    cfma(acc, Mw[row * n2 + r], Ar);
                }
                for (int o = 16; o > 0; o >>= 1) {
                    acc.r += __shfl_xor_sync(0xffffffffu, acc.r, o);
                    acc.i += __shfl_xor_sync(0xffffffffu, acc.i, o);
                }
                if (lane == 0) aux[e] = acc;  // aux[4t + 2p + q]
            }
        }
        __syncthreads();
        if (tid == 0) {
            // obar_t = the stripped expectation of the field's generator, Abar = (1 + Delta_s) Minv A,
            // 1 + Delta_s = A(-gamma x): spin-y Abar[dn t, up t] - Abar[up t, dn t], spin-z
            // i (Abar[up t, up t] - Abar[dn t, dn t]); the proposal weight of x' is exp(x' h),
            // h = gamma Re(obar) (bulk precision)
            T logq = 0;
            int m = 0;
            for (int t = 0; t < n; ++t) {
                const int i = s0 + t, xi = s_x[t];
                const T c = (T)(a.k.c1m1 + 1.0), s = (T)(-xi * a.k.s1);  // spin-y A(-gamma x) = [[c, s], [-s, c]]
                const cx<T> MA00 = aux[4 * t], MA01 = aux[4 * t + 1], MA10 = aux[4 * t + 2], MA11 = aux[4 * t + 3];
                T h;
                if (a.k.hs == AFQMC_SOC_HS_SZ) {  // spin-z A(-gamma x) = diag(c + i s, c - i s)
                    const cx<T> uu = cmul(cmk(c, s), MA00), dd = cmul(cmk(c, -s), MA11);
                    h = -(T)a.k.gamma * (uu.i - dd.i);
                } else {
                    const cx<T> dn_up = cadd(cscale(MA00, -s), cscale(MA10, c));
                    const cx<T> up_dn = cadd(cscale(MA01, c), cscale(MA11, s));
                    h = (T)a.k.gamma * (dn_up.r - up_dn.r);
                }
                const T lp = (T)1 / ((T)1 + exp((T)-2 * h));
                lam[i] = (double)lp;
                const int xp = s_rep[t] >= 0 ? (s_rep[t] ? 1 : -1) : (s_uT[t] < lp ? 1 : -1);
                dec[i] = (uint8_t)(xp > 0);
                if (xp != xi) {
                    cx<T> dl[2][2];
                    site_delta<T>(a.k.hs, a.k.c2m1, a.k.s2, xi, dl);
                    for (int p = 0; p < 2; ++p)
                        for (int q = 0; q < 2; ++q) s_dl[m][p][q] = dl[p][q];
                    s_site[m] = i;
                    logq += (T)(xi - xp) * h;
                    ++m;
                }
            }
            s_m = m;
            s_logq = logq;
        }
        __syncthreads();
        const int m = s_m;
        if (m == 0) {
            if (tid == 0) {
                dec[N + a.blk] = 1;
                ratio[2 * (N + a.blk)] = 1.0;
                ratio[2 * (N + a.blk) + 1] = 0.0;
                a.Kdev[z] = 0;
            }
            return;
        }
        m2 = 2 * m;
        for (int e = tid; e < m2 * m2; e += nt) {
            const int q = e / m2, qq = e - q * m2;
            const int t2 = qq >> 1, p2 = qq & 1;
            const int lq = 2 * (s_site[q >> 1] - s0) + (q & 1);
            cx<T> v = cmk((q == qq) ? (T)1 : (T)0, (T)0);
            for (int p = 0; p < 2; ++p) {
                const int lc = 2 * (s_site[t2] - s0) + p;
                const cx<T> g = gl(lq, lc);
                const cx<T> Aq = cmk((lq == lc ? (T)1 : (T)0) - g.r, -g.i);
                cfma(v, Aq, s_dl[t2][p][p2]);
            }
            Mw[e] = v;
        }
        const bool ok = gj_inverse_2x2<T>(Mw, m2, m2, aux, &s_det);
        if (tid == 0) {
            const cx<T> dt = ok ? s_det : cmk((T)0, (T)0);
            const T f = exp(s_logq);
            const T Rr = dt.r * f, Ri = dt.i * f;
            const T absR = sqrt(Rr * Rr + Ri * Ri);
            ratio[2 * (N + a.blk)] = (double)Rr;
            ratio[2 * (N + a.blk) + 1] = (double)Ri;
            if (!isfinite(absR)) set_err(a.err, DEV_NUMERIC);
            const int racc = rep ? (int)rep[N + a.blk] : -1;
            const int acc = racc >= 0 ? (racc != 0) : ((T)u[N + a.blk] < absR);
            dec[N + a.blk] = (uint8_t)acc;
            s_acc = acc && ok && absR > (T)0 && isfinite(absR);
            if (s_acc) {
                for (int t = 0; t < m; ++t) {
                    sites[t] = s_site[t];
                    x[s_site[t]] = (int8_t)(-x[s_site[t]]);
                }
                a.Kdev[z] = m2;
            } else {
                a.Kdev[z] = 0;
            }
        }
        __syncthreads();
        if (!s_acc) return;
    }
    write_W<T>(Mw, m2, m2, s_dl, W, ldw);
    if (tid == 0) a.Kdev[z] = m2;
}

// ---------------------------------------------------------------------------
// the window's update of the full G, out of place:
//   X' = G0[:, F] W  (2N x 2m);   G1 = G0 - X' (E_F^T - G0[F, :])
// ---------------------------------------------------------------------------
constexpr int XW_ROWS = 16;

// X'[r][q] for 16 rows per block; W (2m x 2m) and the rows' F-columns staged in shared memory.
template <typename T>
__global__ void __launch_bounds__(256) soc_xw_kernel(const T* G0, long gstride, long ldz, int N, const int* sites0,
                                                     int kmax, const int* Kdev, const cx<T>* W0, cx<T>* Xp0) {
    extern __shared__ __align__(16) unsigned char xw_smem[];
    const int z = blockIdx.z;
    const int m2 = Kdev[z];
    if (m2 == 0) return;
    const int ldw = 2 * kmax;
    const T* G = G0 + (long)z * gstride;
    const int* sites = sites0 + (long)z * kmax;
    const cx<T>* W = W0 + (long)z * ldw * ldw;
    cx<T>* Xp = Xp0 + (long)z * 2 * N * ldw;
    cx<T>* Ws = (cx<T>*)xw_smem;     // [m2][m2]
    cx<T>* Gs = Ws + m2 * m2;        // [XW_ROWS][m2]
    const int r0 = blockIdx.x * XW_ROWS;
    for (int e = threadIdx.x; e < m2 * m2; e += blockDim.x) Ws[e] = W[(e / m2) * ldw + e % m2];
    for (int e = threadIdx.x; e < XW_ROWS * m2; e += blockDim.x) {
        const int rr = e / m2, q = e - rr * m2, r = r0 + rr;
        const int o = (q & 1) ? N + sites[q >> 1] : sites[q >> 1];
        Gs[e] = (r < 2 * N) ? g_at(G, ldz, r, o) : cmk((T)0, (T)0);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < XW_ROWS * m2; e += blockDim.x) {
        const int rr = e / m2, q = e - rr * m2, r = r0 + rr;
        if (r >= 2 * N) continue;
        cx<T> a0 = cmk((T)0, (T)0), a1 = cmk((T)0, (T)0);
        int p = 0;
        for (; p + 1 < m2; p += 2) {
            cfma(a0, Gs[rr * m2 + p], Ws[p * m2 + q]);
            cfma(a1, Gs[rr * m2 + p + 1], Ws[(p + 1) * m2 + q]);
        }
        if (p < m2) cfma(a0, Gs[rr * m2 + p], Ws[p * m2 + q]);
        Xp[(long)r * ldw + q] = cadd(a0, a1);
    }
}

constexpr int FL_R = 32, FL_C = 64;

// G1 = G0 - X' Y, Y = E_F^T - G0[F, :]; tiles of 32 rows x 64 columns (complex), 8 outputs per
// thread; m2 = 0 copies the tile.
template <typename T>
__global__ void __launch_bounds__(256) soc_flush_kernel(const T* G0, T* G1, long gstride, long ldz, int N,
                                                        const int* sites0, int kmax, const int* Kdev,
                                                        const cx<T>* Xp0) {
    extern __shared__ __align__(16) unsigned char fl_smem[];
    const int z = blockIdx.z;
    const int m2 = Kdev[z];
    const int ldw = 2 * kmax;
    const T* Ga = G0 + (long)z * gstride;
    T* Gb = G1 + (long)z * gstride;
    const int* sites = sites0 + (long)z * kmax;
    const cx<T>* Xp = Xp0 + (long)z * 2 * N * ldw;
    cx<T>* Xs = (cx<T>*)fl_smem;       // [FL_R][m2]
    cx<T>* Ys = Xs + FL_R * m2;        // [m2][FL_C]
    const int r0 = blockIdx.y * FL_R, c0 = blockIdx.x * FL_C;
    const int N2 = 2 * N;
    const long ld2 = 2 * ldz;
    for (int e = threadIdx.x; e < FL_R * m2; e += blockDim.x) {
        const int rr = e / m2, q = e - rr * m2, r = r0 + rr;
        Xs[e] = (r < N2) ? Xp[(long)r * ldw + q] : cmk((T)0, (T)0);
    }
    for (int e = threadIdx.x; e < m2 * FL_C; e += blockDim.x) {
        const int q = e / FL_C, cc = e - q * FL_C, c = c0 + cc;
        const int o = (q & 1) ? N + sites[q >> 1] : sites[q >> 1];
        cx<T> y = cmk((T)0, (T)0);
        if (c < N2) {
            const cx<T> g = g_at(Ga, ldz, o, c);
            y = cmk((c == o ? (T)1 : (T)0) - g.r, -g.i);
        }
        Ys[e] = y;
    }
    __syncthreads();
    const int tc = threadIdx.x % FL_C, tr = threadIdx.x / FL_C;  // 4 row groups of 8 rows
    const int c = c0 + tc;
    if (c >= N2) return;
    cx<T> acc[FL_R / 4];
#pragma unroll
    for (int i = 0; i < FL_R / 4; ++i) acc[i] = cmk((T)0, (T)0);
    for (int q = 0; q < m2; ++q) {
        const cx<T> y = Ys[q * FL_C + tc];
#pragma unroll
        for (int i = 0; i < FL_R / 4; ++i) cfma(acc[i], Xs[(tr + 4 * i) * m2 + q], y);
    }
#pragma unroll
    for (int i = 0; i < FL_R / 4; ++i) {
        const int r = r0 + tr + 4 * i;
        if (r >= N2) continue;
        const long o = (long)r * ld2 + c;
        Gb[o] = Ga[o] - acc[i].r;
        Gb[o + ldz] = Ga[o + ldz] - acc[i].i;
    }
}

// ---------------------------------------------------------------------------
// FP64 propagation of realified factors through exp(-dtau H0) in momentum space
// ---------------------------------------------------------------------------
struct SocPropArgs {
    double* F0;
    long wstride;             // factor of walker j at F0 + j wstride: 4N x nv row-major
    int nv, L, N;
    int P, Q;                 // L = P Q: the two factors of the lattice DFT (Q = 1: a plain DFT)
    const double* tab;        // complex tables: F_P (P x P), F_Q (Q x Q), twiddles (Q x P), see dft_stage
    const double* lam;        // N x 2 x 2 complex: exp(-dtau h_k) / N, k = kx + L ky
    const int8_t* x;
    long xstride;             // fields M x N of walker j at x + j xstride
    int l_first, l_step, nsl;
    int left;                 // 0: v <- D_l E v (right factor); 1: v <- E D_l^+ v (the left factor carried
                              // as U_L^+: (U_L B_l)^+ = E^+ D_l^+ U_L^+, E Hermitian)
    double cg, sg;
    int hs;                   // AFQMC_SOC_HS_SY (D_l a real rotation, D_l^+ = D_l^T) or AFQMC_SOC_HS_SZ
                              // (D_l phases, D_l^+ their conjugates)
};

constexpr int PROP_VPC_MAX = 4;

// One stage of the length-L DFT w = exp(-+2 pi i / L) along one lattice axis of every vector
// (axis 0: x, element stride 1; axis 1: y, stride L), L = P Q, by the two-factor Cooley-Tukey
// split (input index x = Q x1 + x2, output index k = k1 + P k2):
//   stage 0:  Y[x2 + Q k1] = w^{x2 k1} sum_{x1 < P} w_P^{x1 k1} v[Q x1 + x2]
//   stage 1:  X[k1 + P k2] = sum_{x2 < Q} w_Q^{x2 k2} Y[x2 + Q k1]
// (P + Q + 1 complex multiply-adds per output instead of L).  inverse conjugates every table.
// With Q = 1 stage 0 is the plain DFT and stage 1 is skipped.
__device__ __forceinline__ void dft_stage(const cx<double>* in, cx<double>* out, const cx<double>* tab, int L, int P,
                                          int Q, int N, int vpc, int axis, int inverse, int stage) {
    const cx<double>* FP = tab;
    const cx<double>* FQ = tab + P * P;
    const cx<double>* TW = FQ + Q * Q;
    const double cj = inverse ? -1.0 : 1.0;
    const int n2 = 2 * N;
    for (int e = threadIdx.x; e < vpc * n2; e += blockDim.x) {
        const int v = e / n2, a = e - v * n2;
        const int s = a / N, i = a - s * N;
        const int xx = i % L, yy = i / L;
        const int j = axis ? yy : xx;  // position along the transformed axis
        const int stride = axis ? L : 1;
        const cx<double>* src = in + v * n2 + s * N + (axis ? xx : yy * L);
        cx<double> acc0 = cmk(0.0, 0.0), acc1 = cmk(0.0, 0.0);
        if (stage == 0) {
            const int x2 = j % Q, k1 = j / Q;  // output slot x2 + Q k1
            int x1 = 0;
            for (; x1 + 1 < P; x1 += 2) {
                cx<double> f0 = FP[k1 * P + x1], f1 = FP[k1 * P + x1 + 1];
                f0.i *= cj;
                f1.i *= cj;
                cfma(acc0, f0, src[(Q * x1 + x2) * stride]);
                cfma(acc1, f1, src[(Q * (x1 + 1) + x2) * stride]);
            }
            if (x1 < P) {
                cx<double> f0 = FP[k1 * P + x1];
                f0.i *= cj;
                cfma(acc0, f0, src[(Q * x1 + x2) * stride]);
            }
            acc0 = cadd(acc0, acc1);
            if (Q > 1) {
                cx<double> t = TW[x2 * P + k1];
                t.i *= cj;
                acc0 = cmul(acc0, t);
            }
        } else {
            const int k1 = j % P, k2 = j / P;  // output k1 + P k2 reads Y[x2 + Q k1]
            for (int x2 = 0; x2 < Q; ++x2) {
                cx<double> f = FQ[k2 * Q + x2];
                f.i *= cj;
                cfma((x2 & 1) ? acc1 : acc0, f, src[(x2 + Q * k1) * stride]);
            }
            acc0 = cadd(acc0, acc1);
        }
        out[e] = acc0;
    }
}

__global__ void __launch_bounds__(256) soc_prop_kernel(SocPropArgs a, int vpc) {
    extern __shared__ __align__(16) unsigned char prop_smem[];
    const int N = a.N, L = a.L, n2 = 2 * N, P = a.P, Q = a.Q;
    cx<double>* b0 = (cx<double>*)prop_smem;
    cx<double>* b1 = b0 + vpc * n2;
    cx<double>* tab = b1 + vpc * n2;
    const int ntab = P * P + Q * Q + Q * P;
    const int z = blockIdx.y;
    double* U = a.F0 + (long)z * a.wstride;
    const int8_t* xw = a.x + (long)z * a.xstride;
    const int c0 = blockIdx.x * vpc;
    const int nv = a.nv;
    for (int e = threadIdx.x; e < ntab; e += blockDim.x) tab[e] = cmk(a.tab[2 * e], a.tab[2 * e + 1]);
    for (int e = threadIdx.x; e < vpc * n2; e += blockDim.x) {
        const int r = e / vpc, v = e - r * vpc;  // v fastest: consecutive columns
        const int c = c0 + v;
        b0[v * n2 + r] = (c < nv) ? cmk(U[(long)r * nv + c], U[(long)(n2 + r) * nv + c]) : cmk(0.0, 0.0);
    }
    __syncthreads();
    const cx<double>* lamk = (const cx<double>*)a.lam;
    // one DFT along an axis: the data moves b0 -> b1 (-> b0 again for the two-factor split)
    auto dft = [&](int axis, int inverse) {
        dft_stage(b0, b1, tab, L, P, Q, N, vpc, axis, inverse, 0);
        __syncthreads();
        if (Q > 1) {
            dft_stage(b1, b0, tab, L, P, Q, N, vpc, axis, inverse, 1);
            __syncthreads();
        } else {
            cx<double>* t = b0;
            b0 = b1;
            b1 = t;
        }
    };
    for (int q = 0; q < a.nsl; ++q) {
        const int ell = a.l_first + q * a.l_step;
        const int8_t* xl = xw + (long)(ell - 1) * N;
        if (a.left) {  // v <- D^+ v: spin-y the rotation A(-gamma x), spin-z the conjugate phases
            for (int e = threadIdx.x; e < vpc * N; e += blockDim.x) {
                const int v = e / N, i = e - v * N;
                const cx<double> p0 = b0[v * n2 + i], p1 = b0[v * n2 + N + i];
                if (a.hs == AFQMC_SOC_HS_SZ) {
                    const double s = xl[i] * a.sg;
                    b0[v * n2 + i] = cmul(p0, cmk(a.cg, -s));
                    b0[v * n2 + N + i] = cmul(p1, cmk(a.cg, s));
                } else {
                    const double s = -xl[i] * a.sg;
                    b0[v * n2 + i] = cadd(cscale(p0, a.cg), cscale(p1, s));
                    b0[v * n2 + N + i] = csub(cscale(p1, a.cg), cscale(p0, s));
                }
            }
            __syncthreads();
        }
        dft(0, 0);
        dft(1, 0);
        for (int e = threadIdx.x; e < vpc * N; e += blockDim.x) {
            const int v = e / N, k = e - v * N;
            const cx<double>* l4 = lamk + 4 * k;
            const cx<double> u0 = b0[v * n2 + k], u1 = b0[v * n2 + N + k];
            cx<double> w0 = cmul(l4[0], u0), w1 = cmul(l4[2], u0);
            cfma(w0, l4[1], u1);
            cfma(w1, l4[3], u1);
            b1[v * n2 + k] = w0;
            b1[v * n2 + N + k] = w1;
        }
        __syncthreads();
        {
            cx<double>* t = b0;
            b0 = b1;
            b1 = t;
        }
        dft(1, 1);
        dft(0, 1);
        if (!a.left) {  // v <- D v: A(gamma x) on each pair
            for (int e = threadIdx.x; e < vpc * N; e += blockDim.x) {
                const int v = e / N, i = e - v * N;
                const double s = xl[i] * a.sg;
                const cx<double> p0 = b0[v * n2 + i], p1 = b0[v * n2 + N + i];
                if (a.hs == AFQMC_SOC_HS_SZ) {
                    b0[v * n2 + i] = cmul(p0, cmk(a.cg, s));
                    b0[v * n2 + N + i] = cmul(p1, cmk(a.cg, -s));
                } else {
                    b0[v * n2 + i] = cadd(cscale(p0, a.cg), cscale(p1, s));
                    b0[v * n2 + N + i] = csub(cscale(p1, a.cg), cscale(p0, s));
                }
            }
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < vpc * n2; e += blockDim.x) {
        const int r = e / vpc, v = e - r * vpc;
        const int c = c0 + v;
        if (c < nv) {
            const cx<double> w = b0[v * n2 + r];
            U[(long)r * nv + c] = w.r;
            U[(long)(n2 + r) * nv + c] = w.i;
        }
    }
}

// B (cols x rows per walker) = A^T
__global__ void soc_transpose_kernel(const double* A0, int rows, int cols, long sa, double* B0, long sb) {
    __shared__ double tile[32][33];
    const double* A = A0 + (long)blockIdx.z * sa;
    double* B = B0 + (long)blockIdx.z * sb;
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int r = by + k, c = bx + threadIdx.x;
        tile[k][threadIdx.x] = (r < rows && c < cols) ? A[(long)r * cols + c] : 0.0;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int c = bx + k, r = by + threadIdx.x;
        if (c < cols && r < rows) B[(long)c * rows + r] = tile[threadIdx.x][k];
    }
}

// Bulk G (row-split, T) from P = U_R Z (4N x 2N, FP64): Re G = 1 - P[0:2N], Im G = -P[2N:4N];
// acc2[j] += (||G_old - G_new||^2, ||G_new||^2) when drift != 0.
template <typename T>
__global__ void soc_store_G_kernel(const double* P0, long pstride, int N2, T* G0, long ldz, long gstride, double* acc2,
                                   int drift) {
    const int z = blockIdx.y;
    const double* P = P0 + (long)z * pstride;
    T* G = G0 + (long)z * gstride;
    double d2 = 0.0, n2 = 0.0;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)N2 * N2; e += (long)gridDim.x * blockDim.x) {
        const int r = (int)(e / N2), c = (int)(e - (long)r * N2);
        const double gr = (r == c ? 1.0 : 0.0) - P[(long)r * N2 + c];
        const double gi = -P[(long)(N2 + r) * N2 + c];
        T* pr = G + (long)r * 2 * ldz + c;
        if (drift) {
            const double er = (double)pr[0] - gr, ei = (double)pr[ldz] - gi;
            d2 += er * er + ei * ei;
            n2 += gr * gr + gi * gi;
        }
        pr[0] = (T)gr;
        pr[ldz] = (T)gi;
    }
    if (!drift) return;
    for (int o = 16; o > 0; o >>= 1) {
        d2 += __shfl_xor_sync(0xffffffffu, d2, o);
        n2 += __shfl_xor_sync(0xffffffffu, n2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(acc2 + 2 * z, d2);
        atomicAdd(acc2 + 2 * z + 1, n2);
    }
}

// Energy with the spin-coupled Wick contraction; H0 is applied bond by bond (hopping -t in each
// spin block; spin-flip hopping (dn r, up r+d) = -i lam (d = +y), +i lam (-y), -lam (+x), +lam (-x)
// and its Hermitian conjugate).  out[j] = (Re E, Im E).
template <typename T>
__global__ void soc_energy_kernel(const T* G0, long ldz, long gstride, int L, double t, double lam, double U,
                                  double* out) {
    const int z = blockIdx.x;
    const T* G = G0 + (long)z * gstride;
    const int N = L * L;
    auto A = [&](int r, int c) {
        const cx<T> g = g_at(G, ldz, r, c);
        return cmk((r == c ? 1.0 : 0.0) - (double)g.r, -(double)g.i);
    };
    cx<double> acc = cmk(0.0, 0.0);
    for (int r = threadIdx.x; r < N; r += blockDim.x) {
        const int x = r % L, y = r / L;
        const int dx[4] = {0, 0, 1, -1}, dy[4] = {1, -1, 0, 0};
        const cx<double> amp[4] = {cmk(0.0, -lam), cmk(0.0, lam), cmk(-lam, 0.0), cmk(lam, 0.0)};
        for (int d = 0; d < 4; ++d) {
            const int rp = (x + dx[d] + L) % L + L * ((y + dy[d] + L) % L);
            // kinetic: H0[(s, r)][(s, rp)] = -t  ->  -t A[(s, rp)][(s, r)]
            acc = cadd(acc, cscale(A(rp, r), -t));
            acc = cadd(acc, cscale(A(N + rp, N + r), -t));
            // H0[(dn, r)][(up, rp)] = amp -> amp A[(up, rp)][(dn, r)]; its conjugate entry
            cfma(acc, amp[d], A(rp, N + r));
            cfma(acc, cmk(amp[d].r, -amp[d].i), A(N + r, rp));
        }
        const cx<double> Auu = A(r, r), Add = A(N + r, N + r), Adu = A(N + r, r), Aud = A(r, N + r);
        cx<double> v = csub(cmul(Auu, Add), cmul(Adu, Aud));
        v = csub(v, cscale(cadd(Auu, Add), 0.5));
        acc = cadd(acc, cscale(v, U));
    }
    __shared__ double sr[32], si[32];
    for (int o = 16; o > 0; o >>= 1) {
        acc.r += __shfl_xor_sync(0xffffffffu, acc.r, o);
        acc.i += __shfl_xor_sync(0xffffffffu, acc.i, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sr[wid] = acc.r;
        si[wid] = acc.i;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += sr[w];
            b += si[w];
        }
        out[2 * z] = a;
        out[2 * z + 1] = b;
    }
}

// ---------------------------------------------------------------------------
// pairing observables (Sec. IV), FP64 from the bulk G of one walker
// ---------------------------------------------------------------------------
// A = 1 - G in FP64, row-split like G (2N rows of 2 ldz; grid: (columns, 2N rows)).
template <typename T>
__global__ void soc_one_minus_kernel(const T* G, long ldz, double* A) {
    const long ld2 = 2 * ldz;
    const int r = blockIdx.y;
    for (long c = blockIdx.x * blockDim.x + threadIdx.x; c < ld2; c += (long)gridDim.x * blockDim.x)
        A[(long)r * ld2 + c] = (c == r ? 1.0 : 0.0) - (double)G[(long)r * ld2 + c];
}

// The real-space estimators by Wick's theorem (A_ab = <c_b^+ c_a>, G = 1 - A; u = i, d = N + i):
//   D terms     <n_iu n_id>  = A_uu A_dd - A_du A_ud;
//   pair terms  <D+_i D_j>   = A_{ju,iu} A_{jd,id} - A_{jd,iu} A_{ju,id},
//               <D_i D+_j>   = G_{iu,ju} G_{id,jd} - G_{id,ju} G_{iu,jd};
// out[0..1] += sum_i <n_iu n_id>, out[2..3] += sum_ij (<D+_i D_j> + <D_i D+_j>) (complex; FP64 atomics).
__global__ void __launch_bounds__(256) soc_pair_scalars_kernel(const double* A, long ldz, int N, double* out) {
    const long ld2 = 2 * ldz;
    auto a = [&](int r, int c) { return cmk(A[(long)r * ld2 + c], A[(long)r * ld2 + ldz + c]); };
    auto g = [&](int r, int c) {
        const cx<double> v = a(r, c);
        return cmk((r == c ? 1.0 : 0.0) - v.r, -v.i);
    };
    cx<double> d = cmk(0.0, 0.0), pp = cmk(0.0, 0.0);
    const long NN = (long)N * N;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < NN; e += (long)gridDim.x * blockDim.x) {
        const int i = (int)(e / N), j = (int)(e - (long)i * N);
        cx<double> t = cmul(a(j, i), a(N + j, N + i));
        t = csub(t, cmul(a(N + j, i), a(j, N + i)));
        cfma(t, g(i, j), g(N + i, N + j));
        t = csub(t, cmul(g(N + i, j), g(i, N + j)));
        pp = cadd(pp, t);
        if (i == j) d = cadd(d, csub(cmul(a(i, i), a(N + i, N + i)), cmul(a(N + i, i), a(i, N + i))));
    }
    __shared__ double red[4][8];
    double v[4] = {d.r, d.i, pp.r, pp.i};
    for (int q = 0; q < 4; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        for (int q = 0; q < 4; ++q) red[q][warp] = v[q];
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[threadIdx.x][w];
        atomicAdd(out + threadIdx.x, s);
    }
}

// From At = F2 A F2^+ (row-split, At_{(p s),(q t)} = <c+_{q t} c_{p s}>): nk[k] = At_{ku,ku},
// nk[N + k] = At_{kd,kd} (complex), and Mk[k][k'] = At_{k'u,ku} At_{-k'd,-kd} - At_{-k'd,ku} At_{k'u,-kd}
// (<D+_k D_k'> of one walker, D+_k = c+_{k u} c+_{-k d}; -k = (-kx, -ky) mod L).
__global__ void __launch_bounds__(256) soc_pair_k_kernel(const double* At, long ldz, int L, double* Mk, double* nk) {
    const long ld2 = 2 * ldz;
    const int N = L * L;
    auto at = [&](int r, int c) { return cmk(At[(long)r * ld2 + c], At[(long)r * ld2 + ldz + c]); };
    auto neg = [&](int k) { return (L - k % L) % L + L * ((L - k / L) % L); };
    const long NN = (long)N * N;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < NN; e += (long)gridDim.x * blockDim.x) {
        const int k = (int)(e / N), k2 = (int)(e - (long)k * N);
        const int mk = neg(k), mk2 = neg(k2);
        cx<double> t = cmul(at(k2, k), at(N + mk2, N + mk));
        t = csub(t, cmul(at(N + mk2, k), at(k2, N + mk)));
        Mk[2 * e] = t.r;
        Mk[2 * e + 1] = t.i;
        if (k2 == 0) {
            const cx<double> u = at(k, k), dd = at(N + k, N + k);
            nk[2 * k] = u.r;
            nk[2 * k + 1] = u.i;
            nk[2 * (N + k)] = dd.r;
            nk[2 * (N + k) + 1] = dd.i;
        }
    }
}

__global__ void soc_fields_kernel(uint64_t seed, long count, int8_t* x) {
    const long j = blockIdx.x * (long)blockDim.x + threadIdx.x;
    const int w = blockIdx.y;
    if (j < count) x[(long)w * count + j] = philox_uniform(seed, (uint64_t)w, 0x5F1E1DULL, (uint64_t)j) < 0.5 ? 1 : -1;
}

__global__ void soc_iota_kernel(int* g, int n) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) g[j] = j;
}

}  // namespace
}  // namespace afq

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
using namespace afq;

struct afqmc_soc_ctx {
    afqmc_soc_params p;
    int N = 0, N2 = 0, ne = 0, nv = 0, nwk = 0, kmax = 0, nst = 0;
    long ldz = 0;
    SocConsts k{};
    bool f64 = true, use_tc = false;
    int sticky = 0;
    int pos = 0, last_dir = -1;
    bool need_recompute = false, inited = false;
    cudaStream_t last = nullptr;
    std::vector<void*> allocs;
    // constants
    void *Ers = nullptr, *Einvrs = nullptr;   // [Re E | Im E] rows, bulk precision
    void *Ech = nullptr, *Einvch = nullptr;   // realified right operands (transposed for tensor cores)
    double *dft = nullptr, *lamk = nullptr;   // momentum-space propagation (FP64): DFT tables, e^{-dtau h_k}/N
    int dP = 1, dQ = 1;                       // the lattice DFT as L = dP dQ
    // walkers
    void* G = nullptr;
    void* S = nullptr;
    int8_t* x = nullptr;
    double* u = nullptr;
    uint8_t *rep = nullptr, *dec = nullptr;
    double *ratio = nullptr, *lamp = nullptr;
    int* gid = nullptr;
    unsigned long long* visit = nullptr;
    void* G2 = nullptr;  // the other buffer of the out-of-place flush
    // per-window sets, double-buffered by window parity (window w + 1 reads window w's set while
    // window w's flush runs on sf)
    void *Xp[2] = {nullptr, nullptr}, *W[2] = {nullptr, nullptr};
    int *Kdev[2] = {nullptr, nullptr}, *sites[2] = {nullptr, nullptr};
    int* err = nullptr;
    void* Gw0 = nullptr;  // per walker: the window's block of the current G
    cudaStream_t sf = nullptr;
    cudaEvent_t ev_win[2] = {nullptr, nullptr}, ev_fl[2] = {nullptr, nullptr};
    double *URs = nullptr, *ULs = nullptr, *Ucur = nullptr, *Lrow = nullptr, *O = nullptr, *Z = nullptr,
           *Pb = nullptr, *acc2 = nullptr, *en = nullptr;
    int* perm = nullptr;
    int8_t* flag = nullptr;
    // the recompute's two FP64 products on the tensor cores (digit splitting, ozaki.cu)
    bool oz_O = false, oz_G = false;
    void* ozw = nullptr;
    double* ozs = nullptr;
    // pairing observables (allocated at the first afqmc_soc_measure_pairing): [Re F2 | Im F2] rows,
    // the realified F2^+ (2 ldz x 2 ldz), FP64 scratch A (2N x 2 ldz), S~ (2 ldz x 2 ldz),
    // At (2N x 2 ldz), Mk per walker (N x N complex each) and the per-walker outputs
    double *Frs = nullptr, *Fh = nullptr, *pA = nullptr, *pS = nullptr, *pAt = nullptr, *pMk = nullptr,
           *pOut = nullptr;
    // profiling
    struct Ev {
        int ph;
        cudaEvent_t a, b;
    };
    bool prof_on = false;
    std::vector<Ev> pending;
    std::vector<cudaEvent_t> pool;
    double ms[AFQMC_NPHASE] = {};
    int64_t intervals[AFQMC_NPHASE] = {};
    int64_t launches[AFQMC_NPHASE] = {};

    long gstride() const { return (long)N2 * 2 * ldz; }
    long fsz() const { return (long)2 * N2 * nv; }  // realified factor: 4N x 2 n_e
    double* stackR(int j) const { return URs + (long)j * fsz(); }
    double* stackL(int j) const { return ULs + (long)j * fsz(); }
    long st_w() const { return (long)nst * fsz(); }
};

namespace {

cudaEvent_t soc_event(afqmc_soc_ctx* c) {
    if (!c->pool.empty()) {
        cudaEvent_t e = c->pool.back();
        c->pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

struct SocPhase {
    afqmc_soc_ctx* c;
    int ph;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    long long l0;
    SocPhase(afqmc_soc_ctx* ctx, int phase, cudaStream_t s) : c(ctx), ph(phase), st(s), l0(afqmc_launch_count()) {
        if (c->prof_on) {
            a = soc_event(c);
            cudaEventRecord(a, st);
        }
    }
    ~SocPhase() {
        if (!c->prof_on || !a) return;
        cudaEvent_t b = soc_event(c);
        cudaEventRecord(b, st);
        c->pending.push_back({ph, a, b});
        c->launches[ph] += afqmc_launch_count() - l0;
    }
};

#define SCK(x)                                        \
    do {                                              \
        cudaError_t e_ = (x);                         \
        if (e_ != cudaSuccess) return soc_fail(ctx, e_); \
    } while (0)

int soc_fail(afqmc_soc_ctx* ctx, cudaError_t e) {
    if (e == cudaErrorMemoryAllocation) ctx->sticky = AFQMC_ERR_OOM;
    else ctx->sticky = AFQMC_ERR_CUDA;
    cudaGetLastError();
    return ctx->sticky;
}

template <typename P>
cudaError_t soc_alloc(afqmc_soc_ctx* ctx, P** out, size_t bytes, cudaStream_t st) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes ? bytes : 16);
    if (e != cudaSuccess) return e;
    ctx->allocs.push_back(p);
    *out = (P*)p;
    return cudaMemsetAsync(p, 0, bytes ? bytes : 16, st);
}

int read_err(afqmc_soc_ctx* ctx) {
    int h = 0;
    cudaError_t e = cudaMemcpy(&h, ctx->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return soc_fail(ctx, e);
    if (h == DEV_TIMEOUT) ctx->sticky = AFQMC_ERR_TIMEOUT;
    else if (h == DEV_NUMERIC) ctx->sticky = AFQMC_ERR_NUMERIC;
    else if (h != 0) ctx->sticky = AFQMC_ERR_CUDA;
    return ctx->sticky;
}

// exp(-tau h_k) / N per momentum k = kx + L ky (row-major 2 x 2 complex, interleaved doubles):
// h_k = eps + [[0, conj Lk], [Lk, 0]] and the off-diagonal part squares to |Lk|^2, so
// exp(-tau h_k) = e^{-tau eps} (cosh(tau |Lk|) - sinh(tau |Lk|) / |Lk| [[0, conj Lk], [Lk, 0]]).
void host_lamk(int L, double t, double lam, double tau, std::vector<double>& out) {
    const int N = L * L;
    out.assign((size_t)N * 8, 0.0);
    for (int ky = 0; ky < L; ++ky)
        for (int kx = 0; kx < L; ++kx) {
            const double ax = 2.0 * M_PI * kx / L, ay = 2.0 * M_PI * ky / L;
            const double eps = -2.0 * t * (cos(ax) + cos(ay));
            const double lr = 2.0 * lam * sin(ay), li = -2.0 * lam * sin(ax);  // Lk
            const double mag = sqrt(lr * lr + li * li);
            const double ch = cosh(tau * mag), sh = mag > 0.0 ? sinh(tau * mag) / mag : tau;
            const double f = exp(-tau * eps) / N;
            double* o = &out[(size_t)(kx + L * ky) * 8];
            o[0] = f * ch;                       // [up][up]
            o[2] = -f * sh * lr;                 // [up][dn] = conj Lk coefficient
            o[3] = f * sh * li;
            o[4] = -f * sh * lr;                 // [dn][up] = Lk coefficient
            o[5] = -f * sh * li;
            o[6] = f * ch;                       // [dn][dn]
        }
}

// Dense exp(-tau H0) (2N x 2N complex, interleaved): entries depend on the displacement only.
void host_expH(int L, double t, double lam, double tau, std::vector<double>& E) {
    const int N = L * L, N2 = 2 * N;
    std::vector<double> lk;
    host_lamk(L, t, lam, tau, lk);
    std::vector<double> tab((size_t)N * 8, 0.0);  // [dy][dx][s][s'] complex
    std::vector<double> cs(L), sn(L);
    for (int q = 0; q < L; ++q) {
        cs[q] = cos(2.0 * M_PI * q / L);
        sn[q] = sin(2.0 * M_PI * q / L);
    }
    for (int dy = 0; dy < L; ++dy)
        for (int dx = 0; dx < L; ++dx) {
            double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int ky = 0; ky < L; ++ky)
                for (int kx = 0; kx < L; ++kx) {
                    const int ph = (kx * dx + ky * dy) % L;
                    const double er = cs[ph], ei = sn[ph];
                    const double* o = &lk[(size_t)(kx + L * ky) * 8];
                    for (int q = 0; q < 4; ++q) {
                        acc[2 * q] += er * o[2 * q] - ei * o[2 * q + 1];
                        acc[2 * q + 1] += er * o[2 * q + 1] + ei * o[2 * q];
                    }
                }
            memcpy(&tab[(size_t)(dx + L * dy) * 8], acc, sizeof(acc));
        }
    E.assign((size_t)N2 * N2 * 2, 0.0);
    for (int s = 0; s < 2; ++s)
        for (int i = 0; i < N; ++i)
            for (int sp = 0; sp < 2; ++sp)
                for (int j = 0; j < N; ++j) {
                    const int dx = ((i % L) - (j % L) + L) % L, dy = ((i / L) - (j / L) + L) % L;
                    const double* v = &tab[(size_t)(dx + L * dy) * 8 + 2 * (2 * s + sp)];
                    const size_t o = ((size_t)(s * N + i) * N2 + (sp * N + j)) * 2;
                    E[o] = v[0];
                    E[o + 1] = v[1];
                }
}

template <typename T>
cudaError_t upload_constants(afqmc_soc_ctx* ctx, cudaStream_t st) {
    const int N2 = ctx->N2;
    const long ldz = ctx->ldz, ld2 = 2 * ldz;
    for (int inv = 0; inv < 2; ++inv) {
        std::vector<double> E;
        host_expH(ctx->p.L, ctx->p.t, ctx->p.lam, inv ? -ctx->p.dtau : ctx->p.dtau, E);
        std::vector<T> rs((size_t)N2 * ld2, (T)0), ch((size_t)ld2 * ld2, (T)0);
        for (int r = 0; r < N2; ++r)
            for (int c = 0; c < N2; ++c) {
                const double er = E[((size_t)r * N2 + c) * 2], ei = E[((size_t)r * N2 + c) * 2 + 1];
                rs[(size_t)r * ld2 + c] = (T)er;
                rs[(size_t)r * ld2 + ldz + c] = (T)ei;
                // C~ = [[Re, Im], [-Im, Re]]; the tensor-core path stores its transpose
                const size_t o00 = (size_t)r * ld2 + c, o01 = (size_t)r * ld2 + ldz + c;
                const size_t o10 = (size_t)(ldz + r) * ld2 + c, o11 = (size_t)(ldz + r) * ld2 + ldz + c;
                if (!ctx->use_tc) {
                    ch[o00] = (T)er;
                    ch[o01] = (T)ei;
                    ch[o10] = (T)(-ei);
                    ch[o11] = (T)er;
                } else {
                    ch[(size_t)c * ld2 + r] = (T)er;
                    ch[(size_t)(ldz + c) * ld2 + r] = (T)ei;
                    ch[(size_t)c * ld2 + ldz + r] = (T)(-ei);
                    ch[(size_t)(ldz + c) * ld2 + ldz + r] = (T)er;
                    (void)o00; (void)o01; (void)o10; (void)o11;
                }
            }
        void* drs = inv ? ctx->Einvrs : ctx->Ers;
        void* dch = inv ? ctx->Einvch : ctx->Ech;
        cudaError_t e = cudaMemcpyAsync(drs, rs.data(), rs.size() * sizeof(T), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(dch, ch.data(), ch.size() * sizeof(T), cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return e;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    }
    const int L = ctx->p.L, P = ctx->dP, Q = ctx->dQ;
    // tables of the two-factor DFT: F_P (P x P), F_Q (Q x Q), twiddles w^{x2 k1} (Q x P)
    std::vector<double> F, lk;
    auto root = [&](int num, int den) {
        const double ph = -2.0 * M_PI * (double)(num % den) / den;
        F.push_back(cos(ph));
        F.push_back(sin(ph));
    };
    for (int k = 0; k < P; ++k)
        for (int q = 0; q < P; ++q) root(k * q, P);
    for (int k = 0; k < Q; ++k)
        for (int q = 0; q < Q; ++q) root(k * q, Q);
    for (int x2 = 0; x2 < Q; ++x2)
        for (int k1 = 0; k1 < P; ++k1) root(x2 * k1, L);
    host_lamk(L, ctx->p.t, ctx->p.lam, ctx->p.dtau, lk);
    cudaError_t e = cudaMemcpyAsync(ctx->dft, F.data(), F.size() * 8, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(ctx->lamk, lk.data(), lk.size() * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}

// ---- wrap ----
template <typename T>
cudaError_t soc_wrap(afqmc_soc_ctx* ctx, cudaStream_t st, const int8_t* xl, int dir) {
    SocPhase ps(ctx, AFQMC_PHASE_WRAP, st);
    const int N = ctx->N, N2 = ctx->N2, nwk = ctx->nwk;
    const long ldz = ctx->ldz, ld2 = 2 * ldz, gs = ctx->gstride(), ss = ld2 * ld2;
    const long xs = (long)ctx->p.M * N;
    const T cg = (T)(ctx->k.c1m1 + 1.0), sg = (T)ctx->k.s1;
    T* G = (T*)ctx->G;
    T* S = (T*)ctx->S;
    const dim3 rgrid((N + 31) / 32, (N + 7) / 8, nwk), rblk(32, 8);
    cudaError_t e;
    if (dir < 0) {  // G <- D^{-1} G D first
        count_launch();
        soc_rot_kernel<T><<<rgrid, rblk, 0, st>>>(G, ldz, N, gs, xl, xs, cg, sg, -1, +1, ctx->k.hs);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const T* Cright = (const T*)(dir > 0 ? ctx->Einvch : ctx->Ech);  // S = G E^{-1} (fwd) / G E (bwd)
    const T* Aleft = (const T*)(dir > 0 ? ctx->Ers : ctx->Einvrs);   // G = E S (fwd) / E^{-1} S (bwd)
    if (ctx->use_tc) {
        TcGemmArgs t1;
        t1.M = N2; t1.N = (int)ld2; t1.K = (int)ld2; t1.batch = nwk;
        t1.A = (const float*)G; t1.lda = ld2; t1.sA = gs;
        t1.Bt = (const float*)Cright; t1.ldb = ld2; t1.sB = 0;
        t1.C = (float*)S; t1.ldc = ld2; t1.sC = ss; t1.c_trans = 1;
        t1.split3 = ctx->p.gemm != AFQMC_GEMM_TF32;
        t1.err = ctx->err;
        {
            SocPhase pg(ctx, AFQMC_PHASE_WRAP_GEMM, st);
            if ((e = tc_gemm(st, t1)) != cudaSuccess) return e;
        }
        count_launch();
        soc_realify_kernel<T><<<dim3((N2 + 255) / 256, (unsigned)ld2, nwk), 256, 0, st>>>(S, ldz, N2, ss, 0);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        TcGemmArgs t2;
        t2.M = N2; t2.N = (int)ld2; t2.K = (int)ld2; t2.batch = nwk;
        t2.A = (const float*)Aleft; t2.lda = ld2; t2.sA = 0;
        t2.Bt = (const float*)S; t2.ldb = ld2; t2.sB = ss;
        t2.C = (float*)G; t2.ldc = ld2; t2.sC = gs;
        t2.split3 = t1.split3;
        t2.err = ctx->err;
        SocPhase pg(ctx, AFQMC_PHASE_WRAP_GEMM, st);
        if ((e = tc_gemm(st, t2)) != cudaSuccess) return e;
    } else {
        GemmArgs<T> g1;
        g1.M = N2; g1.N = (int)ld2; g1.K = (int)ld2; g1.batch = nwk;
        g1.A = G; g1.lda = ld2; g1.sA = gs;
        g1.B = Cright; g1.ldb = ld2; g1.sB = 0;
        g1.C = S; g1.ldc = ld2; g1.sC = ss;
        {
            SocPhase pg(ctx, AFQMC_PHASE_WRAP_GEMM, st);
            if ((e = gemm<T>(st, g1)) != cudaSuccess) return e;
        }
        count_launch();
        soc_realify_kernel<T><<<dim3((unsigned)((ld2 + 255) / 256), N2, nwk), 256, 0, st>>>(S, ldz, N2, ss, 1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        GemmArgs<T> g2;
        g2.M = N2; g2.N = (int)ld2; g2.K = (int)ld2; g2.batch = nwk;
        g2.A = Aleft; g2.lda = ld2; g2.sA = 0;
        g2.B = S; g2.ldb = ld2; g2.sB = ss;
        g2.C = G; g2.ldc = ld2; g2.sC = gs;
        SocPhase pg(ctx, AFQMC_PHASE_WRAP_GEMM, st);
        if ((e = gemm<T>(st, g2)) != cudaSuccess) return e;
    }
    if (dir > 0) {  // G <- D G D^{-1}
        count_launch();
        soc_rot_kernel<T><<<rgrid, rblk, 0, st>>>(G, ldz, N, gs, xl, xs, cg, sg, +1, -1, ctx->k.hs);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename T>
size_t window_smem(int kmax) {
    return (size_t)(4 * kmax * kmax + 8 * kmax + 4 * SOC_PIPE_N * SOC_PIPE_N) * sizeof(cx<T>);
}

// ---- one window: chain, then X' = G[:, F] W and the out-of-place flush ----
// Serial (pipe = false): everything on st; G reads the current G and the flush swaps the buffers.
// Pipelined: the window kernel (on st) reads Gin, the G before the previous window's update, and
// applies that update to its block itself; X' and the flush of this window run on sf from Gcur
// (the G this window decided on) into Gnext, after the window kernel and after the previous flush.
template <typename T>
cudaError_t soc_window(afqmc_soc_ctx* ctx, cudaStream_t st, int8_t* xl, const uint8_t* rep, int mode, int s0, int n,
                       int blk, int w, bool pipe, void* Gin, void* Gcur, void* Gnext) {
    const int N = ctx->N, N2 = ctx->N2, nwk = ctx->nwk, kmax = ctx->kmax;
    const long ldz = ctx->ldz;
    const int b = w & 1, pb = (w + 1) & 1;
    cudaError_t e;
    SocWinArgs a;
    a.G0 = pipe ? Gin : ctx->G; a.gstride = ctx->gstride(); a.ldz = ldz; a.N = N;
    a.x0 = xl; a.xstride = (long)ctx->p.M * N;
    a.u0 = ctx->u; a.rep = rep;
    a.mode = mode; a.s0 = s0; a.n = n; a.blk = blk;
    a.k = ctx->k;
    a.dec0 = ctx->dec; a.ratio0 = ctx->ratio; a.lam0 = ctx->lamp;
    a.sites0 = ctx->sites[b]; a.kmax = kmax;
    a.W0 = ctx->W[b]; a.Kdev = ctx->Kdev[b]; a.err = ctx->err;
    a.corr = pipe && w > 0;
    a.pW = ctx->W[pb]; a.psites = ctx->sites[pb]; a.pKdev = ctx->Kdev[pb];
    a.Gw0 = ctx->Gw0;
    cudaStream_t sfl = pipe ? ctx->sf : st;
    if (pipe && w >= 2 && (e = cudaStreamWaitEvent(st, ctx->ev_fl[b], 0)) != cudaSuccess) return e;
    {
        const size_t shm = window_smem<T>(kmax);
        if ((e = ensure_smem_attr((const void*)soc_window_kernel<T>, shm)) != cudaSuccess) return e;
        count_launch();
        soc_window_kernel<T><<<nwk, 512, shm, st>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (pipe) {
        if ((e = cudaEventRecord(ctx->ev_win[b], st)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(sfl, ctx->ev_win[b], 0)) != cudaSuccess) return e;
    }
    const T* Gsrc = (const T*)(pipe ? Gcur : ctx->G);
    T* Gdst = (T*)(pipe ? Gnext : ctx->G2);
    const int m2max = 2 * n;
    {
        const size_t shm = (size_t)(m2max * m2max + XW_ROWS * m2max) * sizeof(cx<T>);
        {
            const int cap = 4 * kmax * kmax + XW_ROWS * 2 * kmax;
            if ((e = ensure_smem_attr((const void*)soc_xw_kernel<T>, cap * sizeof(cx<T>))) != cudaSuccess) return e;
        }
        count_launch();
        soc_xw_kernel<T><<<dim3((N2 + XW_ROWS - 1) / XW_ROWS, 1, nwk), 256, shm, sfl>>>(
            Gsrc, ctx->gstride(), ldz, N, ctx->sites[b], kmax, ctx->Kdev[b], (const cx<T>*)ctx->W[b],
            (cx<T>*)ctx->Xp[b]);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    {
        const size_t shm = (size_t)(FL_R + FL_C) * m2max * sizeof(cx<T>);
        if ((e = ensure_smem_attr((const void*)soc_flush_kernel<T>, (FL_R + FL_C) * 2 * kmax * sizeof(cx<T>))) !=
            cudaSuccess)
            return e;
        count_launch();
        soc_flush_kernel<T><<<dim3((N2 + FL_C - 1) / FL_C, (N2 + FL_R - 1) / FL_R, nwk), 256, shm, sfl>>>(
            Gsrc, Gdst, ctx->gstride(), ldz, N, ctx->sites[b], kmax, ctx->Kdev[b], (const cx<T>*)ctx->Xp[b]);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (pipe) return cudaEventRecord(ctx->ev_fl[b], sfl);
    std::swap(ctx->G, ctx->G2);  // the updated G is the current one
    return cudaSuccess;
}

template <typename T>
int soc_sweep(afqmc_soc_ctx* ctx, int slice, int dir, int mode, int k, int nb, const uint8_t* rep, cudaStream_t st) {
    const int N = ctx->N;
    int8_t* xl = ctx->x + (long)(slice - 1) * N;
    {
        SocPhase ps(ctx, AFQMC_PHASE_PREP, st);
        SCK(launch_uniforms(st, ctx->p.seed, ctx->gid, ctx->visit, 2 * N, ctx->u, ctx->nwk));
        SCK(cudaMemsetAsync(ctx->dec, 0, (size_t)ctx->nwk * 2 * N, st));
    }
    if (dir > 0) SCK(soc_wrap<T>(ctx, st, xl, +1));
    {
        // one interval for the whole update loop (window chains and their flushes): per-window
        // events would add gaps of their own to the local update's thousands of launches
        SocPhase ps(ctx, AFQMC_PHASE_CHAIN, st);
        const int wsz = (mode == AFQMC_MODE_BLOCKFB) ? nb : (mode == AFQMC_MODE_LOCAL ? 1 : k);
        const bool pipe = wsz <= SOC_PIPE_N;
        void* Gb[2] = {ctx->G, ctx->G2};  // G after window w's update: Gb[(w + 1) & 1]
        int w = 0;
        for (int s0 = 0; s0 < N; s0 += wsz, ++w) {
            const int n = std::min(wsz, N - s0);
            // window w decides on G after window w - 1's update: it reads the G before that update
            // (Gb[(w - 1) & 1], complete once flush w - 2 is) and applies the update to its block
            SCK(soc_window<T>(ctx, st, xl, rep, mode == AFQMC_MODE_BLOCKFB ? 1 : 0, s0, n, w, w, pipe,
                              Gb[w == 0 ? 0 : (w + 1) & 1], Gb[w & 1], Gb[(w + 1) & 1]));
        }
        if (pipe) {
            SCK(cudaStreamWaitEvent(st, ctx->ev_fl[(w - 1) & 1], 0));
            ctx->G = Gb[w & 1];
            ctx->G2 = Gb[(w + 1) & 1];
        }
    }
    if (dir < 0) SCK(soc_wrap<T>(ctx, st, xl, -1));
    SCK(launch_bump(st, ctx->visit));
    return AFQMC_OK;
}

// ---- FP64 recompute pieces ----
cudaError_t soc_propagate(afqmc_soc_ctx* ctx, cudaStream_t st, double* F, long wstride, int left, int l_first,
                          int l_step, int nsl) {
    SocPropArgs a;
    a.F0 = F; a.wstride = wstride; a.nv = ctx->nv; a.L = ctx->p.L; a.N = ctx->N;
    a.tab = ctx->dft; a.P = ctx->dP; a.Q = ctx->dQ; a.lam = ctx->lamk;
    a.x = ctx->x; a.xstride = (long)ctx->p.M * ctx->N;
    a.l_first = l_first; a.l_step = l_step; a.nsl = nsl; a.left = left;
    a.cg = ctx->k.c1m1 + 1.0; a.sg = ctx->k.s1; a.hs = ctx->k.hs;
    // vectors per CTA: as many (<= 4) as two buffers of 2N complex doubles allow in 220 KB
    const size_t per = (size_t)2 * ctx->N2 * sizeof(cx<double>),
                 fix = (size_t)(ctx->dP * ctx->dP + ctx->dQ * ctx->dQ + ctx->dP * ctx->dQ) * sizeof(cx<double>);
    const int vpc = (int)std::min<size_t>(PROP_VPC_MAX, (220 * 1024 - fix) / per);
    const size_t shm = vpc * per + fix;
    {
        cudaError_t e = ensure_smem_attr((const void*)soc_prop_kernel, 220 * 1024);
        if (e != cudaSuccess) return e;
    }
    count_launch();
    soc_prop_kernel<<<dim3((ctx->nv + vpc - 1) / vpc, ctx->nwk), 256, shm, st>>>(a, vpc);
    return cudaGetLastError();
}

LuArgs soc_lu_args(afqmc_soc_ctx* ctx, double* A, long wstride, long lda, int m, int n) {
    LuArgs a;
    a.A0 = A; a.wstride = wstride; a.sstride = 0; a.ng = 1;
    a.perm0 = ctx->perm; a.flag0 = ctx->flag; a.pstride = 2L * ctx->N2;
    a.lda = lda; a.m = m; a.n = n; a.nmat = ctx->nwk; a.err = ctx->err;
    return a;
}

// realified factor (4N x 2 n_e) -> its P L basis
cudaError_t soc_stab(afqmc_soc_ctx* ctx, cudaStream_t st, double* F, long wstride) {
    LuArgs a = soc_lu_args(ctx, F, wstride, ctx->nv, 2 * ctx->N2, ctx->nv);
    cudaError_t e;
    {
        SocPhase ps(ctx, AFQMC_PHASE_ELIM, st);
        if ((e = launch_lu(st, a)) != cudaSuccess) return e;
    }
    return launch_lu_unit_rows(st, a);
}

// G = 1 - R (L R)^{-1} L from stack entries R = URs[j], L^+ = ULs[j] (both realified, 4N x 2 n_e)
template <typename T>
cudaError_t soc_form_G(afqmc_soc_ctx* ctx, cudaStream_t st, int j, bool drift) {
    const int N2 = ctx->N2, nv = ctx->nv, nwk = ctx->nwk;
    const long R4 = 2L * N2;
    cudaError_t e;
    double* R = ctx->stackR(j);
    double* Lt = ctx->stackL(j);
    count_launch();
    soc_transpose_kernel<<<dim3((nv + 31) / 32, (unsigned)((R4 + 31) / 32), nwk), dim3(32, 8), 0, st>>>(
        Lt, (int)R4, nv, ctx->st_w(), ctx->Lrow, ctx->fsz());
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (ctx->oz_O) {
        OzGemmArgs o;
        o.M = nv; o.N = nv; o.K = (int)R4; o.batch = nwk;
        o.A = ctx->Lrow; o.lda = R4; o.sA = ctx->fsz();
        o.B = R; o.ldb = nv; o.sB = ctx->st_w();
        o.C = ctx->O; o.ldc = nv; o.sC = (long)nv * nv;
        o.err = ctx->err;
        SocPhase pd(ctx, AFQMC_PHASE_DGEMM, st);
        if ((e = ozaki_gemm(st, o, ctx->ozw, ctx->ozs)) != cudaSuccess) return e;
    } else {
        GemmArgs<double> g;
        g.M = nv; g.N = nv; g.K = (int)R4; g.batch = nwk;
        g.A = ctx->Lrow; g.lda = R4; g.sA = ctx->fsz();
        g.B = R; g.ldb = nv; g.sB = ctx->st_w();
        g.C = ctx->O; g.ldc = nv; g.sC = (long)nv * nv;
        if ((e = gemm<double>(st, g)) != cudaSuccess) return e;
    }
    LuArgs a = soc_lu_args(ctx, ctx->O, (long)nv * nv, nv, nv, nv);
    {
        SocPhase ps(ctx, AFQMC_PHASE_LU_O, st);
        if ((e = launch_lu(st, a)) != cudaSuccess) return e;
    }
    SolveArgs sa;
    sa.LU0 = ctx->O; sa.ostride = (long)nv * nv;
    sa.perm0 = ctx->perm; sa.pstride = a.pstride;
    sa.B0 = ctx->Lrow; sa.wstride = ctx->fsz(); sa.sstride = 0; sa.ng = 1;
    sa.ldb = R4;
    sa.Z0 = ctx->Z; sa.zstride = (long)nv * N2;
    sa.ldl = nv; sa.ns = nv; sa.N = N2; sa.nmat = nwk;
    {
        SocPhase ps(ctx, AFQMC_PHASE_SOLVE, st);
        if ((e = launch_lu_solve(st, sa)) != cudaSuccess) return e;
    }
    if (ctx->oz_G) {
        OzGemmArgs o;
        o.M = (int)R4; o.N = N2; o.K = nv; o.batch = nwk;
        o.A = R; o.lda = nv; o.sA = ctx->st_w();
        o.B = ctx->Z; o.ldb = N2; o.sB = (long)nv * N2;
        o.C = ctx->Pb; o.ldc = N2; o.sC = R4 * N2;
        o.err = ctx->err;
        SocPhase pd(ctx, AFQMC_PHASE_DGEMM, st);
        if ((e = ozaki_gemm(st, o, ctx->ozw, ctx->ozs)) != cudaSuccess) return e;
    } else {
        GemmArgs<double> h;
        h.M = (int)R4; h.N = N2; h.K = nv; h.batch = nwk;
        h.A = R; h.lda = nv; h.sA = ctx->st_w();
        h.B = ctx->Z; h.ldb = N2; h.sB = (long)nv * N2;
        h.C = ctx->Pb; h.ldc = N2; h.sC = R4 * N2;
        if ((e = gemm<double>(st, h)) != cudaSuccess) return e;
    }
    count_launch();
    soc_store_G_kernel<T><<<dim3(256, nwk), 256, 0, st>>>(ctx->Pb, R4 * N2, N2, (T*)ctx->G, ctx->ldz, ctx->gstride(),
                                                         ctx->acc2, drift ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t soc_to_stack(afqmc_soc_ctx* ctx, cudaStream_t st, bool right, int j) {
    double* dst = right ? ctx->stackR(j) : ctx->stackL(j);
    return cudaMemcpy2DAsync(dst, ctx->st_w() * 8, ctx->Ucur, ctx->fsz() * 8, ctx->fsz() * 8, ctx->nwk,
                             cudaMemcpyDeviceToDevice, st);
}
cudaError_t soc_from_stack(afqmc_soc_ctx* ctx, cudaStream_t st, bool right, int j) {
    const double* src = right ? ctx->stackR(j) : ctx->stackL(j);
    return cudaMemcpy2DAsync(ctx->Ucur, ctx->fsz() * 8, src, ctx->st_w() * 8, ctx->fsz() * 8, ctx->nwk,
                             cudaMemcpyDeviceToDevice, st);
}

int check(afqmc_soc_ctx* ctx) {
    if (!ctx) return AFQMC_ERR_ARG;
    return ctx->sticky;
}

}  // namespace

extern "C" {

int afqmc_soc_create(afqmc_soc_ctx** out, const afqmc_soc_params* p) {
    if (!out || !p) return AFQMC_ERR_ARG;
    *out = nullptr;
    const int L = p->L, N = L * L;
    if (L < 2 || L > 48 || p->M < 1 || p->stab_every < 1 || p->M % p->stab_every != 0 || p->n_e < 1 ||
        p->n_e > 2 * N || p->n_walkers < 1 || !(p->U <= 0.0) || !(p->dtau > 0.0) ||
        (p->hs != AFQMC_SOC_HS_SY && p->hs != AFQMC_SOC_HS_SZ))
        return AFQMC_ERR_ARG;
    if (p->precision != AFQMC_PREC_FP64 && p->precision != AFQMC_PREC_FP32) return AFQMC_ERR_ARG;
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return AFQMC_ERR_NODEV;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3) return AFQMC_ERR_NODEV;
    afqmc_soc_ctx* c = new afqmc_soc_ctx();
    c->p = *p;
    c->N = N;
    c->N2 = 2 * N;
    c->ne = p->n_e;
    c->nv = 2 * p->n_e;
    c->nwk = p->n_walkers;
    c->ldz = ((2L * N + 31) / 32) * 32;
    c->f64 = p->precision == AFQMC_PREC_FP64;
    c->use_tc = !c->f64 && p->gemm != AFQMC_GEMM_SIMT;
    c->kmax = c->f64 ? AFQMC_SOC_KMAX_FP64 : AFQMC_SOC_KMAX_FP32;
    c->nst = p->M / p->stab_every + 1;
    // the lattice DFT: the factor pair L = P Q with the fewest multiply-adds per output
    // (P + Q + 1 with a twiddle), else the plain L-term sum
    c->dP = L;
    c->dQ = 1;
    for (int q = 2; q < L; ++q)
        if (L % q == 0 && L / q + q + 1 < c->dP + (c->dQ > 1 ? c->dQ + 1 : 0)) {
            c->dP = L / q;
            c->dQ = q;
        }
    const double g = acos(exp(p->dtau * p->U / 2.0));
    c->k.gamma = g;
    c->k.c2m1 = cos(2.0 * g) - 1.0;
    c->k.s2 = sin(2.0 * g);
    c->k.c1m1 = cos(g) - 1.0;
    c->k.s1 = sin(g);
    c->k.hs = p->hs;
    *out = c;
    return AFQMC_OK;
}

int afqmc_soc_destroy(afqmc_soc_ctx* ctx) {
    if (!ctx) return AFQMC_OK;
    cudaDeviceSynchronize();
    for (void* q : ctx->allocs) cudaFree(q);
    for (int q = 0; q < 2; ++q) {
        if (ctx->ev_win[q]) cudaEventDestroy(ctx->ev_win[q]);
        if (ctx->ev_fl[q]) cudaEventDestroy(ctx->ev_fl[q]);
    }
    if (ctx->sf) cudaStreamDestroy(ctx->sf);
    for (auto& ev : ctx->pending) {
        cudaEventDestroy(ev.a);
        cudaEventDestroy(ev.b);
    }
    for (auto ev : ctx->pool) cudaEventDestroy(ev);
    delete ctx;
    return AFQMC_OK;
}

int afqmc_soc_init(afqmc_soc_ctx* ctx, const double* P, const int8_t* fields, void* stream) {
    int rc = check(ctx);
    if (rc) return rc;
    if (!P || ctx->inited) return AFQMC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    ctx->last = st;
    const int N = ctx->N, N2 = ctx->N2, M = ctx->p.M, S = ctx->p.stab_every, nwk = ctx->nwk, ne = ctx->ne;
    const long ldz = ctx->ldz, ld2 = 2 * ldz;
    const size_t es = ctx->f64 ? 8 : 4;
    const int kmax = ctx->kmax;
    SCK(soc_alloc(ctx, &ctx->Ers, (size_t)N2 * ld2 * es, st));
    SCK(soc_alloc(ctx, &ctx->Einvrs, (size_t)N2 * ld2 * es, st));
    SCK(soc_alloc(ctx, &ctx->Ech, (size_t)ld2 * ld2 * es, st));
    SCK(soc_alloc(ctx, &ctx->Einvch, (size_t)ld2 * ld2 * es, st));
    SCK(soc_alloc(ctx, &ctx->dft, (size_t)(ctx->p.L * ctx->p.L + 2 * ctx->p.L + 2) * 16, st));
    SCK(soc_alloc(ctx, &ctx->lamk, (size_t)N * 64, st));
    SCK(soc_alloc(ctx, &ctx->G, (size_t)nwk * ctx->gstride() * es, st));
    SCK(soc_alloc(ctx, &ctx->S, (size_t)nwk * ld2 * ld2 * es, st));
    SCK(soc_alloc(ctx, &ctx->x, (size_t)nwk * M * N, st));
    SCK(soc_alloc(ctx, &ctx->u, (size_t)nwk * 2 * N * 8, st));
    SCK(soc_alloc(ctx, &ctx->rep, (size_t)nwk * 2 * N, st));
    SCK(soc_alloc(ctx, &ctx->dec, (size_t)nwk * 2 * N, st));
    SCK(soc_alloc(ctx, &ctx->ratio, (size_t)nwk * 4 * N * 8, st));
    SCK(soc_alloc(ctx, &ctx->lamp, (size_t)nwk * N * 8, st));
    SCK(soc_alloc(ctx, &ctx->gid, (size_t)nwk * sizeof(int), st));
    SCK(soc_alloc(ctx, &ctx->visit, 8, st));
    SCK(soc_alloc(ctx, &ctx->G2, (size_t)nwk * ctx->gstride() * es, st));
    for (int q = 0; q < 2; ++q) {
        SCK(soc_alloc(ctx, &ctx->Xp[q], (size_t)nwk * N2 * 4 * kmax * es, st));
        SCK(soc_alloc(ctx, &ctx->W[q], (size_t)nwk * 8 * kmax * kmax * es, st));
        SCK(soc_alloc(ctx, &ctx->Kdev[q], (size_t)nwk * sizeof(int), st));
        SCK(soc_alloc(ctx, &ctx->sites[q], (size_t)nwk * kmax * sizeof(int), st));
        SCK(cudaEventCreateWithFlags(&ctx->ev_win[q], cudaEventDisableTiming));
        SCK(cudaEventCreateWithFlags(&ctx->ev_fl[q], cudaEventDisableTiming));
    }
    SCK(soc_alloc(ctx, &ctx->Gw0, (size_t)nwk * 8 * kmax * kmax * es, st));
    SCK(cudaStreamCreateWithFlags(&ctx->sf, cudaStreamNonBlocking));
    SCK(soc_alloc(ctx, &ctx->err, sizeof(int), st));
    SCK(soc_alloc(ctx, &ctx->URs, (size_t)nwk * ctx->st_w() * 8, st));
    SCK(soc_alloc(ctx, &ctx->ULs, (size_t)nwk * ctx->st_w() * 8, st));
    SCK(soc_alloc(ctx, &ctx->Ucur, (size_t)nwk * ctx->fsz() * 8, st));
    SCK(soc_alloc(ctx, &ctx->Lrow, (size_t)nwk * ctx->fsz() * 8, st));
    SCK(soc_alloc(ctx, &ctx->O, (size_t)nwk * ctx->nv * ctx->nv * 8, st));
    SCK(soc_alloc(ctx, &ctx->Z, (size_t)nwk * ctx->nv * N2 * 8, st));
    SCK(soc_alloc(ctx, &ctx->Pb, (size_t)nwk * 2 * N2 * N2 * 8, st));
    SCK(soc_alloc(ctx, &ctx->perm, (size_t)nwk * 2 * N2 * sizeof(int), st));
    SCK(soc_alloc(ctx, &ctx->flag, (size_t)nwk * 2 * N2, st));
    SCK(soc_alloc(ctx, &ctx->acc2, (size_t)nwk * 16, st));
    SCK(soc_alloc(ctx, &ctx->en, (size_t)nwk * 16, st));
    if (ctx->p.gemm != AFQMC_GEMM_SIMT) {
        const int nv = ctx->nv, R4 = 2 * N2;
        ctx->oz_O = ozaki_pays(nv, nv, R4, nwk);
        ctx->oz_G = ozaki_pays(R4, N2, nv, nwk);
        if (ctx->oz_O || ctx->oz_G) {
            const size_t f1 = ozaki_ws_bytes(nv, nv, R4, nwk), f2 = ozaki_ws_bytes(R4, N2, nv, nwk);
            SCK(soc_alloc(ctx, (char**)&ctx->ozw, f1 > f2 ? f1 : f2, st));
            SCK(soc_alloc(ctx, &ctx->ozs, ozaki_sc_doubles(R4, R4, nwk) * 8, st));
        }
    }
    if (ctx->f64) SCK(upload_constants<double>(ctx, st));
    else SCK(upload_constants<float>(ctx, st));
    count_launch();
    soc_iota_kernel<<<(nwk + 255) / 256, 256, 0, st>>>(ctx->gid, nwk);
    SCK(cudaGetLastError());
    if (fields) {
        SCK(cudaMemcpyAsync(ctx->x, fields, (size_t)nwk * M * N, cudaMemcpyHostToDevice, st));
    } else {
        count_launch();
        soc_fields_kernel<<<dim3((unsigned)(((long)M * N + 255) / 256), nwk), 256, 0, st>>>(ctx->p.seed, (long)M * N,
                                                                                          ctx->x);
        SCK(cudaGetLastError());
    }
    // realified trial determinant [[Re P, -Im P], [Im P, Re P]] (4N x 2 n_e): U_R(0), and also
    // the realified U_L(M)^+ = realified(P)
    std::vector<double> R0((size_t)ctx->fsz());
    const int nv = ctx->nv;
    for (int a = 0; a < N2; ++a)
        for (int c = 0; c < ne; ++c) {
            const double pr = P[((size_t)a * ne + c) * 2], pi = P[((size_t)a * ne + c) * 2 + 1];
            R0[(size_t)a * nv + c] = pr;
            R0[(size_t)a * nv + ne + c] = -pi;
            R0[(size_t)(N2 + a) * nv + c] = pi;
            R0[(size_t)(N2 + a) * nv + ne + c] = pr;
        }
    for (int j = 0; j < nwk; ++j) {
        SCK(cudaMemcpyAsync(ctx->Ucur + (size_t)j * ctx->fsz(), R0.data(), R0.size() * 8, cudaMemcpyHostToDevice, st));
    }
    SCK(cudaStreamSynchronize(st));  // R0 goes out of scope
    SCK(soc_stab(ctx, st, ctx->Ucur, ctx->fsz()));
    SCK(soc_to_stack(ctx, st, true, 0));
    SCK(soc_to_stack(ctx, st, false, M / S));
    for (int jj = M / S; jj >= 1; --jj) {
        SCK(soc_propagate(ctx, st, ctx->Ucur, ctx->fsz(), 1, jj * S, -1, S));
        SCK(soc_stab(ctx, st, ctx->Ucur, ctx->fsz()));
        SCK(soc_to_stack(ctx, st, false, jj - 1));
    }
    if (ctx->f64) SCK(soc_form_G<double>(ctx, st, 0, false));
    else SCK(soc_form_G<float>(ctx, st, 0, false));
    SCK(cudaStreamSynchronize(st));
    ctx->pos = 0;
    ctx->last_dir = -1;
    ctx->need_recompute = false;
    ctx->inited = true;
    return read_err(ctx);
}

int afqmc_soc_sweep_slice(afqmc_soc_ctx* ctx, int slice, int dir, int mode, int k, int nb, const uint8_t* replay,
                          void* stream) {
    int rc = check(ctx);
    if (rc) return rc;
    if (!ctx->inited || slice < 1 || slice > ctx->p.M || (dir != 1 && dir != -1)) return AFQMC_ERR_ARG;
    if (mode != AFQMC_MODE_LOCAL && mode != AFQMC_MODE_DELAYED && mode != AFQMC_MODE_BLOCKFB) return AFQMC_ERR_ARG;
    if (mode == AFQMC_MODE_DELAYED && (k < 1 || k > ctx->kmax)) return AFQMC_ERR_ARG;
    if (mode == AFQMC_MODE_BLOCKFB && (nb < 1 || nb > ctx->kmax)) return AFQMC_ERR_ARG;
    if (ctx->need_recompute) return AFQMC_ERR_STATE;
    if ((dir > 0 && ctx->pos != slice - 1) || (dir < 0 && ctx->pos != slice)) return AFQMC_ERR_STATE;
    cudaStream_t st = (cudaStream_t)stream;
    ctx->last = st;
    const uint8_t* rep = nullptr;
    if (replay) {
        SCK(cudaMemcpyAsync(ctx->rep, replay, (size_t)ctx->nwk * 2 * ctx->N, cudaMemcpyHostToDevice, st));
        SCK(cudaStreamSynchronize(st));
        rep = ctx->rep;
    }
    rc = ctx->f64 ? soc_sweep<double>(ctx, slice, dir, mode, k, nb, rep, st)
                  : soc_sweep<float>(ctx, slice, dir, mode, k, nb, rep, st);
    if (rc) return rc;
    ctx->pos = dir > 0 ? slice : slice - 1;
    ctx->last_dir = dir;
    if (ctx->pos % ctx->p.stab_every == 0) ctx->need_recompute = true;
    return AFQMC_OK;
}

int afqmc_soc_recompute_G(afqmc_soc_ctx* ctx, double* rel_drift, void* stream) {
    int rc = check(ctx);
    if (rc) return rc;
    if (!ctx->inited) return AFQMC_ERR_ARG;
    const int S = ctx->p.stab_every;
    if (ctx->pos % S != 0) return AFQMC_ERR_STATE;
    cudaStream_t st = (cudaStream_t)stream;
    ctx->last = st;
    const int j = ctx->pos / S;
    SocPhase ps(ctx, AFQMC_PHASE_RECOMPUTE, st);
    SCK(cudaMemsetAsync(ctx->acc2, 0, (size_t)ctx->nwk * 16, st));
    const bool fwd = ctx->last_dir > 0;
    const bool prop = fwd ? (j > 0) : (ctx->pos != ctx->p.M);
    if (prop) {
        SCK(soc_from_stack(ctx, st, fwd, fwd ? j - 1 : j + 1));
        if (fwd) SCK(soc_propagate(ctx, st, ctx->Ucur, ctx->fsz(), 0, ctx->pos - S + 1, 1, S));
        else SCK(soc_propagate(ctx, st, ctx->Ucur, ctx->fsz(), 1, ctx->pos + S, -1, S));
        SCK(soc_stab(ctx, st, ctx->Ucur, ctx->fsz()));
        SCK(soc_to_stack(ctx, st, fwd, j));
    }
    if (ctx->f64) SCK(soc_form_G<double>(ctx, st, j, true));
    else SCK(soc_form_G<float>(ctx, st, j, true));
    ctx->need_recompute = false;
    if (rel_drift) {
        SCK(cudaStreamSynchronize(st));
        rc = read_err(ctx);
        if (rc) return rc;
        std::vector<double> h((size_t)ctx->nwk * 2);
        SCK(cudaMemcpy(h.data(), ctx->acc2, h.size() * 8, cudaMemcpyDeviceToHost));
        for (int w = 0; w < ctx->nwk; ++w) rel_drift[w] = h[2 * w + 1] > 0 ? sqrt(h[2 * w] / h[2 * w + 1]) : 0.0;
    }
    return AFQMC_OK;
}

int afqmc_soc_measure_pairing(afqmc_soc_ctx* ctx, double* scalars, double* nk, double* Mk, void* stream) {
    int rc = check(ctx);
    if (rc) return rc;
    if (!ctx->inited || !scalars) return AFQMC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    ctx->last = st;
    const int L = ctx->p.L, N = ctx->N, N2 = ctx->N2, nwk = ctx->nwk;
    const long ldz = ctx->ldz, ld2 = 2 * ldz;
    if (!ctx->Frs) {
        // F2 = diag(F, F), F_{q j} = N^{-1/2} e^{-i q.r_j}: its rows for the left product and the
        // realified right operand of the product by F2^+ (C~ = [[Re C, Im C], [-Im C, Re C]])
        std::vector<double> frs((size_t)N2 * ld2, 0.0), fh((size_t)ld2 * ld2, 0.0);
        const double sN = 1.0 / sqrt((double)N);
        for (int q = 0; q < N; ++q)
            for (int jj = 0; jj < N; ++jj) {
                const double ph = -2.0 * M_PI * ((double)(q % L) * (jj % L) + (double)(q / L) * (jj / L)) / L;
                const double fr = cos(ph) * sN, fi = sin(ph) * sN;
                for (int sp = 0; sp < 2; ++sp) {
                    const long r = sp * N + q, c = sp * N + jj;  // F2[r][c] = F[q][jj]
                    frs[(size_t)r * ld2 + c] = fr;
                    frs[(size_t)r * ld2 + ldz + c] = fi;
                    // C = F2^+: C[c][r] = conj(F2[r][c])
                    fh[(size_t)c * ld2 + r] = fr;
                    fh[(size_t)c * ld2 + ldz + r] = -fi;
                    fh[(size_t)(ldz + c) * ld2 + r] = fi;
                    fh[(size_t)(ldz + c) * ld2 + ldz + r] = fr;
                }
            }
        SCK(soc_alloc(ctx, &ctx->Frs, frs.size() * 8, st));
        SCK(soc_alloc(ctx, &ctx->Fh, fh.size() * 8, st));
        SCK(soc_alloc(ctx, &ctx->pA, (size_t)N2 * ld2 * 8, st));
        SCK(soc_alloc(ctx, &ctx->pS, (size_t)ld2 * ld2 * 8, st));
        SCK(soc_alloc(ctx, &ctx->pAt, (size_t)N2 * ld2 * 8, st));
        SCK(soc_alloc(ctx, &ctx->pMk, (size_t)nwk * N * N * 16, st));
        SCK(soc_alloc(ctx, &ctx->pOut, (size_t)nwk * (4 + 4 * N) * 8, st));
        SCK(cudaMemcpyAsync(ctx->Frs, frs.data(), frs.size() * 8, cudaMemcpyHostToDevice, st));
        SCK(cudaMemcpyAsync(ctx->Fh, fh.data(), fh.size() * 8, cudaMemcpyHostToDevice, st));
        SCK(cudaStreamSynchronize(st));  // the host tables go out of scope
    }
    SCK(cudaMemsetAsync(ctx->pOut, 0, (size_t)nwk * (4 + 4 * N) * 8, st));
    const size_t es = ctx->f64 ? 8 : 4;
    for (int w = 0; w < nwk; ++w) {
        const void* Gw = (const char*)ctx->G + (size_t)w * ctx->gstride() * es;
        double* out = ctx->pOut + (size_t)w * 4;
        double* nkw = ctx->pOut + (size_t)nwk * 4 + (size_t)w * 4 * N;
        const dim3 grid((unsigned)((ld2 + 255) / 256), N2);
        count_launch();
        if (ctx->f64) soc_one_minus_kernel<double><<<grid, 256, 0, st>>>((const double*)Gw, ldz, ctx->pA);
        else soc_one_minus_kernel<float><<<grid, 256, 0, st>>>((const float*)Gw, ldz, ctx->pA);
        SCK(cudaGetLastError());
        count_launch();
        soc_pair_scalars_kernel<<<(unsigned)std::min<long>(((long)N * N + 255) / 256, 1024), 256, 0, st>>>(
            ctx->pA, ldz, N, out);
        SCK(cudaGetLastError());
        if (!nk && !Mk) continue;
        // At = F2 A F2^+: S~ rows [0, 2N) = A (F2^+)~, the realified S~, then [Re F2 | Im F2] S~
        GemmArgs<double> g1;
        g1.M = N2; g1.N = (int)ld2; g1.K = (int)ld2;
        g1.A = ctx->pA; g1.lda = ld2;
        g1.B = ctx->Fh; g1.ldb = ld2;
        g1.C = ctx->pS; g1.ldc = ld2;
        SCK(gemm<double>(st, g1));
        count_launch();
        soc_realify_kernel<double><<<dim3((unsigned)((ld2 + 255) / 256), N2, 1), 256, 0, st>>>(ctx->pS, ldz, N2, 0, 1);
        SCK(cudaGetLastError());
        GemmArgs<double> g2;
        g2.M = N2; g2.N = (int)ld2; g2.K = (int)ld2;
        g2.A = ctx->Frs; g2.lda = ld2;
        g2.B = ctx->pS; g2.ldb = ld2;
        g2.C = ctx->pAt; g2.ldc = ld2;
        SCK(gemm<double>(st, g2));
        count_launch();
        soc_pair_k_kernel<<<(unsigned)std::min<long>(((long)N * N + 255) / 256, 4096), 256, 0, st>>>(
            ctx->pAt, ldz, L, ctx->pMk + (size_t)w * 2 * N * N, nkw);
        SCK(cudaGetLastError());
    }
    std::vector<double> h((size_t)nwk * (4 + 4 * N));
    SCK(cudaMemcpyAsync(h.data(), ctx->pOut, h.size() * 8, cudaMemcpyDeviceToHost, st));
    if (Mk) SCK(cudaMemcpyAsync(Mk, ctx->pMk, (size_t)nwk * N * N * 16, cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    rc = read_err(ctx);
    if (rc) return rc;
    for (int w = 0; w < nwk; ++w) {
        scalars[4 * w + 0] = h[4 * w + 0] / N;
        scalars[4 * w + 1] = h[4 * w + 1] / N;
        scalars[4 * w + 2] = h[4 * w + 2] / (4.0 * N * N);
        scalars[4 * w + 3] = h[4 * w + 3] / (4.0 * N * N);
        if (nk) memcpy(nk + (size_t)w * 4 * N, h.data() + (size_t)nwk * 4 + (size_t)w * 4 * N, (size_t)4 * N * 8);
    }
    return AFQMC_OK;
}

int afqmc_soc_measure_energy(afqmc_soc_ctx* ctx, double* energy, void* stream) {
    int rc = check(ctx);
    if (rc) return rc;
    if (!ctx->inited || !energy) return AFQMC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    ctx->last = st;
    count_launch();
    if (ctx->f64)
        soc_energy_kernel<double><<<ctx->nwk, 256, 0, st>>>((const double*)ctx->G, ctx->ldz, ctx->gstride(), ctx->p.L,
                                                           ctx->p.t, ctx->p.lam, ctx->p.U, ctx->en);
    else
        soc_energy_kernel<float><<<ctx->nwk, 256, 0, st>>>((const float*)ctx->G, ctx->ldz, ctx->gstride(), ctx->p.L,
                                                          ctx->p.t, ctx->p.lam, ctx->p.U, ctx->en);
    SCK(cudaGetLastError());
    SCK(cudaStreamSynchronize(st));
    rc = read_err(ctx);
    if (rc) return rc;
    SCK(cudaMemcpy(energy, ctx->en, (size_t)ctx->nwk * 16, cudaMemcpyDeviceToHost));
    return AFQMC_OK;
}

static int soc_sync_walker(afqmc_soc_ctx* ctx, int walker) {
    int rc = check(ctx);
    if (rc) return rc;
    if (!ctx->inited || walker < 0 || walker >= ctx->nwk) return AFQMC_ERR_ARG;
    if (cudaStreamSynchronize(ctx->last) != cudaSuccess) return soc_fail(ctx, cudaGetLastError());
    return read_err(ctx);
}

int afqmc_soc_get_G(afqmc_soc_ctx* ctx, int walker, double* out) {
    int rc = soc_sync_walker(ctx, walker);
    if (rc) return rc;
    if (!out) return AFQMC_ERR_ARG;
    const int N2 = ctx->N2;
    const long ld2 = 2 * ctx->ldz;
    const size_t es = ctx->f64 ? 8 : 4;
    std::vector<unsigned char> h((size_t)N2 * ld2 * es);
    SCK(cudaMemcpy(h.data(), (char*)ctx->G + (size_t)walker * ctx->gstride() * es, h.size(), cudaMemcpyDeviceToHost));
    for (int r = 0; r < N2; ++r)
        for (int c = 0; c < N2; ++c) {
            double re, im;
            if (ctx->f64) {
                re = ((double*)h.data())[(size_t)r * ld2 + c];
                im = ((double*)h.data())[(size_t)r * ld2 + ctx->ldz + c];
            } else {
                re = ((float*)h.data())[(size_t)r * ld2 + c];
                im = ((float*)h.data())[(size_t)r * ld2 + ctx->ldz + c];
            }
            out[((size_t)r * N2 + c) * 2] = re;
            out[((size_t)r * N2 + c) * 2 + 1] = im;
        }
    return AFQMC_OK;
}

int afqmc_soc_set_G(afqmc_soc_ctx* ctx, int walker, const double* in) {
    int rc = soc_sync_walker(ctx, walker);
    if (rc) return rc;
    if (!in) return AFQMC_ERR_ARG;
    const int N2 = ctx->N2;
    const long ld2 = 2 * ctx->ldz;
    const size_t es = ctx->f64 ? 8 : 4;
    std::vector<unsigned char> h((size_t)N2 * ld2 * es, 0);
    for (int r = 0; r < N2; ++r)
        for (int c = 0; c < N2; ++c) {
            const double re = in[((size_t)r * N2 + c) * 2], im = in[((size_t)r * N2 + c) * 2 + 1];
            if (ctx->f64) {
                ((double*)h.data())[(size_t)r * ld2 + c] = re;
                ((double*)h.data())[(size_t)r * ld2 + ctx->ldz + c] = im;
            } else {
                ((float*)h.data())[(size_t)r * ld2 + c] = (float)re;
                ((float*)h.data())[(size_t)r * ld2 + ctx->ldz + c] = (float)im;
            }
        }
    SCK(cudaMemcpy((char*)ctx->G + (size_t)walker * ctx->gstride() * es, h.data(), h.size(), cudaMemcpyHostToDevice));
    return AFQMC_OK;
}

int afqmc_soc_get_fields(afqmc_soc_ctx* ctx, int walker, int8_t* out) {
    int rc = soc_sync_walker(ctx, walker);
    if (rc) return rc;
    if (!out) return AFQMC_ERR_ARG;
    const size_t n = (size_t)ctx->p.M * ctx->N;
    SCK(cudaMemcpy(out, ctx->x + (size_t)walker * n, n, cudaMemcpyDeviceToHost));
    return AFQMC_OK;
}

int afqmc_soc_get_decisions(afqmc_soc_ctx* ctx, int walker, uint8_t* out) {
    int rc = soc_sync_walker(ctx, walker);
    if (rc) return rc;
    if (!out) return AFQMC_ERR_ARG;
    SCK(cudaMemcpy(out, ctx->dec + (size_t)walker * 2 * ctx->N, 2 * (size_t)ctx->N, cudaMemcpyDeviceToHost));
    return AFQMC_OK;
}

int afqmc_soc_get_ratios(afqmc_soc_ctx* ctx, int walker, double* out) {
    int rc = soc_sync_walker(ctx, walker);
    if (rc) return rc;
    if (!out) return AFQMC_ERR_ARG;
    SCK(cudaMemcpy(out, ctx->ratio + (size_t)walker * 4 * ctx->N, 4 * (size_t)ctx->N * 8, cudaMemcpyDeviceToHost));
    return AFQMC_OK;
}

int afqmc_soc_get_lam_plus(afqmc_soc_ctx* ctx, int walker, double* out) {
    int rc = soc_sync_walker(ctx, walker);
    if (rc) return rc;
    if (!out) return AFQMC_ERR_ARG;
    SCK(cudaMemcpy(out, ctx->lamp + (size_t)walker * ctx->N, (size_t)ctx->N * 8, cudaMemcpyDeviceToHost));
    return AFQMC_OK;
}

int afqmc_soc_get_info(afqmc_soc_ctx* ctx, int* N, int* slice, int* dir) {
    if (!ctx) return AFQMC_ERR_ARG;
    if (N) *N = ctx->N;
    if (slice) *slice = ctx->pos;
    if (dir) *dir = ctx->last_dir;
    return AFQMC_OK;
}

int afqmc_soc_set_profiling(afqmc_soc_ctx* ctx, int on) {
    if (!ctx) return AFQMC_ERR_ARG;
    ctx->prof_on = on != 0;
    for (int q = 0; q < AFQMC_NPHASE; ++q) {
        ctx->ms[q] = 0.0;
        ctx->intervals[q] = 0;
        ctx->launches[q] = 0;
    }
    for (auto& ev : ctx->pending) {
        ctx->pool.push_back(ev.a);
        ctx->pool.push_back(ev.b);
    }
    ctx->pending.clear();
    return AFQMC_OK;
}

int afqmc_soc_get_profile(afqmc_soc_ctx* ctx, double* ms, int64_t* intervals, int64_t* launches) {
    if (!ctx) return AFQMC_ERR_ARG;
    if (ctx->last) cudaStreamSynchronize(ctx->last);
    cudaDeviceSynchronize();
    for (auto& ev : ctx->pending) {
        float t = 0.0f;
        cudaEventElapsedTime(&t, ev.a, ev.b);
        ctx->ms[ev.ph] += t;
        ctx->intervals[ev.ph] += 1;
        ctx->pool.push_back(ev.a);
        ctx->pool.push_back(ev.b);
    }
    ctx->pending.clear();
    for (int q = 0; q < AFQMC_NPHASE; ++q) {
        if (ms) ms[q] = ctx->ms[q];
        if (intervals) intervals[q] = ctx->intervals[q];
        if (launches) launches[q] = ctx->launches[q];
    }
    return AFQMC_OK;
}

}  // extern "C"
