// sweep.cu -- the per-slice site loop of the PQMC update sweep in G form.
//
//   local   : persistent cooperative kernel, one grid barrier per site, the
//             rank-1 update G <- G - (d/r) G_{:,i} (e_i^T - G_{i,:}) applied to
//             the whole of G on every accepted flip (Eqs. DetRatiolocal,
//             UpdateLTRlocal restated for G).
//   delayed : a window of n consecutive sites is decided by ONE CTA on the
//   blockfb   n x n diagonal block of G held in shared memory; the accepted
//             flips I are then applied to the full G as one rank-|I| product
//                 G <- G - G[:, I] W (E_I^T - G[I, :]),  W = D_I (1 + A0_II D_I)^{-1}
//             which equals the buffered sum of the paper's delayed vectors
//             (Eqs. DelayTMat00, DelayRgenk, FinalDelay) and the block
//             force-bias upgrade (Eq. BlkFrcBsTnew2).
#include <math.h>

#include "internal.h"

namespace afq {

// ---------------------------------------------------------------------------
// uniforms of one slice visit
// ---------------------------------------------------------------------------
// The visit counter lives on the device so that a captured slice replays with fresh uniforms.
__global__ void uniforms_kernel(uint64_t seed, const int* gid, const unsigned long long* visit, int count, double* u) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int w = blockIdx.y;
    if (j < count) u[(size_t)w * count + j] = philox_uniform(seed, (uint64_t)gid[w], (uint64_t)*visit, (uint64_t)j);
}

__global__ void bump_kernel(unsigned long long* visit) { *visit += 1ULL; }

cudaError_t launch_uniforms(cudaStream_t st, uint64_t seed, const int* gid, const unsigned long long* visit, int count,
                            double* u, int nwk) {
    count_launch();
    uniforms_kernel<<<dim3((count + 255) / 256, nwk), 256, 0, st>>>(seed, gid, visit, count, u);
    return cudaGetLastError();
}

cudaError_t launch_bump(cudaStream_t st, unsigned long long* visit) {
    count_launch();
    bump_kernel<<<1, 1, 0, st>>>(visit);
    return cudaGetLastError();
}

// Buffers of walker j of a group (see Batch).
template <typename T>
__device__ __forceinline__ WindowBufs wb_walker(WindowBufs wb, int j, int N);
__device__ __forceinline__ SliceOut so_walker(SliceOut so, int j, int N) {
    so.dec += (size_t)j * 2 * N;
    so.ratio += (size_t)j * 2 * N;
    so.stats += (size_t)j * 8;
    so.maxr += j;
    if (so.sign) so.sign += j;
    if (so.cp) so.cp += (size_t)j * 4;
    return so;
}

__device__ __forceinline__ double hs_log_scalar(const SiteParams& sp, int x) {
    return sp.hs == AFQMC_HS_CHARGE_REAL ? -sp.lam * (double)x : 0.0;
}

// ---------------------------------------------------------------------------
// local update: persistent cooperative kernel, one grid barrier per ACCEPT
// ---------------------------------------------------------------------------
// CTA b owns the rows [r0, r1) of both spins.  A phase handles one accepted site:
//   1. thread 0 of every CTA passes the grid barrier (one release reduction on an arrival counter,
//      then polling), and warp 0 at once scans the sites after the last accept (32 sites per round;
//      a ballot finds the first acceptance) from a copy of the two diagonals in global memory.
//      Every CTA reads the same values and runs the same arithmetic, so all reach the same site b;
//   2. every CTA reads row b of both spins (e_b^T - G[b, :]) and column b of its own rows;
//   3. every CTA applies G_s[r, c] -= f_s G_s[r, b] (delta_bc - G_s[b, c]) to its own rows with
//      16-byte accesses and several loads in flight per thread, and writes the new diagonal of its
//      rows to the other diagonal buffer.
// A rejected site leaves G unchanged, so it costs a diagonal read and no barrier.  Two cross-CTA
// hazards inside a phase are avoided without a second grid barrier:
//   * the diagonals are double-buffered by phase parity: the scan reads the buffer the previous
//     phase wrote, and the update writes the other one;
//   * every CTA reads row b while its owner updates its rows, so the owner keeps its new row b in
//     shared memory and stores it to G in the next phase, after the barrier (no CTA reads row b
//     again in this slice).
// The diagonal copy is computed with the same fused multiply-add as the element of G, so the two
// stay bit-identical.  diag: [2 buffers][2 spins][N].
template <typename T> struct Vec16;
template <> struct Vec16<float> { using V = float4; static constexpr int W = 4; };
template <> struct Vec16<double> { using V = double2; static constexpr int W = 2; };

template <typename T>
__device__ __forceinline__ void vfma_rank1(typename Vec16<T>::V& g, T a, const typename Vec16<T>::V& r);
template <>
__device__ __forceinline__ void vfma_rank1<float>(float4& g, float a, const float4& r) {
    g.x = fmaf(a, r.x, g.x); g.y = fmaf(a, r.y, g.y); g.z = fmaf(a, r.z, g.z); g.w = fmaf(a, r.w, g.w);
}
template <>
__device__ __forceinline__ void vfma_rank1<double>(double2& g, double a, const double2& r) {
    g.x = fma(a, r.x, g.x); g.y = fma(a, r.y, g.y);
}

constexpr int LOCAL_THREADS = 1024;
// Loads in flight per thread in the row update (the largest count that fits 64 registers)
template <typename T> struct LocalUnroll { static constexpr int U = sizeof(T) == 4 ? 6 : 4; };

// Shared-memory layout of local_kernel (byte offsets, 16-byte aligned where vectors are read).
struct LocalSmem {
    size_t us, rowb, patch, colb, xs, rp, total;
};
template <typename T>
__host__ __device__ inline LocalSmem local_smem(int N, long ld, int nrmax) {
    auto al = [](size_t b) { return (b + 15) & ~(size_t)15; };
    LocalSmem s;
    s.us = 0;                                              // double us[N]: the site uniforms
    s.rowb = al(s.us + (size_t)N * sizeof(double));        // T rowb[2][ld]: e_b^T - G_s[b, :], 0 beyond N
    s.patch = al(s.rowb + 2 * (size_t)ld * sizeof(T));     // T patch[2][ld]: the owner's new row b
    s.colb = al(s.patch + 2 * (size_t)ld * sizeof(T));     // T colb[2][nrmax]: G_s[r, b] of the own rows
    s.xs = al(s.colb + 2 * (size_t)nrmax * sizeof(T));     // int8 xs[N]: fields of the slice
    s.rp = s.xs + (size_t)N;                               // uint8 rp[N]: forced decisions
    s.total = al(s.rp + (size_t)N);
    return s;
}

template <typename T>
__global__ void __launch_bounds__(LOCAL_THREADS, 1) local_kernel(T* Gu, T* Gd, int8_t* xl_g, const double* u,
                                                                 const uint8_t* replay, SiteParams sp, SliceOut so,
                                                                 T* diag, GridBar* bar, int* err, int nrmax) {
    using V = typename Vec16<T>::V;
    constexpr int VW = Vec16<T>::W;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = sp.N;
    const long ld = sp.ld;
    const int nblk = gridDim.x, b = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const int r0 = (int)((long)N * b / nblk), r1 = (int)((long)N * (b + 1) / nblk);
    const int nr = r1 - r0;
    const int nv = (N + VW - 1) / VW;  // 16-byte vectors per row; VW nv <= ld (ld is padded to 32)
    const LocalSmem L = local_smem<T>(N, ld, nrmax);
    double* us = (double*)(smem_raw + L.us);
    T* rowb = (T*)(smem_raw + L.rowb);
    T* patch = (T*)(smem_raw + L.patch);
    T* colb = (T*)(smem_raw + L.colb);
    int8_t* xs = (int8_t*)(smem_raw + L.xs);
    uint8_t* rp = (uint8_t*)(smem_raw + L.rp);
    __shared__ int s_b, s_nneg;
    __shared__ T s_f[2];
    __shared__ double s_maxr;
    for (int i = tid; i < N; i += nt) {
        us[i] = u[i];
        xs[i] = xl_g[i];
        rp[i] = replay ? replay[i] : 0;
    }
    if (tid == 0) {
        s_nneg = 0;
        s_maxr = 0.0;
    }
    for (int e = tid; e < 2 * nr; e += nt) {  // diagonals of the own rows into buffer 0
        const int s = e >= nr ? 1 : 0, r = r0 + e - s * nr;
        diag[(0 * 2 + s) * N + r] = (s ? Gd : Gu)[(long)r * ld + r];
    }
    // This thread's part of the own rows: the 16-byte column vectors v = vt, vt + vstep, ... of the
    // rows r = g, g + ng, ... of each spin.  With fewer vectors per row than threads the block splits
    // into ng = nt / nv row groups (one vector per thread, threads beyond ng nv idle); otherwise a
    // single group whose threads stride over the vectors.
    const int ng = nv >= nt ? 1 : nt / nv;
    const int g = nv >= nt ? 0 : tid / nv;
    const int vt = nv >= nt ? tid : tid - g * nv;
    const int vstep = nv >= nt ? nt : nv;
    unsigned int* ctr = &bar->count;
    unsigned int nbar = 0;  // grid barriers passed (thread 0)

    // flip constants in T (x = +1: index 0, x = -1: index 1), selected without local-memory indexing
    const T df00 = (T)sp.dflip[0][0], df01 = (T)sp.dflip[0][1], df10 = (T)sp.dflip[1][0],
            df11 = (T)sp.dflip[1][1], sf0 = (T)sp.sflip[0], sf1 = (T)sp.sflip[1];
    int n_acc = 0;
    int p = 0;      // next site to test (warp 0)
    int cur = 0;    // diagonal buffer the scan reads
    int pend = -1;  // own row whose new values wait in `patch`
    __syncthreads();
    for (;;) {
        // grid barrier (thread 0), then the scan for the next accept (warp 0); the other warps wait
        // at the block barrier below
        if (tid < 32) {
            int ok = 1;
            if (tid == 0) ok = grid_arrive_wait(ctr, (++nbar) * (unsigned int)nblk, err) ? 1 : 0;
            __syncwarp();
            ok = __shfl_sync(0xffffffffu, ok, 0);
            int bsel = ok ? N : -1;
            const T* d0 = diag + (cur * 2 + 0) * N;
            const T* d1 = diag + (cur * 2 + 1) * N;
            while (ok && p < N) {
                const int q = p + tid;
                bool acc = false;
                T R = T(0), rr0 = T(1), rr1 = T(1), del0 = df00, del1 = df10;
                if (q < N) {
                    // ratio arithmetic in the bulk precision T (no FP64 division on the FP32 path);
                    // the diagonals were written by other CTAs: read past L1
                    const int xi = xs[q] > 0 ? 0 : 1;
                    del0 = xi ? df01 : df00;
                    del1 = xi ? df11 : df10;
                    rr0 = T(1) + del0 * (T(1) - __ldcg(d0 + q));
                    rr1 = T(1) + del1 * (T(1) - __ldcg(d1 + q));
                    R = (xi ? sf1 : sf0) * rr0 * rr1;
                    acc = replay ? (rp[q] != 0) : (us[q] < (double)fabs(R));
                    if (!isfinite(R)) {
                        if (b == 0) set_err(err, DEV_NUMERIC);
                        acc = false;
                    }
                }
                const unsigned ball = __ballot_sync(0xffffffffu, acc);
                const int first = ball ? __ffs(ball) - 1 : 32;
                if (b == 0 && q < N && tid <= first) {
                    so.dec[q] = (tid == first) ? 1 : 0;
                    so.ratio[q] = (double)R;
                }
                if (tid == first) {
                    s_f[0] = del0 / rr0;
                    s_f[1] = del1 / rr1;
                    if (b == 0) {
                        xl_g[q] = (int8_t)(-xs[q]);
                        if (R < T(0)) s_nneg += 1;
                        s_maxr = fmax(s_maxr, (double)fabs(R));
                    }
                }
                __syncwarp();
                if (first < 32) {
                    bsel = p + first;
                    p = bsel + 1;
                    break;
                }
                p += 32;
            }
            if (tid == 0) s_b = bsel;
        }
        __syncthreads();
        const int bs = s_b;
        if (bs < 0) return;  // a bounded wait expired, or another CTA recorded an error
        if (pend >= 0) {     // every CTA has read row pend in the previous phase: store its new values
            for (int e = tid; e < 2 * nv; e += nt) {
                const int s = e >= nv ? 1 : 0, v = e - s * nv;
                *(V*)((s ? Gd : Gu) + (long)pend * ld + (long)v * VW) = *(const V*)(patch + (long)s * ld + (long)v * VW);
            }
        }
        if (bs >= N) break;
        ++n_acc;
        // row b of both spins (e_b^T - G[b, :], zero beyond N; written by another CTA: read past L1)
        // and column b of the own rows (row pend from `patch`, whose store above may be in flight)
        for (int e = tid; e < 2 * nv; e += nt) {
            const int s = e >= nv ? 1 : 0, v = e - s * nv;
            T gv[VW];
            *(V*)gv = __ldcg((const V*)((s ? Gd : Gu) + (long)bs * ld + (long)v * VW));
            T* o = rowb + (long)s * ld + (long)v * VW;
#pragma unroll
            for (int l = 0; l < VW; ++l) {
                const int c = v * VW + l;
                o[l] = c < N ? ((c == bs ? T(1) : T(0)) - gv[l]) : T(0);
            }
        }
        for (int e = tid; e < 2 * nr; e += nt) {
            const int s = e >= nr ? 1 : 0, r = e - s * nr;
            colb[s * nrmax + r] = (r0 + r == pend) ? patch[(long)s * ld + bs] : (s ? Gd : Gu)[(long)(r0 + r) * ld + bs];
        }
        pend = -1;
        __syncthreads();
        // G_s[r, :] += (-f_s G_s[r, b]) (e_b^T - G_s[b, :]) on the own rows: 16-byte accesses, all
        // LocalUnroll<T>::U loads of a thread issued before its stores.  The owner's row b goes to `patch`.
        const T nf0 = -s_f[0], nf1 = -s_f[1];
        constexpr int U = LocalUnroll<T>::U;
        for (int v = vt; g < ng && v < nv; v += vstep) {
            for (int sp_ = 0; sp_ < 2; ++sp_) {
                const V rv = *(const V*)(rowb + (long)sp_ * ld + (long)v * VW);  // e_b^T - G[b, :] here
                const T nf = sp_ ? nf1 : nf0;
                const T* cb = colb + sp_ * nrmax;
                T* base = (sp_ ? Gd : Gu) + (long)r0 * ld + (long)v * VW;
                T* pb = patch + (long)sp_ * ld + (long)v * VW;
                for (int r = g; r < nr; r += ng * U) {
                    V gv[U];
#pragma unroll
                    for (int q = 0; q < U; ++q) {
                        const int rr = r + q * ng;
                        if (rr < nr) gv[q] = *(const V*)(base + (long)rr * ld);
                    }
#pragma unroll
                    for (int q = 0; q < U; ++q) {
                        const int rr = r + q * ng;
                        if (rr < nr) {
                            vfma_rank1<T>(gv[q], nf * cb[rr], rv);
                            *(V*)((r0 + rr == bs) ? pb : base + (long)rr * ld) = gv[q];
                        }
                    }
                }
            }
        }
        // the new diagonals of the own rows (the same fused multiply-add as the element of G)
        for (int e = tid; e < 2 * nr; e += nt) {
            const int s = e >= nr ? 1 : 0, r = e - s * nr, gr = r0 + r;
            const T a = (s ? nf1 : nf0) * colb[s * nrmax + r];
            diag[((cur ^ 1) * 2 + s) * N + gr] = fma(a, rowb[(long)s * ld + gr], diag[(cur * 2 + s) * N + gr]);
        }
        if (bs >= r0 && bs < r1) pend = bs;
        cur ^= 1;
        __syncthreads();  // every write of the CTA precedes thread 0's arrival at the next barrier
    }
    if (b == 0 && tid == 0) {
        if (so.sign && (s_nneg & 1)) *so.sign = -*so.sign;
        so.stats[0] += N;
        so.stats[1] += n_acc;
        so.stats[2] += n_acc;
        *so.maxr = fmax(*so.maxr, s_maxr);
    }
}

// Grid size of the local kernel: at most max_blocks CTAs (one per SM) and at least one row each.
template <typename T>
cudaError_t launch_local(cudaStream_t st, T* Gu, T* Gd, int8_t* xl, const double* u, const uint8_t* replay,
                         const SiteParams& sp, SliceOut so, T* colbuf, T* rowbuf, GridBar* bar, int* err,
                         int max_blocks) {
    (void)rowbuf;
    const int nblk = max_blocks < sp.N ? max_blocks : sp.N;
    if (nblk < 1) return cudaErrorInvalidValue;
    const int nrmax = (sp.N + nblk - 1) / nblk;
    const size_t shm = local_smem<T>(sp.N, sp.ld, nrmax).total;
    cudaError_t e = ensure_smem_attr((const void*)local_kernel<T>, shm);
    if (e != cudaSuccess) return e;
    SiteParams spc = sp;
    int nrm = nrmax;
    void* args[] = {&Gu, &Gd, &xl, &u, &replay, &spc, &so, &colbuf, &bar, &err, &nrm};
    count_launch();
    return cudaLaunchCooperativeKernel((void*)local_kernel<T>, dim3(nblk), dim3(LOCAL_THREADS), args, shm, st);
}
// ---------------------------------------------------------------------------
// window chain: delayed (MODE 1) and block force-bias (MODE 2)
// ---------------------------------------------------------------------------
template <typename T> struct WinCap;
template <> struct WinCap<float> { static constexpr int NW = 128; };
template <> struct WinCap<double> { static constexpr int NW = 64; };
constexpr int NBMAX = 32;
constexpr int WIN_THREADS = 1024;  // 32 warps: the tail's W solve assigns 16 warps to each spin

template <typename T>
int window_max() { return WinCap<T>::NW; }
template int window_max<float>();
template int window_max<double>();

template <typename T>
__device__ __forceinline__ WindowBufs wb_walker(WindowBufs wb, int j, int N) {
    constexpr int NW = WinCap<T>::NW;
    wb.m += j;
    wb.idx += (size_t)j * NW;
    wb.dtot += (size_t)j * 2 * NW;
    wb.Wm = (T*)wb.Wm + (size_t)j * 2 * NW * NW;
    if (wb.Wx) wb.Wx = (T*)wb.Wx + (size_t)j * 2 * NW * NW;
    wb.X = (T*)wb.X + (size_t)j * 2 * N * NW;
    wb.Y = (T*)wb.Y + (size_t)j * 2 * NW * N;  // this walker's Yraw (the products follow all walkers' Yraw)
    return wb;
}

template <typename T>
static size_t window_smem(int n) {
    size_t P = (size_t)n + 1;
    size_t g = 2 * (size_t)n * P * sizeof(T);  // Gs[2][n][n+1]
    size_t s1 = 2 * (size_t)NBMAX * (NBMAX + 1) * sizeof(T);
    size_t vec = 4 * (size_t)n * sizeof(T) + 2 * (size_t)NBMAX * sizeof(T);  // staging vectors
    size_t misc = (size_t)n * (sizeof(int) + 2 * sizeof(double) + 1) + 8 * (size_t)NBMAX * sizeof(double) + 256;
    return g + s1 + vec + misc;
}

// G_s[r][c] += f_s * G_s[r][a] * G_s[a][c] for r, c in (a, n), both spins; 32 x 32 thread tiles.
template <typename T>
__device__ __forceinline__ void trailing_update(T* Gs, int n, int P, int a, T f0, T f1, int tid, int nt) {
    const int tx = tid & 31, ty = tid >> 5, ny = nt >> 5;
    for (int s = 0; s < 2; ++s) {
        T* Gb = Gs + (size_t)s * n * P;
        const T f = s ? f1 : f0;
        for (int r = a + 1 + ty; r < n; r += ny) {
            const T g = f * Gb[r * P + a];
            for (int c = a + 1 + tx; c < n; c += 32) Gb[r * P + c] = fma(g, Gb[a * P + c], Gb[r * P + c]);
        }
    }
}

// W = -F U1^{-1} L1^{-1} of the window from the frozen coefficients in the block (see the window
// kernel's tail); written to Wx[s][k][j] (pitch NW).  32 warps: spin = warp / 16, columns
// (warp % 16) * WCPW + c; lane l holds rows l + 32 r, r < RPL (RPL >= ceil(m / 32)).  The
// coefficient of the next step is fetched while the current one is applied, and the forward
// pass of a warp starts at its first column (identity columns are zero above the diagonal).
template <typename T, int RPL>
__device__ __forceinline__ void window_w_rpl(const T* Gs, int n, int P, const int* idx, const T (*fk)[WinCap<T>::NW],
                                             int m, T* Wx, int lane, int w) {
    constexpr int NW = WinCap<T>::NW, WCPW = NW / 16;
    const int s = w >> 4, j0 = (w & 15) * WCPW;
    if (j0 >= m) return;
    const T* Gb = Gs + (size_t)s * n * P;
    const T* fks = fk[s];
    int ik[RPL];
    T y[RPL][WCPW];
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
        const int k = lane + 32 * r;
        ik[r] = (k < m) ? idx[k] : 0;
#pragma unroll
        for (int c = 0; c < WCPW; ++c) y[r][c] = (k == j0 + c) ? T(1) : T(0);
    }
    // coefficient cf[r] = C[k][kp] f_kp of this lane's rows for step kp
    auto coef = [&](int kp, T* cf) {
        const int ikp = idx[kp];
        const T f = fks[kp];
#pragma unroll
        for (int r = 0; r < RPL; ++r) cf[r] = Gb[ik[r] * P + ikp] * f;
    };
    T cf[RPL], cfn[RPL];
    // forward: rows k > kp
    if (j0 + 1 < m) coef(j0, cf);
    for (int kp = j0; kp + 1 < m; ++kp) {
        if (kp + 2 < m) coef(kp + 1, cfn);
        const int ro = kp >> 5, lo = kp & 31;
        T v[WCPW];
#pragma unroll
        for (int c = 0; c < WCPW; ++c) {
            T src = y[0][c];
#pragma unroll
            for (int r = 1; r < RPL; ++r)
                if (ro == r) src = y[r][c];
            v[c] = __shfl_sync(0xffffffffu, src, lo);
        }
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
            const int k = lane + 32 * r;
            if (k > kp && k < m) {
#pragma unroll
                for (int c = 0; c < WCPW; ++c) y[r][c] -= cf[r] * v[c];
            }
        }
#pragma unroll
        for (int r = 0; r < RPL; ++r) cf[r] = cfn[r];
    }
    // backward: rows k < kp
    if (m >= 2) coef(m - 1, cf);
    for (int kp = m - 1; kp >= 1; --kp) {
        if (kp >= 2) coef(kp - 1, cfn);
        const int ro = kp >> 5, lo = kp & 31;
        T v[WCPW];
#pragma unroll
        for (int c = 0; c < WCPW; ++c) {
            T src = y[0][c];
#pragma unroll
            for (int r = 1; r < RPL; ++r)
                if (ro == r) src = y[r][c];
            v[c] = __shfl_sync(0xffffffffu, src, lo);
        }
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
            const int k = lane + 32 * r;
            if (k < kp) {
#pragma unroll
                for (int c = 0; c < WCPW; ++c) y[r][c] -= cf[r] * v[c];
            }
        }
#pragma unroll
        for (int r = 0; r < RPL; ++r) cf[r] = cfn[r];
    }
    T* Wd = Wx + (size_t)s * NW * NW;
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
        const int k = lane + 32 * r;
        if (k < m) {
            const T fkk = -fks[k];
#pragma unroll
            for (int c = 0; c < WCPW; ++c)
                if (j0 + c < m) Wd[k * NW + j0 + c] = fkk * y[r][c];
        }
    }
}

template <typename T>
__device__ __forceinline__ void window_w(const T* Gs, int n, int P, const int* idx, const T (*fk)[WinCap<T>::NW],
                                         int m, T* Wx, int tid) {
    constexpr int NW = WinCap<T>::NW;
    const int lane = tid & 31, w = tid >> 5;
    if (w >= 32) return;
    if (m <= 32) window_w_rpl<T, 1>(Gs, n, P, idx, fk, m, Wx, lane, w);
    else if (m <= 64) window_w_rpl<T, 2>(Gs, n, P, idx, fk, m, Wx, lane, w);
    else if (NW > 64 && m <= 96) window_w_rpl<T, (NW > 64 ? 3 : 2)>(Gs, n, P, idx, fk, m, Wx, lane, w);
    else window_w_rpl<T, NW / 32>(Gs, n, P, idx, fk, m, Wx, lane, w);
}

template <typename T, int MODE>
__global__ void __launch_bounds__(WIN_THREADS) window_kernel(const T* __restrict__ Gu0, int8_t* xl0, const double* u0,
                                                             const uint8_t* replay0, SiteParams sp, SliceOut so0,
                                                             int s0, int n, int nb, WindowBufs wb0, const T* blk0,
                                                             int* err, Batch bt) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int P = n + 1;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int N = sp.N;
    const long ld = sp.ld;
    // walker blockIdx.x of the group
    const int wk = blockIdx.x;
    const T* __restrict__ Gu = Gu0 + (size_t)wk * bt.gstride;
    const T* __restrict__ Gd = Gu + (size_t)N * ld;
    int8_t* xl_g = xl0 + (size_t)wk * bt.xstride;
    const double* u = u0 + (size_t)wk * 2 * N;
    const uint8_t* replay = replay0 ? replay0 + (size_t)wk * 2 * N : nullptr;
    const SliceOut so = so_walker(so0, wk, N);
    const WindowBufs wb = wb_walker<T>(wb0, wk, N);
    const T* blk = blk0 ? blk0 + (size_t)wk * 2 * WinCap<T>::NW * WinCap<T>::NW : nullptr;
    T* Gs = (T*)smem_raw;  // [2][n][P]
    size_t off = 2 * (size_t)n * P * sizeof(T);
    T* S1 = (T*)(smem_raw + off);  // [2][NBMAX][NBMAX+1]
    off += 2 * (size_t)NBMAX * (NBMAX + 1) * sizeof(T);
    T* stc = (T*)(smem_raw + off);  // staging: col[2][n], row[2][n]
    off += 4 * (size_t)n * sizeof(T);
    T* stb = (T*)(smem_raw + off);  // small staging [2][NBMAX]
    off += 2 * (size_t)NBMAX * sizeof(T);
    double* dl = (double*)(smem_raw + ((off + 7) & ~(size_t)7));  // [2][n]
    off = ((off + 7) & ~(size_t)7) + 2 * (size_t)n * sizeof(double);
    double* fb = (double*)(smem_raw + off);  // block-FB scalars [8][NBMAX]
    off += 8 * (size_t)NBMAX * sizeof(double);
    int* idx = (int*)(smem_raw + off);  // accepted positions [n]
    off += (size_t)n * sizeof(int);
    int8_t* xw = (int8_t*)(smem_raw + off);  // window fields [n]
    off += (size_t)n;
    __shared__ int s_m, s_nF;
    __shared__ int s_F[NBMAX];
    __shared__ double s_R;
    constexpr int NWC = WinCap<T>::NW;
    __shared__ T s_fk[2][NWC];  // f_k = -Delta_k / r_k of accept k, both spins

    const T* G[2] = {Gu, Gd};
    // the n x n diagonal block of both spins: from G, or from the corrected snapshot the
    // previous window's flush prepared (pitch NW, spin stride NW^2)
    {  // eight loads in flight per thread before their shared-memory stores
        constexpr int NL = 8;
        const int nn2 = n * n;
        for (int e0 = tid; e0 < 2 * nn2; e0 += NL * nt) {
            T v[NL];
#pragma unroll
            for (int q = 0; q < NL; ++q) {
                const int e = e0 + q * nt;
                if (e < 2 * nn2) {
                    const int s = e >= nn2 ? 1 : 0, rem = e - s * nn2, a = rem / n, c = rem - a * n;
                    v[q] = blk ? blk[((size_t)s * WinCap<T>::NW + a) * WinCap<T>::NW + c]
                               : G[s][(long)(s0 + a) * ld + (s0 + c)];
                }
            }
#pragma unroll
            for (int q = 0; q < NL; ++q) {
                const int e = e0 + q * nt;
                if (e < 2 * nn2) {
                    const int s = e >= nn2 ? 1 : 0, rem = e - s * nn2, a = rem / n, c = rem - a * n;
                    Gs[(s * n + a) * P + c] = v[q];
                }
            }
        }
    }
    for (int p = tid; p < n; p += nt) xw[p] = xl_g[s0 + p];
    // the window's site uniforms (and forced decisions) live in shared memory: the scan reads
    // them on its critical path
    // (in the bulk precision: the delayed scan compares them with ratios computed in T)
    __shared__ T s_u[WinCap<float>::NW];
    __shared__ uint8_t s_rep[WinCap<float>::NW];
    __shared__ T s_rat[WinCap<float>::NW];    // ratio of every decided site, written out after the scan
    __shared__ uint8_t s_dec[WinCap<float>::NW];
    __shared__ int s_nneg;                    // number of accepted negative ratios (sign parity)
    __shared__ T s_maxrT;
    for (int p = tid; p < n; p += nt) {
        s_u[p] = (T)u[s0 + p];
        s_rep[p] = replay ? replay[s0 + p] : 0;
    }
    if (tid == 0) {
        s_nneg = 0;
        s_maxrT = T(0);
    }
    __shared__ double c_dflip[2][2], c_dstrip[2][2], c_sflip[2];
    __shared__ T c_dflipT[2][2], c_sflipT[2];  // the same in T for the scan's critical path
    if (tid < 4) {
        c_dflip[tid >> 1][tid & 1] = sp.dflip[tid >> 1][tid & 1];
        c_dstrip[tid >> 1][tid & 1] = sp.dstrip[tid >> 1][tid & 1];
    }
    if (tid < 2) c_sflip[tid] = sp.sflip[tid];
    if (tid < 4) c_dflipT[tid >> 1][tid & 1] = (T)sp.dflip[tid >> 1][tid & 1];
    if (tid < 2) c_sflipT[tid] = (T)sp.sflip[tid];
    if (tid == 0) s_m = 0;
    __syncthreads();

    __shared__ double s_sign, s_maxr;  // walker sign and max |R|, owned by one thread at a time
    if (tid == 0) {
        s_sign = so.sign ? *so.sign : 1.0;
        s_maxr = 0.0;
    }
    __syncthreads();
    int n_prop = 0, n_acc = 0, n_flip = 0;

    __shared__ int8_t s_xch[WinCap<float>::NW];  // constrained path: the field chosen at each site
    __shared__ double s_cpl[2];                  // constrained path: sum ln N_i, sum ln |r_up r_dn|
    __shared__ int s_dead;
    if ((MODE == WIN_MODE_CP || MODE == WIN_MODE_CPB) && tid == 0) {
        s_cpl[0] = 0.0;
        s_cpl[1] = 0.0;
        s_dead = so.cp ? (so.cp[2] != 0.0) : 0;
    }
    __syncthreads();
    if (MODE == AFQMC_MODE_DELAYED || MODE == WIN_MODE_CP) {
        // Warp-serial Metropolis, one accept ahead of the block update: warp 0 keeps its own copy
        // of the two diagonals, applies each accept's effect on them itself, and scans the next
        // sites (32 at a time: a rejection leaves G unchanged, a ballot finds the first
        // acceptance) while warps 1..31 apply the previous accept's trailing update to the block.
        // Warp 0 reads only row a and column a of an accept a, which that accept's own update never
        // writes; the earlier updates that do write them are complete at the barrier before.  One
        // block barrier per accept.
        T* dg = stc;  // [2][n] warp 0's diagonals (the block-FB path's column / row staging, unused here)
        for (int q = tid; q < 2 * n; q += nt) dg[q] = Gs[((q / n) * n + q % n) * P + q % n];
        __shared__ int s_pend[2];
        __syncthreads();
        int pend = -1;  // accept whose block update the workers apply in this iteration
        int p = 0;      // next site to test (warp 0)
        int m_w0 = 0;   // accepts so far (warp 0)
        for (int it = 0;; ++it) {
            if (tid < 32) {
                if (pend >= 0) {  // the pending accept's effect on the later diagonals
                    const int a = idx[pend];
                    const T f0 = -s_fk[0][pend], f1 = -s_fk[1][pend];
                    for (int q = a + 1 + tid; q < n; q += 32) {
                        dg[q] = fma(f0 * Gs[(0 * n + q) * P + a], Gs[(0 * n + a) * P + q], dg[q]);
                        dg[n + q] = fma(f1 * Gs[(1 * n + q) * P + a], Gs[(1 * n + a) * P + q], dg[n + q]);
                    }
                    __syncwarp();
                }
                int next = -1;
                if (MODE == WIN_MODE_CP) {
                    // constrained-path heat bath (Sec. IV.D, Eq. ptilde): lane 0 draws the field of
                    // site p from lambda(x) = p(x) s(x) r_up(x) r_dn(x), r_s(x) = 1 + (e^{c_s x} - 1)
                    // (1 - G_pp), negative lambda clamped to zero (the constraint); the walker is
                    // removed when both vanish.  Every site is an accept of the delayed update.
                    if (p < n && !s_dead) {
                        if (tid == 0) {
                            const int q = p;
                            const T a0 = T(1) - dg[q], a1 = T(1) - dg[n + q];
                            const T rp0 = T(1) + c_dflipT[0][0] * a0, rp1 = T(1) + c_dflipT[1][0] * a1;
                            const T rm0 = T(1) + c_dflipT[0][1] * a0, rm1 = T(1) + c_dflipT[1][1] * a1;
                            const T lp = fmax(c_sflipT[0] * rp0 * rp1, T(0));
                            const T lm = fmax(c_sflipT[1] * rm0 * rm1, T(0));
                            const T nrm = lp + lm;
                            if (!(nrm > T(0)) || !isfinite(nrm)) {
                                s_dead = 1;
                                if (!isfinite(nrm)) set_err(err, DEV_NUMERIC);
                            } else {
                                const bool plus = replay ? (s_rep[q] != 0) : (s_u[q] < lp / nrm);
                                const int xi = plus ? 0 : 1;
                                const T r0 = plus ? rp0 : rm0, r1 = plus ? rp1 : rm1;
                                s_fk[0][m_w0] = -(c_dflipT[0][xi] / r0);
                                s_fk[1][m_w0] = -(c_dflipT[1][xi] / r1);
                                idx[m_w0] = q;
                                s_xch[m_w0] = plus ? 1 : -1;
                                s_dec[q] = plus ? 1 : 0;
                                s_rat[q] = nrm;
                                s_cpl[0] += log((double)nrm);
                                s_cpl[1] += log(fabs((double)r0 * (double)r1));
                                next = m_w0;
                            }
                        }
                        next = __shfl_sync(0xffffffffu, next, 0);
                        if (next >= 0) {
                            ++m_w0;
                            ++n_acc;
                            ++n_flip;
                        }
                        ++n_prop;
                        p = (next >= 0) ? p + 1 : n;
                    }
                }
                while (MODE == AFQMC_MODE_DELAYED && p < n) {
                    // ratio arithmetic in the bulk precision T (FP64 division on this critical path
                    // would cost thousands of cycles on GB300's FP64 pipe)
                    const int q = p + tid;
                    bool acc = false;
                    T R = T(0), rr0 = T(1), rr1 = T(1);
                    int xi = 0;
                    if (q < n) {
                        xi = xw[q] > 0 ? 0 : 1;
                        rr0 = T(1) + c_dflipT[0][xi] * (T(1) - dg[q]);
                        rr1 = T(1) + c_dflipT[1][xi] * (T(1) - dg[n + q]);
                        R = c_sflipT[xi] * rr0 * rr1;
                        acc = replay ? (s_rep[q] != 0) : (s_u[q] < fabs(R));
                        if (!isfinite(R)) {
                            acc = false;
                            set_err(err, DEV_NUMERIC);
                        }
                    }
                    const unsigned ball = __ballot_sync(0xffffffffu, acc);
                    const int first = ball ? __ffs(ball) - 1 : 32;
                    if (q < n && tid <= first) {
                        s_dec[q] = (tid == first) ? 1 : 0;
                        s_rat[q] = R;
                    }
                    if (tid == first) {
                        s_fk[0][m_w0] = -(c_dflipT[0][xi] / rr0);  // recursion factor f = -Delta / r
                        s_fk[1][m_w0] = -(c_dflipT[1][xi] / rr1);
                        idx[m_w0] = q;
                        if (R < T(0)) s_nneg = s_nneg + 1;
                        s_maxrT = fmax(s_maxrT, fabs(R));
                    }
                    if (first < 32) {
                        n_prop += first + 1;
                        p = p + first + 1;
                        next = m_w0++;
                        ++n_acc;
                        ++n_flip;
                        break;
                    }
                    n_prop += min(32, n - p);
                    p = min(n, p + 32);
                }
                if (tid == 0) {
                    s_pend[it & 1] = next;
                    s_m = m_w0;
                }
                __syncwarp();
            } else if (pend >= 0) {
                // warps 1..31: G[r][c] += f G[r][a] G[a][c] for r, c > a, both spins.  Rows and
                // columns <= a are never touched again, so the block keeps row a and column a as
                // they were when site a was accepted (the coefficients of the flush recursion).
                trailing_update(Gs, n, P, idx[pend], -s_fk[0][pend], -s_fk[1][pend], tid - 32, nt - 32);
            }
            __syncthreads();
            const int np = s_pend[it & 1];
            if (np < 0) break;  // nothing accepted in the rest of the window: the last update is applied
            pend = np;
        }
        // off the critical path: decisions, ratios, factors and the sign in their ABI types
        for (int q = tid; q < n; q += nt) {
            so.dec[s0 + q] = s_dec[q];
            so.ratio[s0 + q] = (double)s_rat[q];
        }
        for (int q = tid; q < s_m; q += nt) {
            dl[0 * n + q] = (double)s_fk[0][q];
            dl[1 * n + q] = (double)s_fk[1][q];
        }
        if (tid == 0) {
            if (s_nneg & 1) s_sign = -s_sign;
            s_maxr = fmax(s_maxr, (double)s_maxrT);
        }
        __syncthreads();
    } else if (MODE == WIN_MODE_CPB) {
        // ---- constrained-path block force bias (Sec. IV.D) ----
        // Per block S of nb sites (no field set yet): the force bias F_i of the current block's
        // diagonal (spin channel sum_s c_s A_s[i][i], charge channel lam (A_up + A_dn - 1)[i][i]),
        // each x_i from q(x_i) = e^{x_i F_i} / (2 cosh F_i); the weight factor
        // prod_i s(x_i) cosh F_i e^{-x_i F_i} prod_s det(1 + Delta_s A_s[S][S]) (the determinant as the
        // product of the sequential rank-1 ratios on a copy of the block); a factor <= 0 removes the
        // walker; the fields are then applied as accepts of the delayed update.
        __shared__ T s_phi2[2][NBMAX];
        __shared__ double s_rs2[2];
        T* strow = stc + 2 * n;  // [2][n]
        for (int p0 = 0; p0 < n && !s_dead; p0 += nb) {
            const int nbk = min(nb, n - p0);
            if (tid < nbk) {
                const int a = tid, i = s0 + p0 + a;
                const double a0 = 1.0 - (double)Gs[(0 * n + p0 + a) * P + p0 + a];
                const double a1 = 1.0 - (double)Gs[(1 * n + p0 + a) * P + p0 + a];
                const double F = sp.hs == AFQMC_HS_CHARGE_REAL ? sp.lam * (a0 + a1 - 1.0) : sp.c[0] * a0 + sp.c[1] * a1;
                const double lamp = 1.0 / (1.0 + exp(-2.0 * F));
                const int xp = replay ? (replay[i] ? 1 : -1) : (u[i] < lamp ? 1 : -1);
                so.dec[i] = xp > 0 ? 1 : 0;
                so.ratio[i] = lamp;
                fb[0 * NBMAX + a] = hs_log_scalar(sp, xp) + log(cosh(F)) - xp * F;
                s_xch[s_m + a] = (int8_t)xp;
            }
            for (int e = tid; e < 2 * nbk * nbk; e += nt) {
                int sp2 = e / (nbk * nbk), rem = e % (nbk * nbk), a = rem / nbk, c = rem % nbk;
                S1[(sp2 * NBMAX + a) * (NBMAX + 1) + c] = Gs[(sp2 * n + p0 + a) * P + p0 + c];
            }
            if (tid == 0) {
                s_rs2[0] = 1.0;
                s_rs2[1] = 1.0;
            }
            __syncthreads();
            const int mb = s_m;
            for (int q = 0; q < nbk; ++q) {
                for (int e = tid; e < 2 * nbk; e += nt) {
                    int sp2 = e / nbk, c = e % nbk;
                    T* Sb = S1 + sp2 * NBMAX * (NBMAX + 1);
                    stb[sp2 * NBMAX + c] = Sb[c * (NBMAX + 1) + q];
                    strow[sp2 * n + c] = (c == q ? T(1) : T(0)) - Sb[q * (NBMAX + 1) + c];
                }
                if (tid < 2) {
                    const int xi = s_xch[mb + q] > 0 ? 0 : 1;
                    const T dd = c_dflipT[tid][xi];
                    const T rr = T(1) + dd * (T(1) - S1[(tid * NBMAX + q) * (NBMAX + 1) + q]);
                    s_rs2[tid] *= (double)rr;
                    s_phi2[tid][q] = dd / rr;
                }
                __syncthreads();
                for (int e = tid; e < 2 * nbk * nbk; e += nt) {
                    int sp2 = e / (nbk * nbk), rem = e % (nbk * nbk), r = rem / nbk, c = rem % nbk;
                    T* Sb = S1 + sp2 * NBMAX * (NBMAX + 1);
                    Sb[r * (NBMAX + 1) + c] -= s_phi2[sp2][q] * stb[sp2 * NBMAX + r] * strow[sp2 * n + c];
                }
                __syncthreads();
            }
            if (tid == 0) {
                double lw = 0.0;
                for (int a = 0; a < nbk; ++a) lw += fb[0 * NBMAX + a];
                const double det = s_rs2[0] * s_rs2[1];
                const int blk = (s0 + p0) / nb;
                so.ratio[N + blk] = det;
                if (!(det > 0.0) || !isfinite(det)) {
                    s_dead = 1;
                    if (!isfinite(det)) set_err(err, DEV_NUMERIC);
                } else {
                    s_cpl[0] += lw + log(det);
                    s_cpl[1] += log(det);
                }
                so.dec[N + blk] = s_dead ? 0 : 1;
            }
            __syncthreads();
            if (s_dead) break;
            ++n_prop;
            ++n_acc;
            n_flip += nbk;
            for (int q = 0; q < nbk; ++q) {
                const int a = p0 + q, k = mb + q;
                if (tid == 0) {
                    idx[k] = a;
                    s_fk[0][k] = -s_phi2[0][q];
                    s_fk[1][k] = -s_phi2[1][q];
                    dl[0 * n + k] = -(double)s_phi2[0][q];
                    dl[1 * n + k] = -(double)s_phi2[1][q];
                }
                trailing_update(Gs, n, P, a, s_phi2[0][q], s_phi2[1][q], tid, nt);
                __syncthreads();
            }
            if (tid == 0) s_m = mb + nbk;
            __syncthreads();
        }
    } else {
        // ---- block force-bias (Sec. III.B) ----
        __shared__ T s_fs[2];
        __shared__ double s_rs[2];
        __shared__ int s_accb;
        __shared__ T s_phi[2][NBMAX];
        T* strow = stc + 2 * n;  // [2][n]
        for (int p0 = 0; p0 < n; p0 += nb) {
            const int nbk = min(nb, n - p0);
            const int blk = (s0 + p0) / nb;
            // (a) stripped force bias (Eq. BlkFrcBsTnew1): remove the block's fields one site at a time,
            //     each a rank-1 step G <- G - (d/r) G_{:,a} (e_a^T - G_{a,:}) with d = exp(-c x_a) - 1
            for (int e = tid; e < 2 * nbk * nbk; e += nt) {
                int s = e / (nbk * nbk), rem = e % (nbk * nbk), a = rem / nbk, c = rem % nbk;
                S1[(s * NBMAX + a) * (NBMAX + 1) + c] = Gs[(s * n + p0 + a) * P + p0 + c];
            }
            __syncthreads();
            for (int a = 0; a < nbk; ++a) {
                for (int e = tid; e < 2 * nbk; e += nt) {
                    int s = e / nbk, c = e % nbk;
                    T* Sb = S1 + s * NBMAX * (NBMAX + 1);
                    stb[s * NBMAX + c] = Sb[c * (NBMAX + 1) + a];                       // column a
                    strow[s * n + c] = (c == a ? T(1) : T(0)) - Sb[a * (NBMAX + 1) + c];  // e_a^T - row a
                }
                if (tid < 2) {
                    const int xi = xw[p0 + a] > 0 ? 0 : 1;
                    const T db = (T)c_dstrip[tid][xi];
                    const T rr = T(1) + db * (T(1) - S1[(tid * NBMAX + a) * (NBMAX + 1) + a]);
                    s_fs[tid] = db / rr;
                }
                __syncthreads();
                for (int e = tid; e < 2 * nbk * nbk; e += nt) {
                    int s = e / (nbk * nbk), rem = e % (nbk * nbk), r = rem / nbk, c = rem % nbk;
                    T* Sb = S1 + s * NBMAX * (NBMAX + 1);
                    Sb[r * (NBMAX + 1) + c] -= s_fs[s] * stb[s * NBMAX + r] * strow[s * n + c];
                }
                __syncthreads();
            }
            // (b) proposals from lambda(x') = bbar(x') / sum bbar, bbar(x) = s(x) e^{x h}
            if (tid < nbk) {
                const int a = tid, i = s0 + p0 + a;
                const double nb0 = 1.0 - (double)S1[(0 * NBMAX + a) * (NBMAX + 1) + a];
                const double nb1 = 1.0 - (double)S1[(1 * NBMAX + a) * (NBMAX + 1) + a];
                const double h = sp.c[0] * nb0 + sp.c[1] * nb1;
                const double lp = hs_log_scalar(sp, +1) + h, lm = hs_log_scalar(sp, -1) - h;
                const double lamp = 1.0 / (1.0 + exp(lm - lp));
                const int x = xw[p0 + a];
                const int xp = replay ? (replay[i] ? 1 : -1) : (u[i] < lamp ? 1 : -1);
                so.dec[i] = xp > 0 ? 1 : 0;
                so.ratio[i] = lamp;
                double lpr = 0.0;
                if (xp != x) {
                    double lbx = hs_log_scalar(sp, x) + x * h, lbxp = hs_log_scalar(sp, xp) + xp * h;
                    lpr = (hs_log_scalar(sp, xp) - hs_log_scalar(sp, x)) + (lbx - lbxp);
                }
                fb[0 * NBMAX + a] = lpr;
                fb[1 * NBMAX + a] = (xp != x) ? 1.0 : 0.0;
            }
            __syncthreads();
            if (tid == 0) {
                int nF = 0;
                double lpr = 0.0;
                for (int a = 0; a < nbk; ++a)
                    if (fb[1 * NBMAX + a] != 0.0) {
                        s_F[nF++] = a;
                        lpr += fb[0 * NBMAX + a];
                    }
                s_nF = nF;
                s_R = exp(lpr);
                s_rs[0] = 1.0;
                s_rs[1] = 1.0;
            }
            __syncthreads();
            const int nF = s_nF;
            ++n_prop;
            if (nF == 0) {
                if (tid == 0) {
                    so.dec[N + blk] = 1;
                    so.ratio[N + blk] = 1.0;
                }
                ++n_acc;
                continue;
            }
            // (c) det(1 + D_F A_FF) (Eq. BlkFrcBsTnew2's ratio) as the product of sequential rank-1 ratios
            for (int e = tid; e < 2 * nbk * nbk; e += nt) {
                int s = e / (nbk * nbk), rem = e % (nbk * nbk), a = rem / nbk, c = rem % nbk;
                S1[(s * NBMAX + a) * (NBMAX + 1) + c] = Gs[(s * n + p0 + a) * P + p0 + c];
            }
            __syncthreads();
            for (int q = 0; q < nF; ++q) {
                const int a = s_F[q];
                for (int e = tid; e < 2 * nbk; e += nt) {
                    int s = e / nbk, c = e % nbk;
                    T* Sb = S1 + s * NBMAX * (NBMAX + 1);
                    stb[s * NBMAX + c] = Sb[c * (NBMAX + 1) + a];
                    strow[s * n + c] = (c == a ? T(1) : T(0)) - Sb[a * (NBMAX + 1) + c];
                }
                if (tid < 2) {
                    const int xi = xw[p0 + a] > 0 ? 0 : 1;
                    const T dd = (T)c_dflip[tid][xi];
                    const T rr = T(1) + dd * (T(1) - S1[(tid * NBMAX + a) * (NBMAX + 1) + a]);
                    s_rs[tid] *= (double)rr;
                    s_phi[tid][q] = dd / rr;
                    fb[(4 + tid) * NBMAX + q] = (double)dd;
                }
                __syncthreads();
                for (int e = tid; e < 2 * nbk * nbk; e += nt) {
                    int s = e / (nbk * nbk), rem = e % (nbk * nbk), r = rem / nbk, c = rem % nbk;
                    T* Sb = S1 + s * NBMAX * (NBMAX + 1);
                    Sb[r * (NBMAX + 1) + c] -= s_phi[s][q] * stb[s * NBMAX + r] * strow[s * n + c];
                }
                __syncthreads();
            }
            if (tid == 0) {
                const double R = s_R * s_rs[0] * s_rs[1];
                bool acc = replay ? (replay[N + blk] != 0) : (u[N + blk] < fabs(R));
                if (!isfinite(R)) {
                    acc = false;
                    set_err(err, DEV_NUMERIC);
                }
                so.dec[N + blk] = acc ? 1 : 0;
                so.ratio[N + blk] = R;
                s_accb = acc ? 1 : 0;
                if (acc) {
                    if (R < 0) s_sign = -s_sign;
                    s_maxr = fmax(s_maxr, fabs(R));
                }
            }
            __syncthreads();
            if (!s_accb) continue;
            ++n_acc;
            n_flip += nF;
            // (d) apply the flips in increasing site order, each as the trailing rank-1 step of the
            //     delayed update (rows / columns after the flipped site): the same product of
            //     rank-1 factors as Eq. BlkFrcBsTnew2, and the frozen rows / columns feed the flush
            const int mb = s_m;
            for (int q = 0; q < nF; ++q) {
                const int a = p0 + s_F[q], k = mb + q;
                if (tid == 0) {
                    idx[k] = a;
                    s_fk[0][k] = -s_phi[0][q];
                    s_fk[1][k] = -s_phi[1][q];
                    dl[0 * n + k] = -(double)s_phi[0][q];
                    dl[1 * n + k] = -(double)s_phi[1][q];
                    xw[a] = (int8_t)(-xw[a]);
                }
                trailing_update(Gs, n, P, a, s_phi[0][q], s_phi[1][q], tid, nt);
                __syncthreads();
            }
            if (tid == 0) s_m = mb + nF;
            __syncthreads();
        }
    }
    __syncthreads();
    const int m = s_m;
    if (MODE == AFQMC_MODE_DELAYED) {  // apply the accepted flips (deferred: xw[p] was read by every thread)
        for (int q = tid; q < m; q += nt) xw[idx[q]] = (int8_t)(-xw[idx[q]]);
        __syncthreads();
    }
    if (MODE == WIN_MODE_CP || MODE == WIN_MODE_CPB) {  // the chosen fields, and the walker's weight factors
        for (int q = tid; q < m; q += nt) xw[idx[q]] = s_xch[q];
        if (tid == 0 && so.cp) {
            so.cp[0] += s_cpl[0];
            so.cp[1] += s_cpl[1];
            if (s_dead) so.cp[2] = 1.0;
        }
        __syncthreads();
    }
    for (int p = tid; p < n; p += nt) xl_g[s0 + p] = xw[p];
    for (int q = tid; q < m; q += nt) {
        wb.idx[q] = s0 + idx[q];
        wb.dtot[q] = dl[q];
        wb.dtot[WinCap<T>::NW + q] = dl[n + q];
    }
    // The window's update matrix W (Eq. DelayRgenk in G form).  With C[k][k'] = Gs[idx[k]][idx[k']]
    // the block entries frozen at acceptance time (rows and columns at or before an accepted site
    // are never touched again), f_k = -Delta_k / r_k, L1 = I + Cl F and U1 = I + Cu F (Cl, Cu the
    // strictly lower / upper parts of C, F = diag f), the delayed-update recursions give
    // W = -F U1^{-1} L1^{-1}: per column of the identity a forward and a backward substitution,
    //   y_k = b_k - sum_{k'<k} C[k][k'] f_k' y_k',   z_k = y_k - sum_{k'>k} C[k][k'] f_k' z_k',
    //   W_k = -f_k z_k.
    // Each warp owns WCPW columns of one spin in registers (lane l holds rows l, l + 32, ...) and
    // broadcasts the finished row of every step with a shuffle: no block-wide barrier per step.
    window_w<T>(Gs, n, P, idx, s_fk, m, (T*)wb.Wx, tid);
    if (tid == 0) {
        *wb.m = m;
        if (so.sign) *so.sign = s_sign;
        so.stats[0] += n_prop;
        so.stats[1] += n_acc;
        so.stats[2] += n_flip;
        so.stats[3] += (m > 0) ? 1 : 0;
        *so.maxr = fmax(*so.maxr, s_maxr);
    }
}

template <typename T>
cudaError_t launch_window_chain(cudaStream_t st, int mode, const T* Gu, const T* Gd, int8_t* xl,
                                const double* u, const uint8_t* replay, const SiteParams& sp, SliceOut so,
                                int s0, int n, int nb, WindowBufs wb, const T* blk, int* err, Batch bt) {
    (void)Gd;  // spin down follows spin up (N x ld) in every walker's G
    size_t shm = window_smem<T>(n);
    auto kfn = (mode == AFQMC_MODE_DELAYED) ? (const void*)window_kernel<T, AFQMC_MODE_DELAYED>
               : (mode == WIN_MODE_CP)     ? (const void*)window_kernel<T, WIN_MODE_CP>
               : (mode == WIN_MODE_CPB)    ? (const void*)window_kernel<T, WIN_MODE_CPB>
                                            : (const void*)window_kernel<T, AFQMC_MODE_BLOCKFB>;
    {
        cudaError_t e = ensure_smem_attr(kfn, window_smem<T>(WinCap<T>::NW));
        if (e != cudaSuccess) return e;
    }
    if (bt.nwk < 1) bt.nwk = 1;
    count_launch();
    if (mode == AFQMC_MODE_DELAYED)
        window_kernel<T, AFQMC_MODE_DELAYED><<<bt.nwk, WIN_THREADS, shm, st>>>(Gu, xl, u, replay, sp, so, s0, n, nb,
                                                                              wb, blk, err, bt);
    else if (mode == WIN_MODE_CP)
        window_kernel<T, WIN_MODE_CP><<<bt.nwk, WIN_THREADS, shm, st>>>(Gu, xl, u, replay, sp, so, s0, n, nb, wb,
                                                                       blk, err, bt);
    else if (mode == WIN_MODE_CPB)
        window_kernel<T, WIN_MODE_CPB><<<bt.nwk, WIN_THREADS, shm, st>>>(Gu, xl, u, replay, sp, so, s0, n, nb, wb,
                                                                        blk, err, bt);
    else
        window_kernel<T, AFQMC_MODE_BLOCKFB><<<bt.nwk, WIN_THREADS, shm, st>>>(Gu, xl, u, replay, sp, so, s0, n, nb,
                                                                              wb, blk, err, bt);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// flush: X = G[:, I], Yraw = E_I^T - G[I, :], Y = W Yraw, G <- G - X Y
// ---------------------------------------------------------------------------
template <typename T>
__global__ void gather_kernel(const T* __restrict__ Gu0, long ld, int N, WindowBufs wb0, int NW, long gstride,
                              long sstride) {
    const int wk = blockIdx.z;
    const WindowBufs wb = wb_walker<T>(wb0, wk, N);
    const int m = *wb.m;
    const int s = blockIdx.y;
    const T* G = Gu0 + (size_t)wk * gstride + (long)s * sstride;
    T* X = (T*)wb.X + (size_t)s * N * NW;
    T* Y = (T*)wb.Y + (size_t)s * NW * N;  // Yraw here; the product with W comes after
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * N; e += gridDim.x * blockDim.x) {
        int a = e / N, j = e % N;
        int I = wb.idx[a];
        Y[(size_t)a * N + j] = (j == I ? T(1) : T(0)) - G[(long)I * ld + j];
        int r = e / m, q = e % m;  // X row r, column q (coalesced over q is poor; rows are short)
        X[(size_t)r * NW + q] = G[(long)r * ld + wb.idx[q]];
    }
}

template <typename T>
cudaError_t launch_flush(cudaStream_t st, T* Gu, T* Gd, const SiteParams& sp, WindowBufs wb, int nw) {
    const int N = sp.N;
    const int NWC = WinCap<T>::NW;
    count_launch();
    gather_kernel<T><<<dim3(256, 2, 1), 256, 0, st>>>(Gu, sp.ld, N, wb, NWC, 0, (long)(Gd - Gu));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // Y <- W * Yraw  (rows >= m are never read); written into the X buffer's tail? use a separate pass:
    // compute in place is unsafe, so the product goes to the second half of the Y buffer.
    GemmArgs<T> g;
    g.M = nw; g.N = N; g.K = nw; g.Kdev = wb.m;
    g.A = (const T*)wb.Wm; g.lda = NWC; g.sA = (long)NWC * NWC;
    g.B = (const T*)wb.Y; g.ldb = N; g.sB = (long)NWC * N;
    g.C = (T*)wb.Y + (size_t)2 * NWC * N; g.ldc = N; g.sC = (long)NWC * N;
    g.alpha = T(1); g.beta = T(0);
    g.batch = 2;
    e = gemm<T>(st, g);
    if (e != cudaSuccess) return e;
    // G <- G - X Y
    GemmArgs<T> h;
    h.M = N; h.N = N; h.K = nw; h.Kdev = wb.m;
    h.A = (const T*)wb.X; h.lda = NWC; h.sA = (long)N * NWC;
    h.B = (const T*)wb.Y + (size_t)2 * NWC * N; h.ldb = N; h.sB = (long)NWC * N;
    h.C = Gu; h.ldc = sp.ld; h.sC = (long)(Gd - Gu);
    h.alpha = T(-1); h.beta = T(1);
    h.batch = 2;
    return gemm<T>(st, h);
}

template cudaError_t launch_local<float>(cudaStream_t, float*, float*, int8_t*, const double*, const uint8_t*,
                                         const SiteParams&, SliceOut, float*, float*, GridBar*, int*, int);
template cudaError_t launch_local<double>(cudaStream_t, double*, double*, int8_t*, const double*, const uint8_t*,
                                          const SiteParams&, SliceOut, double*, double*, GridBar*, int*, int);
template cudaError_t launch_window_chain<float>(cudaStream_t, int, const float*, const float*, int8_t*,
                                                const double*, const uint8_t*, const SiteParams&, SliceOut, int,
                                                int, int, WindowBufs, const float*, int*, Batch);
template cudaError_t launch_window_chain<double>(cudaStream_t, int, const double*, const double*, int8_t*,
                                                 const double*, const uint8_t*, const SiteParams&, SliceOut, int,
                                                 int, int, WindowBufs, const double*, int*, Batch);
// ---------------------------------------------------------------------------
// Pipelined flush of one window.
//
// The window kernel leaves W (m x m) in wb.Wm: the accumulated update of the window is
// G <- G - X W Yraw with X = G[:, I] and Yraw = E_I^T - G[I, :] (I the accepted sites).
//   * next_block_kernel (main stream, right after the window): the next window's n' x n' block
//     of G as it will be after this window's update, from three small gathers of G and two
//     small products in shared memory.  The next window starts from it at once.
//   * launch_flush_panels + launch_flush_gemm (flush stream): the panel gathers, Y' = W Yraw
//     and the rank-m product over all of G, overlapping the next window's decisions.
// ---------------------------------------------------------------------------

// snap[s][a][c] = G[sn + a][sn + c] - sum_k X[sn + a][k] Y'[k][sn + c], with X = G[:, I],
// Y' = W Yraw and Yraw[l][sn + c] = -G[I_l][sn + c] (the next window's sites are not in I): the
// block of the next window as it will be after this window's product.  Grid (row blocks of
// NB_ROWS, spin); each CTA forms (X_blk W) and then (X_blk W) Yraw_n for its rows.
constexpr int NB_ROWS = 4;
constexpr int NB_THREADS = 512;
// One CTA per (row block of NB_ROWS rows, spin, walker).  The gathers depend on the accepted sites,
// so the kernel takes two rounds of global loads: the sites, then W, Yraw_n, X_blk and the block's
// own rows of G, each mapped as warps over rows and lanes over columns (no index divisions, every
// load of a thread in flight before its shared-memory stores).  The two products split each
// output's sum over four consecutive lanes (strided partial sums, combined by shuffles), so every
// warp works on them.
template <typename T>
__global__ void __launch_bounds__(NB_THREADS) next_block_kernel(const T* __restrict__ Gu0, long ld, int N,
                                                                WindowBufs wb0, int sn, int nn, T* snap0,
                                                                long gstride) {
    constexpr int NW = WinCap<T>::NW, PP = NW + 1;
    const int wk = blockIdx.z;
    const WindowBufs wb = wb_walker<T>(wb0, wk, N);
    const int m = *wb.m;
    const int s = blockIdx.y, a0 = blockIdx.x * NB_ROWS, tid = threadIdx.x, nt = blockDim.x;
    const int ra = min(NB_ROWS, nn - a0);
    const T* G = Gu0 + (size_t)wk * gstride + (size_t)s * N * ld;
    T* out = snap0 + (size_t)wk * 2 * NW * NW + (size_t)s * NW * NW;
    extern __shared__ __align__(16) unsigned char nb_smem[];
    T* Ws = (T*)nb_smem;         // [m][PP]
    T* Ys = Ws + NW * PP;        // [m][PP]   Yraw_n
    T* Xs = Ys + NW * PP;        // [NB_ROWS][PP]
    T* Ts = Xs + NB_ROWS * PP;   // [NB_ROWS][PP]  X_blk W
    T* Gr = Ts + NB_ROWS * PP;   // [NB_ROWS][PP]  G[sn + a0 + a][sn + c]
    constexpr int CS = NW / 32;
    const int lane = tid & 31, warp = tid >> 5, nwarp = nt >> 5;
    __shared__ int sidx[NW];
    for (int q = tid; q < m; q += nt) sidx[q] = wb.idx[q];
    __syncthreads();
    const T* W = (const T*)wb.Wx + (size_t)s * NW * NW;
    // rows r of W and Yraw_n (r < m), of X_blk and of the block's own rows (r < ra) by warps,
    // columns by lanes
    for (int r = warp; r < m; r += nwarp) {
        const T* wrow = W + (size_t)r * NW;
        const T* grow = G + (long)sidx[r] * ld + sn;
        T vw[CS], vy[CS];
#pragma unroll
        for (int j = 0; j < CS; ++j) {
            const int c = lane + 32 * j;
            vw[j] = c < m ? wrow[c] : T(0);
            vy[j] = c < nn ? grow[c] : T(0);
        }
#pragma unroll
        for (int j = 0; j < CS; ++j) {
            const int c = lane + 32 * j;
            if (c < m) Ws[r * PP + c] = vw[j];
            if (c < nn) Ys[r * PP + c] = -vy[j];
        }
    }
    for (int a = warp; a < ra; a += nwarp) {
        const T* grow = G + (long)(sn + a0 + a) * ld;
        T vx[CS], vg[CS];
#pragma unroll
        for (int j = 0; j < CS; ++j) {
            const int k = lane + 32 * j;
            vx[j] = k < m ? grow[sidx[k]] : T(0);
            vg[j] = k < nn ? grow[sn + k] : T(0);
        }
#pragma unroll
        for (int j = 0; j < CS; ++j) {
            const int k = lane + 32 * j;
            if (k < m) Xs[a * PP + k] = vx[j];
            if (k < nn) Gr[a * PP + k] = vg[j];
        }
    }
    __syncthreads();
    // Ts = X_blk W: output (a, k) summed over l = part, part + 4, ... by lanes 4 g + part
    {
        const int nout = ra * m, iters = (4 * nout + nt - 1) / nt;
        for (int it = 0; it < iters; ++it) {
            const int o4 = tid + it * nt, g = o4 >> 2, part = o4 & 3;
            T acc = T(0);
            if (g < nout) {
                const int a = g / m, k = g - a * m;
                for (int l = part; l < m; l += 4) acc += Xs[a * PP + l] * Ws[l * PP + k];
            }
            acc += __shfl_xor_sync(0xffffffffu, acc, 1);
            acc += __shfl_xor_sync(0xffffffffu, acc, 2);
            if (g < nout && part == 0) Ts[(g / m) * PP + g % m] = acc;
        }
    }
    __syncthreads();
    // snap rows = G[rows, J] - Ts Yraw_n, the same split
    {
        const int nout = ra * nn, iters = (4 * nout + nt - 1) / nt;
        for (int it = 0; it < iters; ++it) {
            const int o4 = tid + it * nt, g = o4 >> 2, part = o4 & 3;
            T acc = T(0);
            int a = 0, c = 0;
            if (g < nout) {
                a = g / nn;
                c = g - a * nn;
                for (int l = part; l < m; l += 4) acc += Ts[a * PP + l] * Ys[l * PP + c];
            }
            acc += __shfl_xor_sync(0xffffffffu, acc, 1);
            acc += __shfl_xor_sync(0xffffffffu, acc, 2);
            if (g < nout && part == 0) out[(a0 + a) * NW + c] = Gr[a * PP + c] - acc;
        }
    }
}

template <typename T>
cudaError_t launch_next_block(cudaStream_t st, const T* Gu, const T* Gd, const SiteParams& sp, WindowBufs wb, int sn,
                              int nn, T* snap, Batch bt) {
    (void)Gd;
    constexpr int NW = WinCap<T>::NW;
    const size_t shm = (2 * (size_t)NW + 3 * NB_ROWS) * (NW + 1) * sizeof(T);
    {
        cudaError_t ea = ensure_smem_attr((const void*)next_block_kernel<T>, shm);
        if (ea != cudaSuccess) return ea;
    }
    count_launch();
    const int nbx = (nn + NB_ROWS - 1) / NB_ROWS;
    next_block_kernel<T><<<dim3(nbx, 2, bt.nwk), NB_THREADS, shm, st>>>(Gu, sp.ld, sp.N, wb, sn, nn, snap,
                                                                         bt.gstride);
    return cudaGetLastError();
}

// The panel gathers X = G[:, I], Yraw = E_I^T - G[I, :] and Y' = W Yraw of one window.
template <typename T>
cudaError_t launch_flush_panels(cudaStream_t sf, T* Gu, T* Gd, const SiteParams& sp, WindowBufs wb, int nw, Batch bt) {
    (void)Gd;
    constexpr int NW = WinCap<T>::NW;
    const int N = sp.N;
    count_launch();
    gather_kernel<T><<<dim3(256, 2, bt.nwk), 256, 0, sf>>>(Gu, sp.ld, N, wb, NW, bt.gstride, (long)N * sp.ld);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    GemmArgs<T> g;  // Y' = W Yraw, batch (walker, spin)
    g.M = nw; g.N = N; g.K = nw; g.Kdev = wb.m; g.kdiv = 2;
    g.A = (const T*)wb.Wx; g.lda = NW; g.sA = (long)NW * NW;
    g.B = (const T*)wb.Y; g.ldb = N; g.sB = (long)NW * N;
    g.C = (T*)wb.Y + (size_t)2 * bt.nwk * NW * N; g.ldc = N; g.sC = (long)NW * N;
    g.batch = 2 * bt.nwk;
    return gemm<T>(sf, g);
}

// G <- G - X Y' (the N x N rank-m product, after launch_flush_panels on the same stream).
template <typename T>
cudaError_t launch_flush_gemm(cudaStream_t sf, T* Gu, T* Gd, const SiteParams& sp, WindowBufs wb, int nw, Batch bt) {
    (void)Gd;
    constexpr int NW = WinCap<T>::NW;
    const int N = sp.N;
    GemmArgs<T> h;
    h.M = N; h.N = N; h.K = nw; h.Kdev = wb.m; h.kdiv = 2;
    h.A = (const T*)wb.X; h.lda = NW; h.sA = (long)N * NW;
    h.B = (const T*)wb.Y + (size_t)2 * bt.nwk * NW * N; h.ldb = N; h.sB = (long)NW * N;
    h.C = Gu; h.ldc = sp.ld; h.sC = (long)N * sp.ld;
    h.alpha = T(-1); h.beta = T(1);
    h.batch = 2 * bt.nwk;
    return gemm<T>(sf, h);
}
// ---------------------------------------------------------------------------
// T form (the paper's walker state: U_R, U_L, T = (U_L U_R)^{-1}; G = 1 - U_R T U_L)
// ---------------------------------------------------------------------------
// For every (walker, spin) z of the batch, with the window's accepted sites I (wb.idx, m = wb.m):
//   ULI[z][a][k] = UL[z][a][I_k]   (ns x m, pitch NW)      URI[z][k][a] = UR[z][I_k][a]   (m x ns, pitch ldr)
// UR: N x ns (leading dimension ldr), UL: ns x N (leading dimension N); batch strides sr, sl.
template <typename T>
__global__ void tform_gather_kernel(const T* __restrict__ UR, const T* __restrict__ UL, int N, int ns, long ldr,
                                    long sr, long sl, WindowBufs wb0, T* ULI, T* URI) {
    constexpr int NW = WinCap<T>::NW;
    const int z = blockIdx.y, wk = z >> 1;
    const WindowBufs wb = wb_walker<T>(wb0, wk, N);
    const int m = *wb.m;
    const T* ur = UR + (size_t)z * sr;
    const T* ul = UL + (size_t)z * sl;
    T* uli = ULI + (size_t)z * ns * NW;
    T* uri = URI + (size_t)z * NW * ldr;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * ns; e += gridDim.x * blockDim.x) {
        const int k = e / ns, a = e - k * ns;
        const int I = wb.idx[k];
        uri[(size_t)k * ldr + a] = ur[(size_t)I * ldr + a];
        uli[(size_t)a * NW + k] = ul[(size_t)a * N + I];
    }
}

// UR[z][I_k][:] *= exp(c_s (x' - x)) = exp(2 c_s x'_k) for the accepted sites (Eq. UpdateLTRMat: the
// row of the slice's B in the right factor takes the new field), x' the field the window kernel
// left in the slice (xl, batch stride xstride per walker).
template <typename T>
__global__ void tform_scale_rows_kernel(T* UR, int N, int ns, long ldr, long sr, WindowBufs wb0, const int8_t* xl,
                                        long xstride, double c0, double c1) {
    const int z = blockIdx.y, wk = z >> 1, s = z & 1;
    const WindowBufs wb = wb_walker<T>(wb0, wk, N);
    const int m = *wb.m;
    T* ur = UR + (size_t)z * sr;
    const int8_t* x = xl + (size_t)wk * xstride;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * ns; e += gridDim.x * blockDim.x) {
        const int k = e / ns, a = e - k * ns;
        const int I = wb.idx[k];
        const T f = (T)exp(2.0 * (s ? c1 : c0) * (double)x[I]);
        ur[(size_t)I * ldr + a] *= f;
    }
}

template <typename T>
cudaError_t launch_tform_gather(cudaStream_t st, const T* UR, const T* UL, int N, int ns, long ldr, long sr, long sl,
                                WindowBufs wb, T* ULI, T* URI, int nbatch) {
    count_launch();
    tform_gather_kernel<T><<<dim3(64, nbatch), 256, 0, st>>>(UR, UL, N, ns, ldr, sr, sl, wb, ULI, URI);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tform_scale_rows(cudaStream_t st, T* UR, int N, int ns, long ldr, long sr, WindowBufs wb,
                                    const int8_t* xl, long xstride, const double* c, int nbatch) {
    count_launch();
    tform_scale_rows_kernel<T><<<dim3(64, nbatch), 256, 0, st>>>(UR, N, ns, ldr, sr, wb, xl, xstride, c[0], c[1]);
    return cudaGetLastError();
}

template cudaError_t launch_tform_gather<float>(cudaStream_t, const float*, const float*, int, int, long, long, long,
                                                WindowBufs, float*, float*, int);
template cudaError_t launch_tform_gather<double>(cudaStream_t, const double*, const double*, int, int, long, long,
                                                 long, WindowBufs, double*, double*, int);
template cudaError_t launch_tform_scale_rows<float>(cudaStream_t, float*, int, int, long, long, WindowBufs,
                                                    const int8_t*, long, const double*, int);
template cudaError_t launch_tform_scale_rows<double>(cudaStream_t, double*, int, int, long, long, WindowBufs,
                                                     const int8_t*, long, const double*, int);
template cudaError_t launch_flush_panels<float>(cudaStream_t, float*, float*, const SiteParams&, WindowBufs, int,
                                               Batch);
template cudaError_t launch_flush_panels<double>(cudaStream_t, double*, double*, const SiteParams&, WindowBufs, int,
                                                Batch);
template cudaError_t launch_flush_gemm<float>(cudaStream_t, float*, float*, const SiteParams&, WindowBufs, int, Batch);
template cudaError_t launch_flush_gemm<double>(cudaStream_t, double*, double*, const SiteParams&, WindowBufs, int,
                                              Batch);
template cudaError_t launch_next_block<float>(cudaStream_t, const float*, const float*, const SiteParams&, WindowBufs,
                                              int, int, float*, Batch);
template cudaError_t launch_next_block<double>(cudaStream_t, const double*, const double*, const SiteParams&,
                                               WindowBufs, int, int, double*, Batch);
template cudaError_t launch_flush<float>(cudaStream_t, float*, float*, const SiteParams&, WindowBufs, int);
template cudaError_t launch_flush<double>(cudaStream_t, double*, double*, const SiteParams&, WindowBufs, int);

}  // namespace afq
