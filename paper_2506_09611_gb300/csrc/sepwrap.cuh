// sepwrap.cuh -- the wrap G <- B G B^{-1} (Eqs. BlMat, GrFMat) with the separable propagator of
// the periodic L x L lattice.  The hopping along x and the hopping along y commute, so
// exp(-tau K) = Ex (x) Ex with the L x L chain factor Ex = exp(-tau K_1d), and on the site index
// i = x + L y the products E G and G E^{-1} are each two L-point passes over one index of G:
// 2 L N^2 multiply-adds per product instead of N^3.
//
// One tile of one matrix at a time:
//   side 0 (G <- (A (x) A) G, the row index):    the tile is all N rows x w columns;
//   side 1 (G <- G (A (x) A), the column index): the tile is h rows x all N columns.
// The tile is staged in shared memory with the optional input scaling G_ij *= rs_in[i] cs_in[j],
// transformed by a pass along x into a second buffer and a pass along y back, and stored with the
// optional output scaling.  A is symmetric.  Each block owns its tile, so the update is in place.
//
// The tile code is written once for the device kernel (sepwrap.cu) and for a host build that runs
// it serially (one "thread", barriers as no-ops), which lets the index arithmetic be checked on a
// CPU against an independent wrap.
#pragma once

#include <stddef.h>

#ifdef __CUDACC__
#define SEP_HD __host__ __device__
#else
#define SEP_HD
#endif

namespace afq {

struct SepArgs {
    void* G = nullptr;       // batch matrices N x N, row-major with leading dimension ld, batch stride sG
    long ld = 0, sG = 0;
    int L = 0, N = 0, batch = 1;
    const double* A = nullptr;  // L x L one-dimensional factor (symmetric)
    int side = 0;               // 0: left product on the row index, 1: right product on the column index
    int w = 16;                 // tile width: columns (side 0) or rows (side 1)
    const void* rs_in = nullptr;   // nullable, [batch] x N (stride sv): rows scaled before
    const void* cs_in = nullptr;   //                                     columns scaled before
    const void* rs_out = nullptr;  //                                     rows scaled after
    const void* cs_out = nullptr;  //                                     columns scaled after
    long sv = 0;
};

// Shared memory of one tile: A, and the two N x w buffers.
template <typename T>
SEP_HD inline size_t sep_smem_bytes(int L, int N, int w) {
    return ((size_t)L * L + 2 * (size_t)N * w) * sizeof(T);
}

// One tile (index t along the tiled dimension) of matrix z.  tid / nt: this thread and the
// block size; smem: sep_smem_bytes<T> bytes; sync(): a block-wide barrier.
template <typename T, typename Sync>
SEP_HD inline void sep_tile(const SepArgs& a, int t, int z, int tid, int nt, unsigned char* smem, Sync sync) {
    const int L = a.L, N = a.N, w = a.w;
    const int o0 = t * w;                         // first column (side 0) or row (side 1) of the tile
    const int wt = (N - o0 < w) ? N - o0 : w;     // its width (the last tile may be ragged)
    if (wt <= 0) return;
    T* G = (T*)a.G + (size_t)z * a.sG;
    const T* ri = a.rs_in ? (const T*)a.rs_in + (size_t)z * a.sv : nullptr;
    const T* ci = a.cs_in ? (const T*)a.cs_in + (size_t)z * a.sv : nullptr;
    const T* ro = a.rs_out ? (const T*)a.rs_out + (size_t)z * a.sv : nullptr;
    const T* co = a.cs_out ? (const T*)a.cs_out + (size_t)z * a.sv : nullptr;
    T* As = (T*)smem;                 // [L][L]
    T* S0 = As + (size_t)L * L;       // the tile; side 0: [N][w] (k, c), side 1: [w][N] (r, k)
    T* S1 = S0 + (size_t)N * w;       // after the pass along x
    for (int e = tid; e < L * L; e += nt) As[e] = (T)a.A[e];
    // stage: consecutive e run along a row of G (coalesced)
    for (int e = tid; e < N * wt; e += nt) {
        int row, col, s;
        if (a.side == 0) {
            const int k = e / wt, c = e - k * wt;
            row = k; col = o0 + c; s = k * w + c;
        } else {
            const int r = e / N, k = e - r * N;
            row = o0 + r; col = k; s = r * N + k;
        }
        T v = G[(size_t)row * a.ld + col];
        if (ri) v *= ri[row];
        if (ci) v *= ci[col];
        S0[s] = v;
    }
    sync();
    // pass along x: site k = x + L y takes sum_x' A[x][x'] S0[(x', y)]
    for (int e = tid; e < N * wt; e += nt) {
        int k, c;
        if (a.side == 0) { k = e / wt; c = e - k * wt; } else { c = e / N; k = e - c * N; }
        const int y = k / L, x = k - y * L;
        T acc = 0;
        if (a.side == 0) {
            const T* src = S0 + (size_t)(L * y) * w + c;
            for (int xp = 0; xp < L; ++xp) acc += As[x * L + xp] * src[(size_t)xp * w];
            S1[(size_t)k * w + c] = acc;
        } else {
            const T* src = S0 + (size_t)c * N + L * y;
            for (int xp = 0; xp < L; ++xp) acc += src[xp] * As[xp * L + x];
            S1[(size_t)c * N + k] = acc;
        }
    }
    sync();
    // pass along y: site k = x + L y takes sum_y' A[y][y'] S1[(x, y')]
    for (int e = tid; e < N * wt; e += nt) {
        int k, c;
        if (a.side == 0) { k = e / wt; c = e - k * wt; } else { c = e / N; k = e - c * N; }
        const int y = k / L, x = k - y * L;
        T acc = 0;
        if (a.side == 0) {
            const T* src = S1 + (size_t)x * w + c;
            for (int yp = 0; yp < L; ++yp) acc += As[y * L + yp] * src[(size_t)(L * yp) * w];
            S0[(size_t)k * w + c] = acc;
        } else {
            const T* src = S1 + (size_t)c * N + x;
            for (int yp = 0; yp < L; ++yp) acc += src[L * yp] * As[yp * L + y];
            S0[(size_t)c * N + k] = acc;
        }
    }
    sync();
    for (int e = tid; e < N * wt; e += nt) {
        int row, col, s;
        if (a.side == 0) {
            const int k = e / wt, c = e - k * wt;
            row = k; col = o0 + c; s = k * w + c;
        } else {
            const int r = e / N, k = e - r * N;
            row = o0 + r; col = k; s = r * N + k;
        }
        T v = S0[s];
        if (ro) v *= ro[row];
        if (co) v *= co[col];
        G[(size_t)row * a.ld + col] = v;
    }
}

// The two passes of the wrap for a batch of matrices G (N = L^2, leading dimension ld, batch
// stride sG), with Ex = exp(-dtau K_1d), Exi = exp(+dtau K_1d) and the field scales
// d = exp(c x), dinv = exp(-c x) ([batch][N], stride sv):
//   forward  (direction > 0): G <- D (E G) E^{-1} D^{-1}: side 0 with Ex, then side 1 with Exi
//                             storing rows times d and columns times dinv;
//   backward (direction < 0): G <- E^{-1} (D^{-1} G D E): side 1 with Ex loading rows times dinv
//                             and columns times d, then side 0 with Exi.
inline void sep_wrap_passes(int direction, void* G, long ld, long sG, int L, int batch, const double* Ex,
                            const double* Exi, const void* d, const void* dinv, long sv, SepArgs* a1, SepArgs* a2) {
    SepArgs a;
    a.G = G; a.ld = ld; a.sG = sG; a.L = L; a.N = L * L; a.batch = batch; a.sv = sv;
    *a1 = a;
    *a2 = a;
    if (direction > 0) {
        a1->side = 0; a1->A = Ex;
        a2->side = 1; a2->A = Exi; a2->rs_out = d; a2->cs_out = dinv;
    } else {
        a1->side = 1; a1->A = Ex; a1->rs_in = dinv; a1->cs_in = d;
        a2->side = 0; a2->A = Exi;
    }
}

}  // namespace afq
