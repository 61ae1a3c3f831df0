// sepwrap.cuh -- the wrap G <- B G B^{-1} (Eqs. BlMat, GrFMat) with the separable propagator of
// the periodic L x L lattice.  The hopping along x and the hopping along y commute, so
// exp(-tau K) = Ex (x) Ex with the L x L chain factor Ex = exp(-tau K_1d), and on the site index
// i = x + L y the products E G and G E^{-1} are each two L-point passes over one index of G:
// 2 L N^2 multiply-adds per product instead of N^3.
//
// One tile of one matrix at a time:
//   side 0 (G <- (A (x) A) G, the row index):    the tile is all N rows x w columns;
//   side 1 (G <- G (A (x) A), the column index): the tile is h rows x all N columns.
// The untransformed index may have any extent C (N x C matrices on side 0, C x N on side 1), so
// the same tiles also move the factors U_R (N x N_sigma) and U_L (N_sigma x N) of the T form.
// The tile is staged in shared memory with the optional input scaling G_ij *= rs_in[i] cs_in[j],
// transformed by a pass along x into a second buffer and a pass along y back, and stored with the
// optional output scaling.  A is symmetric.  Each block owns its tile, so the update is in place.
// The passes are register-blocked (4 sites x 4 columns per thread, vector loads from shared
// memory) when L is a multiple of 4, which every configured lattice is.
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

#ifndef __CUDA_ARCH__
// Host build only: the number of vector accesses so far that would be misaligned on the device.
inline int& sep_misaligned_count() {
    static int n = 0;
    return n;
}
#endif

struct SepArgs {
    void* G = nullptr;       // batch matrices N x N, row-major with leading dimension ld, batch stride sG
    long ld = 0, sG = 0;
    int L = 0, N = 0, batch = 1;
    int C = 0;                  // extent of the untransformed index (0: N): side 0 takes N x C
                                // matrices (e.g. U_R, N x N_sigma), side 1 C x N ones (U_L)
    const double* A = nullptr;  // L x L one-dimensional factor (symmetric)
    int side = 0;               // 0: left product on the row index, 1: right product on the column index
    int w = 0;                  // tile width: columns (side 0) or rows (side 1); 0: the launcher's choice
    const void* rs_in = nullptr;   // nullable scale vectors, one entry per row (rs) or column (cs)
    const void* cs_in = nullptr;   // of the matrix -- N for the transformed index, C for the other --
    const void* rs_out = nullptr;  // applied before (in) or after (out) the product; matrix z uses
    const void* cs_out = nullptr;  // the vector at offset z * sv (sv >= the vector's length)
    long sv = 0;
    int circ = 0;  // A is circulant (A[x][x'] = A[0][(x' - x) mod L]), as the periodic chain's
                   // factors exp(-+tau K_1d) are: the line passes may then keep its first row in
                   // registers
};

// Shared memory of one tile: A, and the two N x w buffers.
template <typename T>
SEP_HD inline size_t sep_smem_bytes(int L, int N, int w) {
    return ((size_t)L * L + 2 * (size_t)N * w) * sizeof(T);
}

// Four consecutive elements, one vector access on the device (16-byte aligned: float4, or two
// double2).  The host build counts accesses that would be misaligned, since those fault on the
// device.
template <typename T>
SEP_HD inline void sep_ld4(const T* p, T v[4]) {
#ifdef __CUDA_ARCH__
    if constexpr (sizeof(T) == 4) {
        const float4 q = *(const float4*)p;
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
        const double2 q0 = *(const double2*)p, q1 = *((const double2*)p + 1);
        v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
    }
#else
    if (((size_t)p) % 16 != 0) ++sep_misaligned_count();
    for (int q = 0; q < 4; ++q) v[q] = p[q];
#endif
}
template <typename T>
SEP_HD inline void sep_st4(T* p, const T v[4]) {
#ifdef __CUDA_ARCH__
    if constexpr (sizeof(T) == 4) {
        *(float4*)p = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        *(double2*)p = make_double2(v[0], v[1]);
        *((double2*)p + 1) = make_double2(v[2], v[3]);
    }
#else
    if (((size_t)p) % 16 != 0) ++sep_misaligned_count();
    for (int q = 0; q < 4; ++q) p[q] = v[q];
#endif
}

// One L-point pass over the site index k = x + L y of the N x w buffer src (row k, column c),
// into dst: along x (dim 0) dst[(x, y)][c] = sum_x' A[x][x'] src[(x', y)][c]; along y (dim 1)
// dst[(x, y)][c] = sum_y' A[y][y'] src[(x, y')][c].  With L and w multiples of 4 each thread
// computes 4 sites x 4 columns from one vector load of A and one of src per step (A is
// symmetric, so its row is also its column); otherwise one output at a time.
template <typename T>
SEP_HD inline void sep_pass(const T* As, const T* src, T* dst, int L, int N, int w, int dim, int tid, int nt) {
    if (L % 4 == 0 && w % 4 == 0) {
        const int L4 = L / 4, w4 = w / 4, items = L * L4 * w4;
        for (int it = tid; it < items; it += nt) {
            const int cb = it % w4, rest = it / w4, ob = rest % L4, fixed = rest / L4;
            // dim 0: fixed = y, outputs x = 4 ob + r; dim 1: fixed = x, outputs y = 4 ob + r
            const long step = dim == 0 ? (long)w : (long)L * w;             // next x' (dim 0) or y' (dim 1)
            const long base = dim == 0 ? (long)L * fixed * w : (long)fixed * w;
            T acc[4][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}};
            for (int p = 0; p < L; ++p) {
                T a[4], b[4];
                sep_ld4(As + (size_t)p * L + 4 * ob, a);                // A[4 ob + r][p] = A[p][4 ob + r]
                sep_ld4(src + base + p * step + 4 * cb, b);             // src[site p][4 cb + j]
                for (int r = 0; r < 4; ++r)
                    for (int j = 0; j < 4; ++j) acc[r][j] += a[r] * b[j];
            }
            for (int r = 0; r < 4; ++r) {
                const int k = dim == 0 ? (4 * ob + r) + L * fixed : fixed + L * (4 * ob + r);
                sep_st4(dst + (size_t)k * w + 4 * cb, acc[r]);
            }
        }
        return;
    }
    for (int e = tid; e < N * w; e += nt) {
        const int k = e / w, c = e - k * w;
        const int y = k / L, x = k - y * L;
        T acc = 0;
        if (dim == 0) {
            const T* col = src + (size_t)(L * y) * w + c;
            for (int p = 0; p < L; ++p) acc += As[x * L + p] * col[(size_t)p * w];
        } else {
            const T* col = src + (size_t)x * w + c;
            for (int p = 0; p < L; ++p) acc += As[y * L + p] * col[(size_t)(L * p) * w];
        }
        dst[(size_t)k * w + c] = acc;
    }
}

// One tile (index t along the tiled dimension) of matrix z.  tid / nt: this thread and the
// block size; smem: sep_smem_bytes<T> bytes (16-byte aligned); sync(): a block-wide barrier.
// The tile is held as an N x w buffer (row k = the transformed index, column c): side 0 keeps
// G's columns o0 + c, side 1 holds G's rows o0 + c transposed, since (G A)[r][k] =
// sum_k' A[k][k'] G[r][k'] for a symmetric A.  Columns c >= wt of a ragged tile are zero-filled
// and never stored (each column is transformed on its own, so they do not reach the others).
template <typename T, typename Sync>
SEP_HD inline void sep_tile(const SepArgs& a, int t, int z, int tid, int nt, unsigned char* smem, Sync sync) {
    const int L = a.L, N = a.N, w = a.w;
    const int ext = a.C > 0 ? a.C : N;            // columns (side 0) or rows (side 1) of the matrix
    const int o0 = t * w;                         // first column (side 0) or row (side 1) of the tile
    const int wt = (ext - o0 < w) ? ext - o0 : w; // its width (the last tile may be ragged)
    if (wt <= 0) return;
    T* G = (T*)a.G + (size_t)z * a.sG;
    const T* ri = a.rs_in ? (const T*)a.rs_in + (size_t)z * a.sv : nullptr;
    const T* ci = a.cs_in ? (const T*)a.cs_in + (size_t)z * a.sv : nullptr;
    const T* ro = a.rs_out ? (const T*)a.rs_out + (size_t)z * a.sv : nullptr;
    const T* co = a.cs_out ? (const T*)a.cs_out + (size_t)z * a.sv : nullptr;
    T* As = (T*)smem;                 // [L][L]
    T* S0 = As + (size_t)L * L;       // [N][w]
    T* S1 = S0 + (size_t)N * w;       // [N][w]
    for (int e = tid; e < L * L; e += nt) As[e] = (T)a.A[e];
    // Side 1 moves four consecutive k of one row per thread (one 16-byte global access, a 2-way
    // shared-memory conflict on the transposed store) when the lattice allows it.
    const bool quad = a.side == 1 && L % 4 == 0 && a.ld % 4 == 0 && ((size_t)G) % 16 == 0;
    if (quad) {
        const int items = (N / 4) * w;
        for (int it = tid; it < items; it += nt) {
            const int c = it % w, k0 = 4 * (it / w);
            T v[4] = {0, 0, 0, 0};
            if (c < wt) {
                const int row = o0 + c;
                sep_ld4(G + (size_t)row * a.ld + k0, v);
                for (int q = 0; q < 4; ++q) {
                    if (ri) v[q] *= ri[row];
                    if (ci) v[q] *= ci[k0 + q];
                }
            }
            for (int q = 0; q < 4; ++q) S0[(size_t)(k0 + q) * w + c] = v[q];
        }
    } else {
        // consecutive e run along a row of G (coalesced); side 1 stores transposed
        for (int e = tid; e < N * w; e += nt) {
            int row, col, s, c;
            if (a.side == 0) {
                const int k = e / w;
                c = e - k * w;
                row = k; col = o0 + c; s = k * w + c;
            } else {
                c = e / N;
                const int k = e - c * N;
                row = o0 + c; col = k; s = k * w + c;
            }
            T v = 0;
            if (c < wt) {
                v = G[(size_t)row * a.ld + col];
                if (ri) v *= ri[row];
                if (ci) v *= ci[col];
            }
            S0[s] = v;
        }
    }
    sync();
    sep_pass<T>(As, S0, S1, L, N, w, 0, tid, nt);
    sync();
    sep_pass<T>(As, S1, S0, L, N, w, 1, tid, nt);
    sync();
    if (quad) {
        const int items = (N / 4) * wt;
        for (int it = tid; it < items; it += nt) {
            const int c = it % wt, k0 = 4 * (it / wt), row = o0 + c;
            T v[4];
            for (int q = 0; q < 4; ++q) {
                v[q] = S0[(size_t)(k0 + q) * w + c];
                if (ro) v[q] *= ro[row];
                if (co) v[q] *= co[k0 + q];
            }
            sep_st4(G + (size_t)row * a.ld + k0, v);
        }
        return;
    }
    for (int e = tid; e < N * wt; e += nt) {
        int row, col, s;
        if (a.side == 0) {
            const int k = e / wt, c = e - k * wt;
            row = k; col = o0 + c; s = k * w + c;
        } else {
            const int c = e / N, k = e - c * N;
            row = o0 + c; col = k; s = k * w + c;
        }
        T v = S0[s];
        if (ro) v *= ro[row];
        if (co) v *= co[col];
        G[(size_t)row * a.ld + col] = v;
    }
}

// ---------------------------------------------------------------------------------------------
// Line passes.  One launch applies A along ONE of the four lattice coordinates of G's two site
// indices (i = x + L y for the row, k = x' + L y' for the column):
//   axis 0: x of the row index     G[(x, y)][j]   <- sum_x'' A[x][x''] G[(x'', y)][j]
//   axis 1: y of the row index     G[(x, y)][j]   <- sum_y'' A[y][y''] G[(x, y'')][j]
//   axis 2: x of the column index  G[r][(x', y')] <- sum_x'' G[r][(x'', y')] A[x''][x']
//   axis 3: y of the column index  G[r][(x', y')] <- sum_y'' G[r][(x', y'')] A[y''][y']
// The L elements one pass mixes form a line; each thread owns one line, loads it into registers
// (all L loads in flight), forms the L outputs four at a time from one broadcast 16-byte
// shared-memory read of A per step (A is symmetric, so row p holds A[p][x..x+3] = A[x..x+3][p]),
// and writes them back in place (no other thread touches the line).  Consecutive threads take
// consecutive columns j (axes 0, 1), consecutive y' of one row (axis 2, each thread reading 4L
// contiguous bytes) or consecutive x' of one row (axis 3), so the warp's loads coalesce.  A side
// of the wrap is two launches (axes 0 and 1, or 2 and 3); the input scaling is applied by the
// first one on load and the output scaling by the second one on store.  LM (a multiple of 4,
// L <= LM) is the compile-time line length: A is zero-padded to LM x LM and the line's elements
// beyond L are zero.
struct SepLineArgs {
    void* G = nullptr;          // batch matrices R x C, row-major, leading dimension ld, batch stride sG
    long ld = 0, sG = 0;
    int L = 0, R = 0, C = 0, batch = 1;
    int axis = 0;
    const void* rs_in = nullptr, *cs_in = nullptr;    // as in SepArgs (matrix z: offset z * sv)
    const void* rs_out = nullptr, *cs_out = nullptr;
    long sv = 0;
    int circ = 0;  // as in SepArgs
};

// Lines of one matrix: L per column on the row axes, L per row on the column axes.
SEP_HD inline long sep_line_count(const SepLineArgs& a) {
    return a.axis < 2 ? (long)a.L * a.C : (long)a.R * a.L;
}

// The compile-time line length for a lattice side L (0: L > 64, no line kernel).
SEP_HD inline int sep_line_lm(int L) {
    const int lms[9] = {8, 12, 16, 20, 24, 32, 40, 48, 64};
    for (int q = 0; q < 9; ++q)
        if (L <= lms[q]) return lms[q];
    return 0;
}

// Line `line` (matrix z = line / lines per matrix) of a pass; As is A as LM x LM in T, zero-padded.
template <typename T, int LM>
SEP_HD inline void sep_line(const SepLineArgs& a, long line, const T* As) {
    const int L = a.L;
    const long nl = sep_line_count(a);
    const int z = (int)(line / nl);
    const long l = line - (long)z * nl;
    T* G = (T*)a.G + (size_t)z * a.sG;
    const T* ri = a.rs_in ? (const T*)a.rs_in + (size_t)z * a.sv : nullptr;
    const T* ci = a.cs_in ? (const T*)a.cs_in + (size_t)z * a.sv : nullptr;
    const T* ro = a.rs_out ? (const T*)a.rs_out + (size_t)z * a.sv : nullptr;
    const T* co = a.cs_out ? (const T*)a.cs_out + (size_t)z * a.sv : nullptr;
    // element p of the line: G[base + p * stride], row index i0 + p * di, column index k0 + p * dk
    long base, stride;
    int i0, di, k0, dk;
    if (a.axis < 2) {
        const int j = (int)(l % a.C), o = (int)(l / a.C);  // o = y (axis 0) or x (axis 1)
        i0 = a.axis == 0 ? L * o : o;
        di = a.axis == 0 ? 1 : L;
        k0 = j; dk = 0;
        base = (long)i0 * a.ld + j;
        stride = (long)di * a.ld;
    } else {
        const int o = (int)(l % L), r = (int)(l / L);      // o = y' (axis 2) or x' (axis 3)
        k0 = a.axis == 2 ? L * o : o;
        dk = a.axis == 2 ? 1 : L;
        i0 = r; di = 0;
        base = (long)r * a.ld + k0;
        stride = dk;
    }
    T* g = G + base;
    // the fixed factor of the scalings (the column on the row axes, the row on the column axes)
    T fin = 1, fout = 1;
    if (a.axis < 2) {
        if (ci) fin = ci[k0];
        if (co) fout = co[k0];
    } else {
        if (ri) fin = ri[i0];
        if (ro) fout = ro[i0];
    }
    const T* vin = a.axis < 2 ? ri : ci;    // the scalings along the line
    const T* vout = a.axis < 2 ? ro : co;
    const int vo = a.axis < 2 ? i0 : k0, vd = a.axis < 2 ? di : dk;
    T v[LM];
    const bool vec = stride == 1 && L % 4 == 0 && a.ld % 4 == 0 && a.sG % 4 == 0 && ((size_t)a.G) % 16 == 0;
    if (vec) {
#pragma unroll
        for (int p = 0; p < LM; p += 4) {
            if (p < L) {
                sep_ld4(g + p, v + p);
            } else {
                v[p] = v[p + 1] = v[p + 2] = v[p + 3] = 0;
            }
        }
    } else {
#pragma unroll
        for (int p = 0; p < LM; ++p) v[p] = p < L ? g[(long)p * stride] : (T)0;
    }
#pragma unroll
    for (int p = 0; p < LM; ++p) {
        if (p < L) v[p] *= vin ? fin * vin[vo + p * vd] : fin;
    }
#pragma unroll 1
    for (int q = 0; q < L; q += 4) {
        T acc[4] = {0, 0, 0, 0};
#pragma unroll
        for (int p = 0; p < LM; ++p) {
            T a4[4];
            sep_ld4(As + (size_t)p * LM + q, a4);
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[r] += a4[r] * v[p];
        }
        if (vec) {
            T o4[4];
            for (int r = 0; r < 4; ++r) o4[r] = acc[r] * (vout ? fout * vout[vo + (q + r) * vd] : fout);
            sep_st4(g + q, o4);
        } else {
            for (int r = 0; r < 4 && q + r < L; ++r)
                g[(long)(q + r) * stride] = acc[r] * (vout ? fout * vout[vo + (q + r) * vd] : fout);
        }
    }
}

// The same line for a circulant A of compile-time side L, given by its first row c[d] = A[0][d]
// (A[x][p] = c[(p - x) mod L]; A is symmetric, so the column passes use the same formula):
//   out[x] = sum_d c[d] v[(x + d) mod L].
// A symmetric circulant A has c[d] = c[L - d], so only c[0..L/2] is read (half the registers).
// c (the caller keeps it in registers across lines), the line and a chunk of H outputs are
// register operands, so the pass runs on the FMA pipes: L^2 multiply-adds per line and no memory
// access besides the line's own loads and stores.  H = L for lines up to 80 bytes, else L / 2
// rounded up to a multiple of 4 (fewer live registers, so two blocks fit per SM).
template <typename T, int L>
SEP_HD constexpr int sep_circ_chunk() {
    return sizeof(T) * L <= 80 ? L : ((L / 2 + 3) / 4) * 4;
}

template <typename T, int L>
SEP_HD inline void sep_line_circ(const SepLineArgs& a, long line, const T (&c)[L]) {
    const long nl = sep_line_count(a);
    const int z = (int)(line / nl);
    const long l = line - (long)z * nl;
    T* G = (T*)a.G + (size_t)z * a.sG;
    const T* ri = a.rs_in ? (const T*)a.rs_in + (size_t)z * a.sv : nullptr;
    const T* ci = a.cs_in ? (const T*)a.cs_in + (size_t)z * a.sv : nullptr;
    const T* ro = a.rs_out ? (const T*)a.rs_out + (size_t)z * a.sv : nullptr;
    const T* co = a.cs_out ? (const T*)a.cs_out + (size_t)z * a.sv : nullptr;
    long base, stride;
    int i0, di, k0, dk;
    if (a.axis < 2) {
        const int j = (int)(l % a.C), o = (int)(l / a.C);
        i0 = a.axis == 0 ? L * o : o;
        di = a.axis == 0 ? 1 : L;
        k0 = j; dk = 0;
        base = (long)i0 * a.ld + j;
        stride = (long)di * a.ld;
    } else {
        const int o = (int)(l % L), r = (int)(l / L);
        k0 = a.axis == 2 ? L * o : o;
        dk = a.axis == 2 ? 1 : L;
        i0 = r; di = 0;
        base = (long)r * a.ld + k0;
        stride = dk;
    }
    T* g = G + base;
    T fin = 1, fout = 1;
    if (a.axis < 2) {
        if (ci) fin = ci[k0];
        if (co) fout = co[k0];
    } else {
        if (ri) fin = ri[i0];
        if (ro) fout = ro[i0];
    }
    const T* vin = a.axis < 2 ? ri : ci;
    const T* vout = a.axis < 2 ? ro : co;
    const int vo = a.axis < 2 ? i0 : k0, vd = a.axis < 2 ? di : dk;
    T v[L];
    const bool vec = stride == 1 && L % 4 == 0 && a.ld % 4 == 0 && a.sG % 4 == 0 && ((size_t)a.G) % 16 == 0;
    if (vec) {
#pragma unroll
        for (int p = 0; p < L; p += 4) sep_ld4(g + p, v + p);
    } else {
#pragma unroll
        for (int p = 0; p < L; ++p) v[p] = g[(long)p * stride];
    }
#pragma unroll
    for (int p = 0; p < L; ++p) v[p] *= vin ? fin * vin[vo + p * vd] : fin;
    constexpr int H = sep_circ_chunk<T, L>();
#pragma unroll
    for (int x0 = 0; x0 < L; x0 += H) {
        T o[H];
#pragma unroll
        for (int x = 0; x < H; ++x) o[x] = 0;
#pragma unroll
        for (int d = 0; d < L; ++d)
#pragma unroll
            for (int x = 0; x < H; ++x)
                if (x0 + x < L) o[x] += c[d <= L / 2 ? d : L - d] * v[(x0 + x + d) % L];
#pragma unroll
        for (int x = 0; x < H; ++x)
            if (x0 + x < L) o[x] *= vout ? fout * vout[vo + (x0 + x) * vd] : fout;
        if (vec) {
#pragma unroll
            for (int x = 0; x < H; x += 4)
                if (x0 + x < L) sep_st4(g + x0 + x, o + x);
        } else {
#pragma unroll
            for (int x = 0; x < H; ++x)
                if (x0 + x < L) g[(long)(x0 + x) * stride] = o[x];
        }
    }
}

// The lattice sides with a circulant line kernel (FP64 up to 16: the line and its outputs stay in
// registers without spills); other sides take the LM kernel.
template <typename T>
SEP_HD inline bool sep_circ_side(int L) {
    switch (L) {
        case 4: case 6: case 8: case 12: case 16: return true;
        case 20: case 24: case 32: case 40: return sizeof(T) == 4;
        default: return false;
    }
}

// A (FP64, L x L) into the LM x LM shared-memory copy in T, zero-padded; thread tid of nt.
template <typename T>
SEP_HD inline void sep_line_load_A(const double* A, int L, int LM, T* As, int tid, int nt) {
    for (int e = tid; e < LM * LM; e += nt) {
        const int p = e / LM, q = e - p * LM;
        As[e] = (p < L && q < L) ? (T)A[p * L + q] : (T)0;
    }
}

// The two line passes of one side of a SepArgs (side 0: axes 0 then 1 on N x C matrices; side 1:
// axes 2 then 3 on C x N ones), with the input scaling on the first and the output scaling on
// the second.
inline void sep_line_passes(const SepArgs& s, SepLineArgs* p1, SepLineArgs* p2) {
    SepLineArgs a;
    a.G = s.G; a.ld = s.ld; a.sG = s.sG; a.L = s.L; a.batch = s.batch; a.sv = s.sv; a.circ = s.circ;
    const int ext = s.C > 0 ? s.C : s.N;
    a.R = s.side == 0 ? s.N : ext;
    a.C = s.side == 0 ? ext : s.N;
    *p1 = a;
    *p2 = a;
    p1->axis = s.side == 0 ? 0 : 2;
    p2->axis = s.side == 0 ? 1 : 3;
    p1->rs_in = s.rs_in; p1->cs_in = s.cs_in;
    p2->rs_out = s.rs_out; p2->cs_out = s.cs_out;
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
    a.circ = 1;  // Ex and Exi of the periodic chain
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
