// lu.cu -- blocked, partially pivoted LU in FP64 for the recompute (Sec. II.C, Eq. GrFMatNew).
//
// The re-orthonormalisation of the propagated factor U (N x Nsigma) and the solve
// (U_L U_R) Z = U_L both rest on an LU factorisation with partial pivoting.  GB300 runs FP64
// at a small fraction of its FP32 rate and every pivot is a grid-wide dependency, so the
// factorisation is blocked:
//   * a panel of LU_NB columns is factored by one thread-block cluster per matrix: each CTA
//     keeps its share of the rows in shared memory and the CTAs agree on every pivot through
//     distributed shared memory and one cluster barrier per column;
//   * the pivot rows' trailing part is finished inside the cluster (U12 = L11^{-1} A12);
//   * the trailing update A22 -= L21 U12 is an FP64 tiled product over the whole GPU.
// Rows are not swapped: a pivoted row is flagged, keeps its multipliers left of its pivot
// column and its U entries from there on, and perm[j] names the pivot row of column j.  Both
// spins go through every launch (two independent matrices).
#include <cooperative_groups.h>
#include <limits.h>

#include "internal.h"

namespace afq {
namespace cg = cooperative_groups;

__device__ __forceinline__ double* lu_A(const LuArgs& a, int b) {
    return a.A0 + (long)(b / a.ng) * a.wstride + (long)(b % a.ng) * a.sstride;
}

constexpr int LU_NB = 32;
constexpr int LU_NBP = LU_NB + 1;

// One cluster of CS CTAs per matrix (blockIdx.x / CS = matrix).  Factors columns
// [j0, j0 + nbk) over the rows not yet pivoted and finishes the pivot rows' columns
// [j0 + nbk, n).
// Pivot candidates compare |a| through the bit pattern of the double with the sign cleared:
// for finite non-negative doubles the integer order is the numeric order, and integer compares
// avoid the long FP64 latency on the pivot search's critical path.  Ties go to the lower row.
__device__ __forceinline__ unsigned long long lu_key(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffULL;
}
__device__ __forceinline__ void lu_pick(unsigned long long& k, int& r, double& x, unsigned long long ok, int orr,
                                        double ox) {
    if (ok > k || (ok == k && orr < r)) {
        k = ok;
        r = orr;
        x = ox;
    }
}

template <int CS>
__global__ void __launch_bounds__(256) lu_panel_kernel(LuArgs a, int j0, int nbk) {
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int mat = blockIdx.x / CS;
    double* A = lu_A(a, mat);
    int* perm = a.perm0 + (long)mat * a.pstride;
    int8_t* flag = a.flag0 + (long)mat * a.pstride;
    const int m = a.m, n = a.n;
    const long lda = a.lda;
    const int r0 = (int)((long)m * rank / CS), r1 = (int)((long)m * (rank + 1) / CS), nr = r1 - r0;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
    extern __shared__ __align__(16) double lu_smem[];
    double* Pn = lu_smem;                    // [nr][LU_NBP] own rows of the panel
    int8_t* fl = (int8_t*)(Pn + (size_t)nr * LU_NBP);
    // each warp's candidate of the step (by step parity): key, row, signed value
    __shared__ unsigned long long cand_k[2][8];
    __shared__ int cand_r[2][8];
    __shared__ double cand_x[2][8];
    __shared__ double L11[LU_NB][LU_NBP];    // pivot rows' panel values at their pivot step
    __shared__ int s_prow[LU_NB];            // pivot row of each step
    __shared__ int s_bad;
    __shared__ double s_pinv;
    for (int e = tid; e < nr * nbk; e += nt) {
        const int q = e / nbk, c = e - q * nbk;
        Pn[q * LU_NBP + c] = A[(long)(r0 + q) * lda + j0 + c];
    }
    for (int q = tid; q < nr; q += nt) fl[q] = flag[r0 + q];
    if (tid == 0) s_bad = 0;
    __syncthreads();
    // candidate of column 0 (later columns: found during the previous step's row update)
    unsigned long long bk = 0;
    int br = INT_MAX;
    double bx = 0.0;
    for (int q = tid; q < nr; q += nt)
        if (!fl[q]) {
            const double x = Pn[q * LU_NBP];
            lu_pick(bk, br, bx, lu_key(x), r0 + q, x);
        }
    for (int jj = 0; jj < nbk; ++jj) {
        const int par = jj & 1;
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
            const int orr = __shfl_xor_sync(0xffffffffu, br, o);
            const double ox = __shfl_xor_sync(0xffffffffu, bx, o);
            lu_pick(bk, br, bx, ok, orr, ox);
        }
        if (lane == 0) {
            cand_k[par][wid] = (br == INT_MAX) ? 0ULL : bk;
            cand_r[par][wid] = br;
            cand_x[par][wid] = bx;
        }
        cl.sync();  // every warp's candidate is published
        if (wid == 0) {
            // the winner over the cluster's 8 x CS warp candidates (4 per lane), then the pivot
            // row straight from the owner's shared memory (a pivoted row is never written again)
            unsigned long long k = 0;
            int r = INT_MAX;
            double x = 0.0;
#pragma unroll
            for (int t = 0; t < (8 * CS + 31) / 32; ++t) {
                const int slot = lane + 32 * t;
                if (slot < 8 * CS) {
                    const int cta = slot % CS, w = slot / CS;
                    const unsigned long long ok = *cl.map_shared_rank(&cand_k[par][w], cta);
                    const int orr = *cl.map_shared_rank(&cand_r[par][w], cta);
                    const double ox = *cl.map_shared_rank(&cand_x[par][w], cta);
                    if (orr != INT_MAX) lu_pick(k, r, x, ok, orr, ox);
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long ok = __shfl_xor_sync(0xffffffffu, k, o);
                const int orr = __shfl_xor_sync(0xffffffffu, r, o);
                const double ox = __shfl_xor_sync(0xffffffffu, x, o);
                lu_pick(k, r, x, ok, orr, ox);
            }
            const bool bad = (k == 0ULL) || (k >= 0x7ff0000000000000ULL) || r >= m;
            const int p = (r >= m) ? 0 : r;
            if (lane == jj) s_pinv = bad ? 0.0 : 1.0 / x;  // one FP64 division, overlapping the row read
            int own = (int)(((long)p * CS) / m);
            while (own > 0 && (int)((long)m * own / CS) > p) --own;
            while (own < CS - 1 && (int)((long)m * (own + 1) / CS) <= p) ++own;
            const int pr0 = (int)((long)m * own / CS);
            const double* prow = cl.map_shared_rank(Pn, own) + (size_t)(p - pr0) * LU_NBP;
            if (lane < nbk) L11[jj][lane] = prow[lane];
            if (lane == 0) {
                if (bad) s_bad = 1;
                s_prow[jj] = p;
                if (p >= r0 && p < r1) fl[p - r0] = 1;
                if (rank == 0) perm[j0 + jj] = p;
            }
        }
        __syncthreads();
        const double pinv = s_pinv;
        // own unpivoted rows: multiplier into column jj, rank-1 step on the later panel columns
        // (four independent multiply-adds at a time: FP64 latency is long on this part), and the
        // candidate for column jj + 1
        bk = 0;
        br = INT_MAX;
        bx = 0.0;
        for (int q = tid; q < nr; q += nt) {
            if (fl[q]) continue;
            double* __restrict__ row = Pn + q * LU_NBP;
            const double l = row[jj] * pinv;
            row[jj] = l;
            int c = jj + 1;
            for (; c + 3 < nbk; c += 4) {
                const double u0 = L11[jj][c], u1 = L11[jj][c + 1], u2 = L11[jj][c + 2], u3 = L11[jj][c + 3];
                const double v0 = row[c], v1 = row[c + 1], v2 = row[c + 2], v3 = row[c + 3];
                row[c] = v0 - l * u0;
                row[c + 1] = v1 - l * u1;
                row[c + 2] = v2 - l * u2;
                row[c + 3] = v3 - l * u3;
            }
            for (; c < nbk; ++c) row[c] -= l * L11[jj][c];
            if (jj + 1 < nbk) {
                const double x = row[jj + 1];
                lu_pick(bk, br, bx, lu_key(x), r0 + q, x);
            }
        }
    }
    cl.sync();  // no CTA leaves while another may still read its shared memory
    if (s_bad && tid == 0 && rank == 0) set_err(a.err, DEV_NUMERIC);
    for (int e = tid; e < nr * nbk; e += nt) {
        const int q = e / nbk, c = e - q * nbk;
        A[(long)(r0 + q) * lda + j0 + c] = Pn[q * LU_NBP + c];
    }
    for (int q = tid; q < nr; q += nt) flag[r0 + q] = fl[q];
    // U12 = L11^{-1} A12 on the pivot rows, columns dealt round-robin over the cluster's CTAs
    // (the FP64 work of a column is sequential, so every SM should get a share)
    for (int c = j0 + nbk + rank + CS * tid; c < n; c += CS * nt) {
        double x[LU_NB];
#pragma unroll
        for (int k = 0; k < LU_NB; ++k) x[k] = (k < nbk) ? A[(long)s_prow[k] * lda + c] : 0.0;
        // right-looking: each step's updates are independent of one another
#pragma unroll
        for (int kp = 0; kp + 1 < LU_NB; ++kp)
#pragma unroll
            for (int k = kp + 1; k < LU_NB; ++k)
                if (k < nbk) x[k] -= L11[k][kp] * x[kp];
#pragma unroll
        for (int k = 1; k < LU_NB; ++k)
            if (k < nbk) A[(long)s_prow[k] * lda + c] = x[k];
    }
}

// A[r][c] -= sum_k A[r][j0 + k] U12[k][c] for the unpivoted rows r and c in [j0 + nbk, n), with
// U12[k] the pivot row perm[j0 + k].  64 x 64 tiles, 4 x 4 outputs per thread; grid (row tiles,
// column tiles, matrix).
__global__ void __launch_bounds__(256) lu_update_kernel(LuArgs a, int j0, int nbk) {
    const int mat = blockIdx.z;
    double* A = lu_A(a, mat);
    const int* perm = a.perm0 + (long)mat * a.pstride;
    const int8_t* flag = a.flag0 + (long)mat * a.pstride;
    const long lda = a.lda;
    const int m = a.m, n = a.n;
    const int r0 = blockIdx.x * 64, c0 = j0 + nbk + blockIdx.y * 64;
    __shared__ double Ls[64][LU_NBP];
    __shared__ double Us[LU_NB][64 + 1];
    __shared__ int8_t fl[64];
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int q = tid; q < 64; q += nt) fl[q] = (r0 + q < m) ? flag[r0 + q] : 1;
    __syncthreads();
    for (int e = tid; e < 64 * LU_NB; e += nt) {
        const int q = e / LU_NB, k = e - q * LU_NB;
        Ls[q][k] = (k < nbk && !fl[q]) ? A[(long)(r0 + q) * lda + j0 + k] : 0.0;
    }
    for (int e = tid; e < LU_NB * 64; e += nt) {
        const int k = e >> 6, c = e & 63;
        Us[k][c] = (k < nbk && c0 + c < n) ? A[(long)perm[j0 + k] * lda + c0 + c] : 0.0;
    }
    __syncthreads();
    const int tx = tid & 15, ty = tid >> 4;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int k = 0; k < nbk; ++k) {
        double lv[4], uv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) lv[i] = Ls[ty + 16 * i][k];
#pragma unroll
        for (int j = 0; j < 4; ++j) uv[j] = Us[k][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] += lv[i] * uv[j];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int q = ty + 16 * i;
        if (fl[q]) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = c0 + tx + 16 * j;
            if (c < n) A[(long)(r0 + q) * lda + c] -= acc[i][j];
        }
    }
}

// Pivot rows of the factored tall matrix become unit rows: A[perm[j]][c] = (c == j) for c >= j,
// so A = P L (unit lower trapezoidal, rows in the original order) spans the same columns.
__global__ void lu_unit_rows_kernel(LuArgs a) {
    const int mat = blockIdx.y;
    double* A = lu_A(a, mat);
    const int* perm = a.perm0 + (long)mat * a.pstride;
    const int n = a.n;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < (long)n * n; e += (long)gridDim.x * blockDim.x) {
        const int j = (int)(e / n), c = (int)(e % n);
        if (c >= j) A[(long)perm[j] * a.lda + c] = (c == j) ? 1.0 : 0.0;
    }
}

// *sign_out *= the sign of the product of the pivots of every matrix (times each permutation's
// parity when `parity`): the sign of det(A) for square A.  One thread; visited holds m ints.
__global__ void lu_sign_kernel(LuArgs a, int parity, double* sign_out, int* visited) {
    const int wk = blockIdx.x * blockDim.x + threadIdx.x;  // one thread per walker
    if (wk * a.ng >= a.nmat) return;
    int* vis = visited + (size_t)wk * a.m;
    double sg = 1.0;
    for (int q = 0; q < a.ng; ++q) {
        const int mat = wk * a.ng + q;
        const double* A = lu_A(a, mat);
        const int* perm = a.perm0 + (long)mat * a.pstride;
        for (int j = 0; j < a.n; ++j)
            if (A[(long)perm[j] * a.lda + j] < 0.0) sg = -sg;
        if (parity) {
            for (int r = 0; r < a.m; ++r) vis[r] = 0;
            for (int r = 0; r < a.m; ++r) {
                if (vis[r]) continue;
                int len = 0, p = r;
                while (!vis[p]) {
                    vis[p] = 1;
                    p = perm[p];
                    ++len;
                }
                if ((len & 1) == 0) sg = -sg;
            }
        }
    }
    sign_out[wk] *= sg;
}

template <int CS>
static cudaError_t launch_panel(cudaStream_t st, const LuArgs& a, int j0, int nbk) {
    const int rpc = (a.m + CS - 1) / CS;
    const size_t shm = (size_t)rpc * LU_NBP * sizeof(double) + (size_t)rpc + 16;
    {
        cudaError_t e = ensure_smem_attr((const void*)lu_panel_kernel<CS>, 227 * 1024 - 16 * 1024);
        if (e != cudaSuccess) return e;
        if (CS > 8) {
            e = ensure_func_attr((const void*)lu_panel_kernel<CS>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (e != cudaSuccess) return e;
        }
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CS * a.nmat);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = shm;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    count_launch();
    return cudaLaunchKernelEx(&cfg, lu_panel_kernel<CS>, a, j0, nbk);
}

// Cluster size: enough CTAs per matrix that a panel step's FP64 work per SM stays small, few
// enough that all nmat clusters of a batch are resident together (about two CTAs per SM).
// Rows per CTA stay at or below 512 (shared memory); 16-CTA clusters are used only if two of
// them fit on the device at once (else 8).
static int lu_big_cluster(const LuArgs& a) {
    static int big = 0;
    if (big) return big;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(32);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = (size_t)((a.m + 15) / 16) * LU_NBP * sizeof(double) + (a.m + 15) / 16 + 16;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 16;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int ncl = 0;
    ensure_func_attr((const void*)lu_panel_kernel<16>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    ensure_smem_attr((const void*)lu_panel_kernel<16>, 227 * 1024 - 16 * 1024);
    if (cudaOccupancyMaxActiveClusters(&ncl, (void*)lu_panel_kernel<16>, &cfg) == cudaSuccess && ncl >= 2) big = 16;
    else big = 8;
    cudaGetLastError();
    return big;
}

static int lu_cluster_size(const LuArgs& a) {
    int nsm = 152, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int cs = 1;
    while (cs < 16 && (a.m + cs - 1) / cs > 64 && cs * a.nmat <= nsm) cs *= 2;  // spread rows
    while (cs < 16 && (a.m + cs - 1) / cs > 512) cs *= 2;                              // shared memory
    if (cs == 16) cs = lu_big_cluster(a);
    return cs;
}

cudaError_t launch_lu(cudaStream_t st, const LuArgs& a) {
    if (a.m < a.n || a.n < 1 || a.nmat < 1 || a.pstride < a.m) return cudaErrorInvalidValue;
    const int cs = lu_cluster_size(a);
    if ((a.m + cs - 1) / cs * (LU_NBP * sizeof(double) + 1) > 200 * 1024) return cudaErrorInvalidValue;
    cudaError_t e;
    if ((e = cudaMemsetAsync(a.flag0, 0, (size_t)(a.nmat - 1) * a.pstride + a.m, st)) != cudaSuccess) return e;
    for (int j0 = 0; j0 < a.n; j0 += LU_NB) {
        const int nbk = (a.n - j0 < LU_NB) ? a.n - j0 : LU_NB;
        switch (cs) {
            case 1: e = launch_panel<1>(st, a, j0, nbk); break;
            case 2: e = launch_panel<2>(st, a, j0, nbk); break;
            case 4: e = launch_panel<4>(st, a, j0, nbk); break;
            case 8: e = launch_panel<8>(st, a, j0, nbk); break;
            default: e = launch_panel<16>(st, a, j0, nbk); break;
        }
        if (e != cudaSuccess) return e;
        const int nc = a.n - j0 - nbk;
        if (nc > 0) {
            count_launch();
            lu_update_kernel<<<dim3((a.m + 63) / 64, (nc + 63) / 64, a.nmat), 256, 0, st>>>(a, j0, nbk);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

cudaError_t launch_lu_unit_rows(cudaStream_t st, const LuArgs& a) {
    count_launch();
    lu_unit_rows_kernel<<<dim3(256, a.nmat), 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_lu_sign(cudaStream_t st, const LuArgs& a, int parity, double* sign_out, int* visited) {
    if (!sign_out) return cudaSuccess;
    count_launch();
    const int nw = (a.nmat + a.ng - 1) / a.ng;
    lu_sign_kernel<<<(nw + 63) / 64, 64, 0, st>>>(a, parity, sign_out, visited);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Z = O^{-1} B for a factored square O (ns x ns, no-swap form: row perm[j] holds L[j][0..j)
// and U[j][j..ns)) and B (ns x N), both matrices of the batch:
//   forward  y_j = B[perm[j]] - sum_{k<j} L[j][k] y_k,
//   backward z_j = (y_j - sum_{k>j} U[j][k] z_k) / U[j][j],   Z[j] = z_j.
// The right-hand sides are independent: each CTA owns SV_COLS columns in shared memory and
// walks the rows in blocks of 32 (a product with the finished rows, then the 32 x 32 diagonal
// block column by column).  Grid (column blocks, matrix).
// ---------------------------------------------------------------------------
constexpr int SV_COLS = 10, SV_YP = SV_COLS + 1, SV_KB = 64;

__global__ void __launch_bounds__(256) lu_solve_kernel(SolveArgs a) {
    const int mat = blockIdx.y;
    const double* LU = a.LU0 + (long)mat * a.ostride;
    const int* perm = a.perm0 + (long)mat * a.pstride;
    const double* B = a.B0 + (long)(mat / a.ng) * a.wstride + (long)(mat % a.ng) * a.sstride;
    double* Z = a.Z0 + (long)mat * a.zstride;
    const int ns = a.ns, N = a.N;
    const long ldl = a.ldl, ldb = a.ldb ? a.ldb : N;
    const int c0 = blockIdx.x * SV_COLS, nc = min(SV_COLS, N - c0);
    const int tid = threadIdx.x, nt = blockDim.x;
    extern __shared__ __align__(16) double sv_smem[];
    double* y = sv_smem;                        // [ns][SV_YP]
    double* Lc = y + (size_t)ns * SV_YP;        // [32][SV_KB + 1]
    double* rinv = Lc + 32 * (SV_KB + 1);       // [ns]
    int* sp = (int*)(rinv + ns);                // [ns]
    for (int j = tid; j < ns; j += nt) sp[j] = perm[j];
    __syncthreads();
    const bool eye = a.eye != 0;
    for (int e = tid; e < ns * SV_COLS; e += nt) {
        const int j = e / SV_COLS, c = e - j * SV_COLS;
        y[j * SV_YP + c] = (c < nc) ? (eye ? (j == c0 + c ? 1.0 : 0.0) : B[(long)sp[j] * ldb + c0 + c]) : 0.0;
    }
    for (int j = tid; j < ns; j += nt) rinv[j] = 1.0 / LU[(long)sp[j] * ldl + j];
    __syncthreads();
    // forward substitution (unit lower L); with the pivot-ordered identity every y_j with j < c0
    // is zero in this block of columns, so the rows above c0 and their products are skipped
    const int j_first = eye ? c0 : 0;
    for (int J0 = (j_first / 32) * 32; J0 < ns; J0 += 32) {
        const int jb = min(32, ns - J0);
        for (int k0 = (j_first / SV_KB) * SV_KB; k0 < J0; k0 += SV_KB) {
            const int kb = min(SV_KB, J0 - k0);
            for (int e = tid; e < jb * SV_KB; e += nt) {
                const int r = e / SV_KB, k = e - r * SV_KB;
                Lc[r * (SV_KB + 1) + k] = (k < kb) ? LU[(long)sp[J0 + r] * ldl + k0 + k] : 0.0;
            }
            __syncthreads();
            for (int e = tid; e < jb * SV_COLS; e += nt) {
                const int r = e / SV_COLS, c = e - r * SV_COLS;
                double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;  // independent chains (FP64 latency)
                int k = 0;
                for (; k + 3 < kb; k += 4) {
                    a0 += Lc[r * (SV_KB + 1) + k] * y[(k0 + k) * SV_YP + c];
                    a1 += Lc[r * (SV_KB + 1) + k + 1] * y[(k0 + k + 1) * SV_YP + c];
                    a2 += Lc[r * (SV_KB + 1) + k + 2] * y[(k0 + k + 2) * SV_YP + c];
                    a3 += Lc[r * (SV_KB + 1) + k + 3] * y[(k0 + k + 3) * SV_YP + c];
                }
                for (; k < kb; ++k) a0 += Lc[r * (SV_KB + 1) + k] * y[(k0 + k) * SV_YP + c];
                y[(J0 + r) * SV_YP + c] -= (a0 + a1) + (a2 + a3);
            }
            __syncthreads();
        }
        for (int e = tid; e < jb * 32; e += nt) {
            const int r = e >> 5, k = e & 31;
            Lc[r * (SV_KB + 1) + k] = (k < jb) ? LU[(long)sp[J0 + r] * ldl + J0 + k] : 0.0;
        }
        __syncthreads();
        for (int rp = 0; rp + 1 < jb; ++rp) {  // diagonal block, right-looking
            for (int e = tid; e < (jb - rp - 1) * SV_COLS; e += nt) {
                const int r = rp + 1 + e / SV_COLS, c = e % SV_COLS;
                y[(J0 + r) * SV_YP + c] -= Lc[r * (SV_KB + 1) + rp] * y[(J0 + rp) * SV_YP + c];
            }
            __syncthreads();
        }
    }
    // backward substitution (U)
    const int nblk = (ns + 31) / 32;
    for (int bj = nblk - 1; bj >= 0; --bj) {
        const int J0 = bj * 32, jb = min(32, ns - J0), J1 = J0 + jb;
        for (int k0 = J1; k0 < ns; k0 += SV_KB) {
            const int kb = min(SV_KB, ns - k0);
            for (int e = tid; e < jb * SV_KB; e += nt) {
                const int r = e / SV_KB, k = e - r * SV_KB;
                Lc[r * (SV_KB + 1) + k] = (k < kb) ? LU[(long)sp[J0 + r] * ldl + k0 + k] : 0.0;
            }
            __syncthreads();
            for (int e = tid; e < jb * SV_COLS; e += nt) {
                const int r = e / SV_COLS, c = e - r * SV_COLS;
                double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
                int k = 0;
                for (; k + 3 < kb; k += 4) {
                    a0 += Lc[r * (SV_KB + 1) + k] * y[(k0 + k) * SV_YP + c];
                    a1 += Lc[r * (SV_KB + 1) + k + 1] * y[(k0 + k + 1) * SV_YP + c];
                    a2 += Lc[r * (SV_KB + 1) + k + 2] * y[(k0 + k + 2) * SV_YP + c];
                    a3 += Lc[r * (SV_KB + 1) + k + 3] * y[(k0 + k + 3) * SV_YP + c];
                }
                for (; k < kb; ++k) a0 += Lc[r * (SV_KB + 1) + k] * y[(k0 + k) * SV_YP + c];
                y[(J0 + r) * SV_YP + c] -= (a0 + a1) + (a2 + a3);
            }
            __syncthreads();
        }
        for (int e = tid; e < jb * 32; e += nt) {
            const int r = e >> 5, k = e & 31;
            Lc[r * (SV_KB + 1) + k] = (k < jb) ? LU[(long)sp[J0 + r] * ldl + J0 + k] : 0.0;
        }
        __syncthreads();
        for (int rp = jb - 1; rp >= 1; --rp) {  // diagonal block, right-looking: z_rp = y_rp / U_rp,rp
            for (int e = tid; e < rp * SV_COLS; e += nt) {
                const int r = e / SV_COLS, c = e % SV_COLS;
                y[(J0 + r) * SV_YP + c] -= Lc[r * (SV_KB + 1) + rp] * (y[(J0 + rp) * SV_YP + c] * rinv[J0 + rp]);
            }
            __syncthreads();
        }
        for (int e = tid; e < jb * SV_COLS; e += nt) {
            const int r = e / SV_COLS, c = e % SV_COLS;
            y[(J0 + r) * SV_YP + c] *= rinv[J0 + r];
        }
        __syncthreads();
    }
    for (int e = tid; e < ns * SV_COLS; e += nt) {
        const int j = e / SV_COLS, c = e - j * SV_COLS;
        if (c < nc) Z[(long)j * N + (eye ? sp[c0 + c] : c0 + c)] = y[j * SV_YP + c];
    }
}

cudaError_t launch_lu_solve(cudaStream_t st, const SolveArgs& a) {
    const size_t shm = ((size_t)a.ns * SV_YP + 32 * (SV_KB + 1) + a.ns) * sizeof(double) + (size_t)a.ns * sizeof(int);
    if (shm > 220 * 1024) return cudaErrorInvalidValue;
    {
        cudaError_t e = ensure_smem_attr((const void*)lu_solve_kernel, 220 * 1024);
        if (e != cudaSuccess) return e;
    }
    count_launch();
    lu_solve_kernel<<<dim3((a.N + SV_COLS - 1) / SV_COLS, a.nmat), 256, shm, st>>>(a);
    return cudaGetLastError();
}

}  // namespace afq
