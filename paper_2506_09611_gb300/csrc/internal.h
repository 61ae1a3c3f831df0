// internal.h -- host-side declarations shared by the libafqmc translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"

namespace afq {

// Every kernel launch site calls count_launch() (the counter behind afqmc_launch_count()).
void count_launch(int n = 1);

// cudaFuncSetAttribute(fn, attr, value) once per (device, kernel, attribute), thread-safe; a
// larger value than the one set before on the device sets it again.
cudaError_t ensure_func_attr(const void* fn, cudaFuncAttribute attr, int value);
inline cudaError_t ensure_smem_attr(const void* fn, size_t bytes) {
    return ensure_func_attr(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Row-major batched GEMM with diagonal scalings (all pointers device):
//   C[z] = alpha * diag(rs[z]) * A[z] * diag(bs[z]) * B[z] * diag(cs[z]) + beta * C[z]
// A is M x K (lda), B is K x N (ldb), C is M x N (ldc).  Null scale pointers
// mean 1.  If Kdev is non-null the inner dimension is read from *Kdev on the
// device (<= K).  beta == 0 never reads C.
template <typename T>
struct GemmArgs {
    int M = 0, N = 0, K = 0;
    const int* Kdev = nullptr;  // device K (min with K); with kdiv > 0, batch z reads Kdev[z / kdiv]
    int kdiv = 0;
    const T* A = nullptr; long lda = 0, sA = 0;
    const T* B = nullptr; long ldb = 0, sB = 0;
    T* C = nullptr; long ldc = 0, sC = 0;
    T alpha = 1, beta = 0;
    const T* rs = nullptr; long srs = 0;
    const T* cs = nullptr; long scs = 0;
    const T* bs = nullptr; long sbs = 0;
    int batch = 1;
};

template <typename T>
cudaError_t gemm(cudaStream_t st, const GemmArgs<T>& g);

// tcgen05 tensor-core GEMM (tc_gemm.cu), FP32 in/out:
//   C[z] = alpha * diag(rs[z]) * A[z] * Bt[z]^T * diag(cs[z]) + beta * C[z]
// A (M x K) and Bt (N x K) row-major (K contiguous); sA / sB = 0 share one matrix across the
// batch.  c_trans writes C^T (C[n * ldc + m]).  split3 selects the three-term TF32 split (FP32
// accuracy); otherwise one TF32 pass.  Base pointers and leading dimensions must be 16-byte
// aligned (TMA).  err receives DEV_TIMEOUT if a bounded wait expires.
struct TcGemmArgs {
    int M = 0, N = 0, K = 0, batch = 1;
    const float* A = nullptr; long lda = 0, sA = 0;
    const float* Bt = nullptr; long ldb = 0, sB = 0;
    float* C = nullptr; long ldc = 0, sC = 0;
    int c_trans = 0;
    const float* rs = nullptr; long srs = 0;
    const float* cs = nullptr; long scs = 0;
    float alpha = 1.0f, beta = 0.0f;
    int split3 = 1;
    int* err = nullptr;
};
cudaError_t tc_gemm(cudaStream_t st, const TcGemmArgs& g);

// One group of digit-plane products on the tensor cores (tc_gemm.cu), for ozaki_gemm:
//   C[z] (+)= gscale * diag(rsc[z]) * (sum_i Ad[z][pa[i]] * Bd[z][pb[i]]^T) * diag(csc[z])
// Ad: [batch][ns][M][Kp] and Bd: [batch][ns][N][Kp] bf16 planes of small integers (K used,
// zero-padded to Kp, a multiple of 8); rsc [batch][M], csc [batch][N]; C FP64 row-major
// (ldc, batch stride sC).  first = 1 overwrites C.  The caller guarantees that the sum of the
// magnitudes of all products of one output stays below 2^24 (exact in the FP32 accumulator).
constexpr int TC_OZ_MAXP = 16;
struct TcOzArgs {
    int M = 0, N = 0, K = 0, Kp = 0, batch = 1, ns = 0;
    const uint16_t* Ad = nullptr;  // bf16 bit patterns
    const uint16_t* Bd = nullptr;
    int np = 0;
    int pa[TC_OZ_MAXP] = {}, pb[TC_OZ_MAXP] = {};
    double* C = nullptr; long ldc = 0, sC = 0;
    const double* rsc = nullptr;
    const double* csc = nullptr;
    double gscale = 1.0;
    int first = 1;
    int* err = nullptr;
};
cudaError_t tc_gemm_oz(cudaStream_t st, const TcOzArgs& g);

// FP64 GEMM C[z] = A[z] B[z] (A: M x K, B: K x N, C: M x N, all row-major FP64 with the given
// leading dimensions and batch strides) on the TF32 tensor cores by error-free digit splitting
// (ozaki.cu).  ws / sc: workspace of ozaki_ws_bytes bytes / ozaki_sc_doubles elements.
struct OzGemmArgs {
    int M = 0, N = 0, K = 0, batch = 1;
    const double* A = nullptr; long lda = 0, sA = 0;
    const double* B = nullptr; long ldb = 0, sB = 0;
    double* C = nullptr; long ldc = 0, sC = 0;
    int* err = nullptr;
};
size_t ozaki_ws_bytes(int M, int N, int K, int batch);
size_t ozaki_sc_doubles(int M, int N, int batch);
// true when the digit-split product is expected to beat the FP64 SIMT GEMM at this shape
bool ozaki_pays(int M, int N, int K, int batch);
cudaError_t ozaki_gemm(cudaStream_t st, const OzGemmArgs& g, void* ws, double* sc);
// The plan ozaki_gemm uses for a shape (host only): digit width b, digits s, and per group its
// pairs (1-based digit indices, TC_OZ_MAXP slots per group, the first `cap` groups).  -1 when K is
// beyond the exact range of every digit width.
int ozaki_plan_info(int M, int N, int K, int batch, int* b, int* s, int* ngroups, int cap, int* np, int* pa,
                    int* pb);

// ---- setup / recompute kernels (setup.cu) ----
cudaError_t launch_expK(cudaStream_t st, int L, double t, double tau, double* E, long ld);
cudaError_t launch_expK1d(cudaStream_t st, int L, double t, double tau, double* Ex);  // L x L factor
cudaError_t launch_scale_rows(cudaStream_t st, double* U, int rows, int cols, const double* d);  // U[r,:] *= d[r]
cudaError_t launch_scale_cols(cudaStream_t st, double* U, int rows, int cols, const double* d);  // U[:,c] *= d[c]

template <typename T>
cudaError_t launch_cast(cudaStream_t st, const double* src, long lds, T* dst, long ldd, int rows, int cols,
                        int nbatch = 1, long ssrc = 0, long sdst = 0);
template <typename T>
cudaError_t launch_to_double(cudaStream_t st, const T* src, long lds, double* dst, long ldd, int rows, int cols);
cudaError_t launch_field_scales(cudaStream_t st, const int8_t* x, int N, double c, double* d, double* dinv);
template <typename T>
cudaError_t launch_field_scales_T(cudaStream_t st, const int8_t* x, int N, const double* c2, T* d, T* dinv, long sd,
                                  int nwk = 1, long xstride = 0);

// Fused FP64 propagation over nsl slices l = l_first, l_first + l_step, ... (setup.cu) of nmat
// factors: factor b (walker j = b / 2, spin s = b % 2) at U0 + j wstride + s sstride holds
// nvec[s] vectors of length N = L*L (element i of vector v at [v * vs[s] + i * es[s]]);
// right factors: v <- D_l (E v); left factors (left != 0): v <- E (D_l v); E = Ex (x) Ex,
// D_l = diag(x_{l,i} > 0 ? dplus[s] : dminus[s]) with x the walker's M x N fields.
struct PropArgs {
    double* U0 = nullptr;
    long wstride = 0, sstride = 0;
    long vs[2] = {0, 0}, es[2] = {0, 0};
    int nvec[2] = {0, 0};
    double dplus[2] = {1.0, 1.0}, dminus[2] = {1.0, 1.0};
    const double* Ex = nullptr;
    const int8_t* x = nullptr;
    long xstride = 0;
    int L = 0, l_first = 1, l_step = 1, nsl = 0, left = 0, nmat = 2;
};
cudaError_t launch_prop(cudaStream_t st, const PropArgs& a);

// Blocked partially pivoted LU in FP64 (lu.cu) of nmat row-major m x n matrices (m >= n) without
// row swaps.  Matrix b (walker j = b / ng, spin q = b % ng) sits at A0 + j wstride + q sstride;
// its pivot rows go to perm0 + b pstride (perm[c] = pivot row of column c) and flag0 + b pstride
// is m bytes of scratch.  After launch_lu a pivot row holds its multipliers left of its column
// and its U entries from there on; unpivoted rows hold multipliers.  err receives DEV_NUMERIC
// on a zero pivot.
struct LuArgs {
    double* A0 = nullptr;
    long wstride = 0, sstride = 0;
    int ng = 1;
    int* perm0 = nullptr;
    int8_t* flag0 = nullptr;
    long pstride = 0;
    long lda = 0;
    int m = 0, n = 0, nmat = 1;
    int* err = nullptr;
};
cudaError_t launch_lu(cudaStream_t st, const LuArgs& a);
// After launch_lu: pivot rows become unit rows, so A = P L spans the factored columns.
cudaError_t launch_lu_unit_rows(cudaStream_t st, const LuArgs& a);
// After launch_lu: sign_out[j] *= sign(prod of pivots) (times the row permutation's parity when
// parity != 0) over the ng matrices of walker j; visited: nmat * m ints of scratch.
cudaError_t launch_lu_sign(cudaStream_t st, const LuArgs& a, int parity, double* sign_out, int* visited);
// Z = O^{-1} B for the O factored by launch_lu (ns x ns, leading dimension ldl, matrix b at
// LU0 + b ostride with pivots perm0 + b pstride), B (ns x N) at B0 + j wstride + q sstride
// (b = j ng + q), row stride ldb (0: N), and Z (ns x N) at Z0 + b zstride.
struct SolveArgs {
    const double* LU0 = nullptr;
    long ostride = 0;
    const int* perm0 = nullptr;
    long pstride = 0;
    const double* B0 = nullptr;
    long wstride = 0, sstride = 0;
    int ng = 1;
    double* Z0 = nullptr;
    long zstride = 0;
    long ldl = 0;
    long ldb = 0;  // row stride of B (0: N)
    int ns = 0, N = 0, nmat = 1;
    // eye != 0: B is the identity with its columns in pivot order (column c = e_{perm[c]}, N = ns,
    // B0 unused), so the forward substitution of column c starts at row c; the solution's column c
    // is stored at column perm[c], which makes Z = O^{-1}
    int eye = 0;
};
cudaError_t launch_lu_solve(cudaStream_t st, const SolveArgs& a);
template <typename T>
cudaError_t launch_identity_minus(cudaStream_t st, T* G, long ld, int N, int nbatch = 1, long sG = 0);  // G = I - G
template <typename T>
cudaError_t launch_drift(cudaStream_t st, const T* Gold, const T* Gnew, long ld, int N, double* acc2, int nbatch = 1,
                         long sold = 0, long snew = 0, int adiv = 1);
template <typename T>
cudaError_t launch_energy(cudaStream_t st, const T* Gu, long ld, int L, double t, double U, double* out, int nwk = 1,
                          long gstride = 0);

// ---- sweep kernels (sweep.cu) ----
// Per-slice constants of the site loop.  The field-change factors depend only on the
// spin and the current field value, so they are four numbers computed once on the host:
//   dflip[s][xi]  = exp(-2 c_s x) - 1   (flip x -> -x; Sec. II.D)
//   dstrip[s][xi] = exp(-c_s x) - 1     (remove the field: the stripped force bias, Sec. III.B)
//   sflip[xi]     = s(-x) / s(x)        (scalar prefactor of the decoupling)
// with xi = 0 for x = +1 and xi = 1 for x = -1.
struct SiteParams {
    int N;
    long ld;
    double c[2];     // c_up, c_dn
    double lam;      // HS coupling (for the scalar prior of the charge channel)
    int hs;
    uint64_t seed, walker, visit;
    double dflip[2][2];
    double dstrip[2][2];
    double sflip[2];
};

struct SliceOut {      // device-side per-walker outputs of one slice
    uint8_t* dec;      // 2N replay-layout decisions
    double* ratio;     // 2N ratios
    int* stats;        // [proposals, accepts, flipped, flushes]
    double* maxr;      // max |R|
    double* sign;      // walker sign (updated in place)
    double* cp = nullptr;  // constrained-path heat bath: per walker [sum ln N_i, sum ln |r_up r_dn|,
                           // removed flag] (nullable; accumulated)
};

// The window kernel's constrained-path heat bath (Sec. IV.D; not a public sweep mode): every site
// of the window gets a field drawn from lambda(x) = dflip-style constants -- SiteParams.dflip[s][xi]
// = e^{c_s x} - 1 (the field set from none) and sflip[xi] = p(x) s(x) -- with the chosen one applied
// as an accept of the delayed update.
constexpr int WIN_MODE_CP = 16;
// ... and its block force bias (blocks of nb sites drawn from the force bias, weight factor by the
// block's determinant; the same constants).
constexpr int WIN_MODE_CPB = 17;

// u[j][0..count) for the walkers gid[j] (device array), j < nwk, at the device visit counter;
// launch_bump advances the counter by one.
cudaError_t launch_uniforms(cudaStream_t st, uint64_t seed, const int* gid, const unsigned long long* visit, int count,
                            double* u, int nwk);
cudaError_t launch_bump(cudaStream_t st, unsigned long long* visit);

template <typename T>
cudaError_t launch_local(cudaStream_t st, T* Gu, T* Gd, int8_t* xl, const double* u, const uint8_t* replay,
                         const SiteParams& sp, SliceOut so, T* colbuf, T* rowbuf, GridBar* bar, int* err,
                         int max_blocks);

struct WindowBufs {    // device scratch of the window chain + flush
    int* m;            // accepted count of the window
    int* idx;          // accepted site indices (global), capacity NW
    double* dtot;      // per spin, 2 x NW: sweep: recursion factor -Delta/r; apply_flips: unused
    void* Wm;          // per spin NW x NW (T): sweep: frozen block coefficients; apply_flips: W
    void* Wx;          // per spin NW x NW (T): sweep: the window's update matrix W
    void* X;           // per spin N x NW column panel (T)
    void* Y;           // per spin NW x N row panel (T), plus room for a second product
    int nwk = 1;       // walkers in the group: every buffer above holds nwk back-to-back copies
};

// A group of walkers with the same lattice and particle numbers: their per-walker buffers are
// laid out back to back and every launch of a slice covers the whole group.
struct Batch {
    int nwk = 1;        // walkers in the group
    long gstride = 0;   // elements between consecutive walkers' G ([2][N][ld])
    long xstride = 0;   // bytes between consecutive walkers' fields (M x N)
};

template <typename T>
int window_max();      // largest window (sites) the chain kernel holds in shared memory

// Separable wrap products (sepwrap.cu, code in sepwrap.cuh): G <- (A (x) A) G (side 0) or
// G <- G (A (x) A) (side 1) for the batch of N x N matrices of a SepArgs, with its optional row /
// column scalings before and after.  SepArgs::w == 0 takes the line passes where L <= 64 (else
// tiles of the default width), w > 0 tiles of w columns.  cudaErrorInvalidValue when N != L^2 or
// the requested tiles do not fit on chip.  sep_width: the default tile width (0: none fits).
struct SepArgs;
template <typename T>
int sep_width(int L, int N);
template <typename T>
bool sep_width_fits(int L, int N, int w);  // a tile of w columns (w % 4 == 0) fits on chip
template <typename T>
bool sep_available(int L, int N);          // launch_sep with w = 0 applies (line passes or tiles)
template <typename T>
cudaError_t launch_sep(cudaStream_t st, const SepArgs& a);

template <typename T>
cudaError_t launch_window_chain(cudaStream_t st, int mode, const T* Gu, const T* Gd, int8_t* xl, const double* u,
                                const uint8_t* replay, const SiteParams& sp, SliceOut so, int s0, int n, int nb,
                                WindowBufs wb, const T* blk, int* err, Batch bt = Batch());
template <typename T>
cudaError_t launch_flush(cudaStream_t st, T* Gu, T* Gd, const SiteParams& sp, WindowBufs wb, int nw);
// Pipelined flush of a window (the window kernel leaves its update matrix W in wb.Wx):
//   launch_next_block   -- the next window's block [sn, sn + nn) of both spins as it will be
//                          after this window's update; run right after the window kernel;
//   launch_flush_panels -- X = G[:, I], Yraw = E_I^T - G[I, :], Y' = W Yraw;
//   launch_flush_gemm   -- G <- G - X Y'.
template <typename T>
cudaError_t launch_next_block(cudaStream_t st, const T* Gu, const T* Gd, const SiteParams& sp, WindowBufs wb, int sn,
                              int nn, T* snap, Batch bt = Batch());
template <typename T>
cudaError_t launch_flush_panels(cudaStream_t sf, T* Gu, T* Gd, const SiteParams& sp, WindowBufs wb, int nw,
                                Batch bt = Batch());
template <typename T>
cudaError_t launch_flush_gemm(cudaStream_t sf, T* Gu, T* Gd, const SiteParams& sp, WindowBufs wb, int nw,
                              Batch bt = Batch());
// T form: the gathers of the window's accepted sites I for every (walker, spin) z of the batch,
// ULI[z] = UL[z][:, I] (ns x m, pitch window_max<T>()) and URI[z] = UR[z][I, :] (m x ns, pitch ldr),
// and the row scaling UR[z][I_k, :] *= exp(2 c_s x'_{I_k}) with the slice's new fields.  UR: N x ns
// (leading dimension ldr), UL: ns x N; batch strides sr, sl; z = 2 walker + spin.
template <typename T>
cudaError_t launch_tform_gather(cudaStream_t st, const T* UR, const T* UL, int N, int ns, long ldr, long sr, long sl,
                                WindowBufs wb, T* ULI, T* URI, int nbatch);
template <typename T>
cudaError_t launch_tform_scale_rows(cudaStream_t st, T* UR, int N, int ns, long ldr, long sr, WindowBufs wb,
                                    const int8_t* xl, long xstride, const double* c, int nbatch);
// G_s[i][j] *= a_s[i] * b_s[j] for both spins (a, b: [2][N], spin stride N)
template <typename T>
cudaError_t launch_scale2(cudaStream_t st, T* G, long ld, int N, long sG, const T* a, const T* b, int nbatch = 2);

}  // namespace afq
