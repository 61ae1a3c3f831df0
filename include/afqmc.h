/*
 * afqmc.h -- C ABI of libafqmc.so: the ground-state AFQMC (PQMC) auxiliary-field
 * update sweep on the walker's equal-time Green's function G, on one GB300
 * (sm_103a).
 *
 * The method: H. Du and Y.-Y. He, "Accelerating ground-state auxiliary-field
 * quantum Monte Carlo simulations by delayed update and block force-bias
 * update" (arXiv:2506.09611).  Section / equation names below are the paper's.
 *
 * Conventions.
 *   Sites i = x + Lx*y on an L x L periodic lattice, N = L*L.
 *   G_ij = <c_i c_j^+> (Eq. GrFMat); A = 1 - G.  Both spins are stored.
 *   Slices l = 1..M (Eq. ExpDtH); B_l^s = diag(exp(c_s x_{l,i})) exp(-dtau K)
 *   (Eq. BlMat).  Fields x_{l,i} = +-1.
 *   Matrices crossing the ABI are dense row-major unless stated otherwise.
 *
 * Ownership.  The library owns every device buffer it allocates (in
 * afqmc_create / afqmc_init_walkers) and frees them in afqmc_destroy.  Host
 * pointers passed in are only read (or written, for outputs) during the call;
 * the caller keeps ownership.  `stream` is a cudaStream_t passed as void*
 * (NULL = the legacy default stream); all device work of a call is enqueued
 * on it.  Calls on one context are not thread-safe.
 *
 * Errors.  Every call returns 0 on success or a negative AFQMC_ERR_* code.
 * An error other than AFQMC_ERR_ARG / AFQMC_ERR_STATE is sticky: later calls
 * on the context return it until afqmc_destroy.  afqmc_strerror gives text.
 */
#ifndef AFQMC_H
#define AFQMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AFQMC_OK 0
#define AFQMC_ERR_ARG (-1)      /* bad argument (sizes, modes, null pointers) */
#define AFQMC_ERR_OOM (-2)      /* device allocation failed */
#define AFQMC_ERR_CUDA (-3)     /* a CUDA runtime call or kernel launch failed */
#define AFQMC_ERR_NUMERIC (-4)  /* non-finite ratio / singular matrix on the device */
#define AFQMC_ERR_TIMEOUT (-5)  /* a bounded device-side wait expired */
#define AFQMC_ERR_STATE (-6)    /* call out of sequence (wrong slice / direction) */
#define AFQMC_ERR_NODEV (-7)    /* no sm_103 device */

/* Hubbard-Stratonovich decouplings (Sec. II.B, Eq. HSspinDecomp and Hirsch's real channels). */
#define AFQMC_HS_SZ_REAL 0      /* U >= 0: cosh(lam) = exp(dtau U/2), c_up = lam, c_dn = -lam */
#define AFQMC_HS_CHARGE_REAL 1  /* U <= 0: cosh(lam) = exp(dtau|U|/2), c_up = c_dn = lam, prefactor exp(-lam x) */

/* Bulk precision of G and of the update / wrap arithmetic. */
#define AFQMC_PREC_FP64 0       /* FP64 everywhere (parity mode) */
#define AFQMC_PREC_FP32 1       /* FP32 G; GEMMs at FP32 accuracy */

/* Update schemes of afqmc_sweep_slice (Sec. II.D and Sec. III). */
#define AFQMC_MODE_LOCAL 0      /* conventional local update (Eqs. DetRatiolocal, UpdateLTRlocal) */
#define AFQMC_MODE_DELAYED 1    /* delayed update (Eqs. DelayRatio, DelayRgenk, FinalDelay) */
#define AFQMC_MODE_BLOCKFB 2    /* block force-bias update (Eqs. BlockFrcbsRatio, BlkFrcBsTnew1/2) */

typedef struct afqmc_ctx afqmc_ctx;

/* Physical and numerical parameters shared by all walkers of a context. */
typedef struct {
    int hs;             /* AFQMC_HS_* */
    int precision;      /* AFQMC_PREC_* */
    int M;              /* number of imaginary-time slices, 2 Theta = M dtau */
    int stab_every;     /* slices between QR/LU re-orthonormalisations and G recomputes (k_tau) */
    double t;           /* nearest-neighbour hopping */
    double U;           /* Hubbard interaction */
    double dtau;        /* imaginary-time step */
    uint64_t seed;      /* Philox4x64-10 key word 0 (word 1 = walker index) */
    int gemm;           /* AFQMC_GEMM_* engine of the wrap and flush products (FP32 bulk) and of
                           the recompute's two FP64 products (both bulk precisions) */
} afqmc_params;

/* GEMM engines.  The wrap and flush products of the FP64 bulk are always FP64 SIMT products.
 * The recompute's FP64 products U_L U_R and U_R (U_L U_R)^{-1} U_L run on the FP64 pipe under
 * AFQMC_GEMM_SIMT; under TC3 and TF32 they run on the tcgen05 tensor cores as FP64-accurate
 * products of exact integer digit planes (error-free splitting; afqmc_debug_dgemm kind 1) where
 * the shape makes that faster. */
#define AFQMC_GEMM_TC3 0        /* tcgen05 tensor cores, three-term TF32 split (FP32 accuracy; default) */
#define AFQMC_GEMM_SIMT 1       /* FP32 FMA pipes */
#define AFQMC_GEMM_TF32 2       /* tcgen05 tensor cores, one TF32 pass (drift reported, not gated) */

/* Per-walker statistics of the last afqmc_sweep_slice (valid after a stream sync). */
typedef struct {
    int32_t proposals;  /* Metropolis tests (sites, or blocks for block FB) */
    int32_t accepts;    /* accepted tests */
    int32_t flipped;    /* fields changed */
    int32_t flushes;    /* rank-m updates applied to the full G */
    double max_abs_ratio;
    double sign;        /* sign of the walker weight W(X) after the slice */
} afqmc_slice_stats;

/* Create a context.  Checks for an sm_103 device; allocates nothing on it yet.
 * p is copied.  Returns AFQMC_ERR_ARG for M < 1, stab_every < 1, a bad mode or
 * a sign of U the decoupling does not allow. */
int afqmc_create(afqmc_ctx** out, const afqmc_params* p);

/* Free every device and host resource of the context.  NULL is a no-op. */
int afqmc_destroy(afqmc_ctx* ctx);

/* Allocate and initialise n_walkers walkers (Sec. II.B, Eqs. ConfgWeight, GrFMatNew).
 *   L[w]       linear lattice size of walker w (N_w = L[w]^2, 2 <= L <= 64).
 *   n_up[w], n_dn[w]  particles per spin, 1 <= n <= N_w.
 *   P          host, caller-owned: the trial determinants, concatenated per walker then
 *              per spin (up, dn), each N_w x n_s row-major (the columns are orbitals).
 *   fields     host, nullable: M x N_w int8 (+-1) per walker, concatenated; NULL draws
 *              i.i.d. +-1 fields from Philox(seed, walker).
 * Builds exp(-+dtau K), the left (U_L) stack of the slices, and G(0) on the device in
 * FP64, then stores G in the bulk precision.  The walker is left at slice 0, forward. */
int afqmc_init_walkers(afqmc_ctx* ctx, int n_walkers, const int* L, const int* n_up, const int* n_dn,
                       const double* P, const int8_t* fields, void* stream);

/* One slice of the sweep for every walker (Sec. II.C; forward l = 1..M, backward l = M..1).
 *   dir = +1: wrap G(l-1) -> G(l) = B_l G B_l^{-1}, then update the fields of slice l.
 *   dir = -1: update the fields of slice l, then wrap G(l) -> G(l-1) = B_l^{-1} G B_l.
 *   mode  AFQMC_MODE_*;  k  delay rank (sites per delayed step, 1 <= k <= 128 for FP32,
 *         <= 64 for FP64);  nb  block size for block FB (1 <= nb <= 32).
 *   replay  host, nullable: forced decisions, 2*N bytes per walker (concatenated):
 *         local / delayed: replay[i] = accept site i;  block FB: replay[i] = propose
 *         x'_i = +1 (else -1), replay[N + b] = accept block b.
 *   stats  host, nullable: one afqmc_slice_stats per walker (the call syncs the stream).
 * Uniforms come from Philox4x64-10, key (seed, walker), counter (j + 1, visit, 0, 0), where
 * visit counts the afqmc_sweep_slice calls of the walker; j < N are the site uniforms,
 * j = N + b the block-acceptance uniforms.  Returns AFQMC_ERR_STATE if the walker is not
 * at slice l-1 (forward) / l (backward), or if a re-orthonormalisation point was passed
 * without afqmc_recompute_G. */
int afqmc_sweep_slice(afqmc_ctx* ctx, int slice, int dir, int mode, int k, int nb, const uint8_t* replay,
                      afqmc_slice_stats* stats, void* stream);

/* FP64 recompute of G at the current slice (Sec. II.B, Eq. GrFMatNew): propagate the right
 * (forward) or left (backward) factor from the last re-orthonormalisation point, re-orthonormalise
 * it (pivoted LU in FP64), and form G = 1 - U_R (U_L U_R)^{-1} U_L, replacing the bulk G.  With an
 * FP32 bulk G (G form) G is formed from the propagated factor first and the re-orthonormalisation
 * follows on a side stream, only when the next interval would otherwise carry the basis over more
 * than 10 slices of propagation.
 * Must be called whenever the walker sits at a multiple of stab_every (and may be called only
 * there).  rel_drift (host, nullable, one per walker): ||G_bulk - G_new||_F / ||G_new||_F,
 * averaged over the spins (the call syncs the stream). */
int afqmc_recompute_G(afqmc_ctx* ctx, double* rel_drift, void* stream);

/* Mixed-estimator energy of every walker from its current G by Wick's theorem
 * (Eqs. 2DHubbard, Oxformula): E = sum_s tr(K A^s) + U sum_i (A^up_ii A^dn_ii - (A^up_ii + A^dn_ii)/2).
 * energy, sign: host, one double per walker (sign of W(X)).  Syncs the stream. */
int afqmc_measure_energy(afqmc_ctx* ctx, double* energy, double* sign, void* stream);

/* Accessors for tests and replay; all sync the stream of the last call. */
int afqmc_get_G(afqmc_ctx* ctx, int walker, int spin, double* host_out);          /* N x N row-major */
int afqmc_set_G(afqmc_ctx* ctx, int walker, int spin, const double* host_in);     /* N x N row-major */
int afqmc_get_fields(afqmc_ctx* ctx, int walker, int8_t* host_out);              /* M x N */
int afqmc_get_decisions(afqmc_ctx* ctx, int walker, uint8_t* host_out);          /* 2N, replay layout */
int afqmc_get_ratios(afqmc_ctx* ctx, int walker, double* host_out);              /* 2N: per site / N + block */
int afqmc_get_info(afqmc_ctx* ctx, int walker, int* N, int* n_up, int* n_dn, int* slice, int* dir);

/* Philox4x64-10 uniforms of the device generator, for checking the stream:
 * out[j] = u(seed, walker, visit, j) for j < count (device generator, copied to the host). */
int afqmc_debug_uniforms(uint64_t seed, uint64_t walker, uint64_t visit, int count, double* host_out);

/* Validation hook for the bounded device waits: one thread waits on a device flag that nothing
 * sets, for limit_ns nanoseconds of %globaltimer (1000 <= limit_ns <= 2e9), then records the device
 * timeout code and returns.  Every bounded wait of the library (grid barriers, mbarrier waits)
 * takes this path when it expires.  Allocates and frees 8 bytes of device memory; syncs the
 * stream.  Returns AFQMC_ERR_TIMEOUT, the expected outcome, with the CUDA context still usable;
 * AFQMC_ERR_ARG for a limit out of range (checked before any device call). */
int afqmc_debug_wait_timeout(long long limit_ns, void* stream);

/* Apply accepted field changes at the sites I to both spins' G in one rank-m product -- the G form
 * of the delayed flush (Eq. FinalDelay) and of the block force-bias upgrade (Eq. BlkFrcBsTnew2):
 *     G_s <- G_s - G_s[:, I] W_s (E_I^T - G_s[I, :]),  W_s = D_s (1 + (1 - G_s[I, I]) D_s)^{-1}.
 * Stateless (no context).  All pointers are device pointers, caller-owned:
 *   G_up, G_dn  N x N row-major with leading dimension ld (>= N), double for AFQMC_PREC_FP64 and
 *               float for AFQMC_PREC_FP32; updated in place.
 *   sites       m distinct site indices in [0, N), in the order the changes were accepted.
 *   delta       2*m doubles, delta[s*m + a] = exp(c_s (x'_a - x_a)) - 1 (spin s = 0 up, 1 down).
 *   m           0 <= m <= 128 (FP32) or 64 (FP64); 0 is a no-op.
 * Work is enqueued on `stream`; device scratch comes from cudaMallocAsync on that stream and is freed
 * there.  The call then copies the device's status word back and waits for the stream, so it returns
 * after the update.  Returns AFQMC_ERR_ARG for bad sizes or null pointers (checked before any device
 * work) and for a site outside [0, N) (found on the device; G is left unchanged), and
 * AFQMC_ERR_NUMERIC when 1 + (1 - G_II) D has a zero pivot for either spin (G is left unchanged). */
int afqmc_apply_flips(int precision, int N, long long ld, void* G_up, void* G_dn, const int* sites,
                      const double* delta, int m, void* stream);

/* afqmc_apply_flips without any device allocation.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory where they apply an update -- code
 * running under a fixed device-memory budget owned by a host framework, a real-time loop in which
 * cudaMalloc / cudaMallocAsync (and the synchronisation they may cause) is not allowed, or a plugin
 * whose host process gives it no allocator.  It computes exactly what afqmc_apply_flips computes,
 * with the same arguments and limits, plus:
 *   N <= AFQMC_NOALLOC_MAX_N, else AFQMC_ERR_ARG.
 * Its scratch is one file-scope __device__ array of about 12.7 MB (enough for N = 4096 in either
 * precision); every GPU that loads libafqmc.so holds that array until the process exits.  The
 * first call on a device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current, so make the first call on each device before any stream capture.  All calls
 * share the array and it keeps the last call's contents; nothing in it has to start at zero (every
 * call rewrites the status word and the sizes it reads), but calls whose work overlaps on the GPU
 * (e.g. on two streams) race on it.  Like afqmc_apply_flips it reads the status word back and waits
 * for the stream, with the same error codes.  It calls no cudaMalloc, cudaFree or allocating library
 * routine. */
#define AFQMC_NOALLOC_MAX_N 4096
int afqmc_apply_flips_noalloc(int precision, int N, long long ld, void* G_up, void* G_dn, const int* sites,
                              const double* delta, int m, void* stream);

/* Walker representation (Sec. II.C, Eq. GrFMatNew).
 *   AFQMC_FORM_G  the equal-time Green's function G (N x N per spin) is the state: the wrap moves G
 *                 (G <- B G B^{-1}) and every window's update is a rank-m product over all of G.
 *   AFQMC_FORM_T  the paper's own state: U_R (N x Nsigma), U_L (Nsigma x N) and T = (U_L U_R)^{-1}
 *                 (Nsigma x Nsigma) per spin, G = 1 - U_R T U_L formed only when asked for
 *                 (afqmc_get_G, afqmc_measure_energy, the drift of afqmc_recompute_G).  The wrap moves
 *                 the factors (U_R <- B U_R, U_L <- U_L B^{-1}) and leaves T; a window's accepted
 *                 sites I update T <- T - (T U_L[:, I]) W (U_R[I, :] T) (Eqs. FinalDelay,
 *                 BlkFrcBsTnew2) and scale the rows I of U_R (Eq. UpdateLTRMat); the recompute takes
 *                 U_R and U_L from the FP64 factors, the left one as (U_L U_R)^{-1} U_L so that T = 1
 *                 (the same G; the FP32 state stays accurate).  Decisions and G equal the G form's.
 *                 Requires n_up = n_dn for every walker; AFQMC_MODE_LOCAL is not offered (delayed
 *                 with k = 1 is the local update); afqmc_set_G returns AFQMC_ERR_STATE; no CUDA-graph
 *                 capture (afqmc_set_graphs is ignored).
 * afqmc_set_form must come before afqmc_init_walkers (AFQMC_ERR_STATE after it); AFQMC_ERR_ARG for
 * a NULL ctx or an unknown form.  The default is AFQMC_FORM_G. */
#define AFQMC_FORM_G 0
#define AFQMC_FORM_T 1
int afqmc_set_form(afqmc_ctx* ctx, int form);

/* ---- Ground-state constrained-path AFQMC (CPQMC, Sec. IV.D, Eqs. CPWvfct1, CPWvfct2, ptilde) ----
 * The ensemble |Psi> = sum_k w_k |phi_k> / <psi_T|phi_k> of the context's walkers, each a Slater
 * determinant phi_k per spin (N x n_s, n_s = n_up = n_dn) carried in the T form: U_R = phi_k,
 * U_L = psi_T^+ (fixed), T = (U_L U_R)^{-1}.  Requires a context with AFQMC_FORM_T, FP64 precision
 * and one lattice for all walkers (afqmc_init_walkers builds the buffers; its fields are scratch
 * for the current step).  AFQMC_ERR_STATE otherwise.
 *
 * afqmc_cp_init: psi_T = P (host, N x n_s row-major, the same for both spins and every walker),
 *   phi_k = phi0 (host, nullable: per walker (in afqmc_init_walkers order) spin up then spin down,
 *   each N x n_s; NULL starts every walker at P); weights 1.
 * afqmc_cp_step: one projection step e^{-dtau K} then the fields of one slice for every walker:
 *   the kinetic step multiplies w_k by <psi_T|e^{-dtau K} phi_k> / <psi_T|phi_k> (determinants of
 *   U_L U_R before and after, from a fresh pivoted LU that also gives T); then every site i in
 *   order draws its field from lambda(x) = p(x) s(x) r_up(x) r_dn(x), p = 1/2, s(x) the
 *   decoupling's scalar (e^{-lam x} charge channel, 1 spin channel), r_s(x) = 1 + (e^{c_s x} - 1)
 *   A_s[i][i] with A = U_R T U_L, negative lambda clamped to 0 (the constrained path),
 *   x = +1 iff u_i < lambda(+1) / N_i, N_i = lambda(+1) + lambda(-1) (heat bath, Philox uniform
 *   u_i of the walker's visit as in afqmc_sweep_slice), w_k <- w_k N_i; the chosen field updates
 *   T and U_R as an accept of the delayed update: mode AFQMC_MODE_LOCAL (one site per window) or
 *   AFQMC_MODE_DELAYED (windows of k sites, rank-k updates of T; the same fields and weights).
 *   AFQMC_MODE_BLOCKFB (blocks of nb <= 32 sites): the force bias F_i of a block's sites before any
 *   is set (spin channel sum_s c_s A_s[i][i], charge channel lam (A_up + A_dn - 1)[i][i]), each
 *   x_i drawn from e^{x_i F_i} / (2 cosh F_i) (site uniforms), and w_k times
 *   prod_i s(x_i) cosh F_i e^{-x_i F_i} prod_s det(1 + Delta_s A_s[S][S]), removed when that
 *   factor is <= 0 (nb = 1 is a heat bath with the linearised weights).
 *   A walker whose overlap would change sign or whose N_i vanishes is removed (weight 0; its slot
 *   holds a copy of a live walker's basis until the next afqmc_cp_comb).  logw_step (host,
 *   nullable, one per walker): ln of the step's weight factor (-inf when removed).
 *   AFQMC_ERR_NUMERIC when every walker is removed.
 * afqmc_cp_comb: population control by the comb: with W the total weight, positions (q + u0) W / n_w
 *   (0 <= u0 < 1) in the cumulative weights select walker idx[q] for slot q; every new weight is
 *   W / n_w.  idx_out (host, nullable, n_w).
 * afqmc_cp_reorth: re-orthonormalise every phi_k (pivoted LU basis of its columns), which changes
 *   no weight (Eq. CPWvfct1 divides the scale out).
 * afqmc_cp_energy: the mixed estimator E_L(k) = <psi_T|H|phi_k> / <psi_T|phi_k> per walker
 *   (e_local, host, nullable) and sum_k w_k E_L(k) / sum_k w_k (e_mean, host, nullable).
 * afqmc_cp_get_walker: phi_k (host, 2 N n_s doubles, nullable) and ln w_k (nullable).
 * All sync the stream. */
int afqmc_cp_init(afqmc_ctx* ctx, const double* P, const double* phi0, void* stream);
int afqmc_cp_step(afqmc_ctx* ctx, int mode, int k, int nb, double* logw_step, void* stream);
int afqmc_cp_comb(afqmc_ctx* ctx, double u0, int* idx_out, void* stream);
int afqmc_cp_reorth(afqmc_ctx* ctx, void* stream);
int afqmc_cp_energy(afqmc_ctx* ctx, double* e_local, double* e_mean, void* stream);
int afqmc_cp_get_walker(afqmc_ctx* ctx, int walker, double* phi, double* logw);

/* Profiling.  With profiling on, every phase of afqmc_sweep_slice / afqmc_recompute_G is
 * bracketed by CUDA events recorded on the call's stream (the stream its kernels run on).
 * Phases: */
#define AFQMC_PHASE_PREP 0       /* uniforms, field scales, stats reset */
#define AFQMC_PHASE_WRAP 1       /* the two wrap products G <- B G B^{-1} (Eq. BlMat) */
#define AFQMC_PHASE_LOCAL 2      /* the local-update site loop */
#define AFQMC_PHASE_CHAIN 3      /* delayed / block-FB window decisions (one CTA per window) */
#define AFQMC_PHASE_FLUSH 4      /* panel gather + rank-m product of the delayed / block-FB update */
#define AFQMC_PHASE_RECOMPUTE 5  /* FP64 propagation, re-orthonormalisation and G = 1 - U_R T U_L */
/* Nested intervals inside the phases above, one per kernel launch (for per-kernel rooflines): */
#define AFQMC_PHASE_ELIM 6       /* each re-orthonormalisation LU, N x Nsigma, both spins (inside RECOMPUTE) */
#define AFQMC_PHASE_WRAP_GEMM 7  /* each wrap product launch (inside WRAP) */
#define AFQMC_PHASE_FLUSH_GEMM 8 /* each rank-m product launch of the flush (inside FLUSH) */
#define AFQMC_PHASE_LU_O 9       /* each LU of U_L U_R, Nsigma x Nsigma, both spins (inside RECOMPUTE) */
#define AFQMC_PHASE_SOLVE 10     /* each solve (U_L U_R) Z = U_L, both spins (inside RECOMPUTE) */
#define AFQMC_PHASE_DGEMM 11     /* each digit-split FP64 product U_L U_R or U_R Z, both spins (inside RECOMPUTE) */
#define AFQMC_NPHASE 12
/* on != 0 enables profiling and clears the accumulators; on == 0 disables it. */
int afqmc_set_profiling(afqmc_ctx* ctx, int on);

/* CUDA graphs (a deployment option, not in the paper).  With on != 0, afqmc_sweep_slice captures
 * each walker group's slice -- uniforms, wrap, window chain, the flush stream's panels and
 * products -- the first time it meets a given (slice, dir, mode, k, nb), and replays the graph
 * from then on: one graph launch per group and slice.  Calls with replay decisions or with
 * profiling on run uncaptured.  The uniforms stay fresh because the visit counter that keys them
 * lives on the device.  Returns AFQMC_ERR_ARG for a NULL ctx. */
int afqmc_set_graphs(afqmc_ctx* ctx, int on);

/* How the wrap G <- B G B^{-1} (Eqs. BlMat, GrFMat) forms E G and G E^{-1}, E = exp(-dtau K):
 *   AFQMC_WRAP_DENSE      two dense N x N products (tensor cores for FP32 bulk);
 *   AFQMC_WRAP_SEPARABLE  the periodic L x L lattice has E = Ex (x) Ex, so each product is two
 *                         L-point passes over one index of G (2 L N^2 instead of N^3 multiply-adds),
 *                         in the bulk precision, with the field scalings folded into the passes.
 * A new context uses the separable wrap for every walker group whose lattice it covers (every
 * lattice up to 64 x 64: four line passes of one lattice coordinate each; larger ones while a tile
 * of 4 columns fits on chip) and the dense wrap otherwise; afqmc_set_wrap fixes one mode for all
 * groups.  Applies to the following slices.  AFQMC_ERR_ARG for a NULL ctx, an unknown mode, or
 * (separable) a walker lattice it does not cover. */
#define AFQMC_WRAP_DENSE 0
#define AFQMC_WRAP_SEPARABLE 1
int afqmc_set_wrap(afqmc_ctx* ctx, int mode);
/* Form of the separable wrap.  width = 0 (the default): four line passes per wrap, each applying Ex
 * along one lattice coordinate of G's row or column index, one L-point line per thread in
 * registers (lattices up to 64 x 64; larger ones take tiles of 4).  width > 0: two tile passes,
 * each thread block transforming `width` columns (rows) of G over all N rows (columns) in shared
 * memory; width must be a multiple of 4 whose tile fits in shared memory for every walker's
 * lattice, else AFQMC_ERR_ARG.  A performance knob (the tuner times it); the result agrees to
 * rounding. */
int afqmc_set_wrap_tile(afqmc_ctx* ctx, int width);
/* Sync the last stream and return, per phase, the summed device milliseconds, the number of
 * bracketed intervals, and the number of library kernels launched in that phase.  Each array
 * has AFQMC_NPHASE entries; any pointer may be NULL. */
int afqmc_get_profile(afqmc_ctx* ctx, double* ms, int64_t* intervals, int64_t* launches);
/* Number of library kernels launched by this process so far (every launch site counts). */
int64_t afqmc_launch_count(void);

/* Validation hook for the tensor-core GEMM: C = A * Bt^T (FP32, device pointers, row-major
 * A: M x K, Bt: N x K, C: M x N; c_trans = 1 writes C^T, N x M), with kind 1 = tcgen05 one-pass
 * TF32, kind 2 = tcgen05 three-term TF32 split (FP32 accuracy).  lda, ldb >= K and ldc >= N
 * (>= M with c_trans); pointers and leading dimensions must be 16-byte aligned.  Syncs the
 * stream.  AFQMC_ERR_ARG for bad sizes, pointers or strides; AFQMC_ERR_TIMEOUT if a device wait
 * expired. */
int afqmc_debug_gemm(int kind, int M, int N, int K, const float* A, long long lda, const float* Bt,
                     long long ldb, float* C, long long ldc, int c_trans, void* stream);

/* Validation hook for the recompute's FP64 products: C = A * B (FP64, device pointers, row-major
 * A: M x K, B: K x N, C: M x N with leading dimensions lda >= K, ldb >= N, ldc >= N), kind 0 =
 * FP64 SIMT product, kind 1 = digit-split product on the tcgen05 tensor cores (every element of A
 * and B split into b-bit integer digits relative to the largest exponent of its row of A or
 * column of B; digit planes stored as bf16, which holds such small integers exactly, and
 * multiplied by tcgen05 kind::f16 with exact FP32 accumulation; levels summed in FP64).  Allocates and frees its own workspace; syncs the stream.  AFQMC_ERR_NUMERIC for an
 * element of magnitude >= 2^1023 or non-finite, AFQMC_ERR_TIMEOUT if a device wait expired,
 * AFQMC_ERR_ARG for K beyond the exact range of the split. */
int afqmc_debug_dgemm(int kind, int M, int N, int K, const double* A, long long lda, const double* B,
                      long long ldb, double* C, long long ldc, void* stream);

/* The digit-split plan of afqmc_debug_dgemm kind 1 (and of the recompute) for an M x N x K
 * product with `batch` entries; host only, no device use.  Writes the digit width *b (bits), the
 * digits per element *s and the number of groups *ngroups (one tensor-core pass each); for the first
 * `cap` groups, np[g] plane pairs with 1-based digit indices pa[16 g + i], pb[16 g + i] (host,
 * caller-owned, 16 slots per group).  Every pair of a group has the same level p + q, and
 * np[g] K (2^b - 1)^2 < 2^24 (the FP32 accumulator stays exact).  AFQMC_ERR_ARG for K beyond the
 * exact range or bad pointers. */
int afqmc_debug_ozaki_plan(int M, int N, int K, int batch, int* b, int* s, int* ngroups, int cap, int* np,
                           int* pa, int* pb);

const char* afqmc_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* AFQMC_H */
