/*
 * afqmc_soc.h -- C ABI of the spin-orbit-coupled (spin-mixing) sweep in libafqmc.so:
 * the PQMC auxiliary-field update on the walker's complex equal-time Green's function
 * G of the 2N orbitals (Appendix A of H. Du and Y.-Y. He, arXiv:2506.09611).
 *
 * Model (Appendix A, Eqs. 2DSocHubbard, HSspinSyDep, A2times2).
 *   Orbitals a = i (site i, spin up) and a = N + i (site i, spin down), i = x + L*y on an
 *   L x L periodic lattice, N = L*L.  H0 = sum_k c_k^+ h_k c_k with
 *   h_k = [[eps_k, conj(L_k)], [L_k, eps_k]], eps_k = -2t(cos kx + cos ky),
 *   L_k = 2 lam (sin ky - i sin kx) (the coefficient of c_{k,dn}^+ c_{k,up}).
 *   Interaction U sum_i [n_iu n_id - (n_iu + n_id)/2], U <= 0, gamma = arccos(exp(dtau U / 2)),
 *   decoupled (afqmc_soc_params.hs) in
 *     the spin-y channel (AFQMC_SOC_HS_SY, Eq. HSspinSyDep): the field x_{l,i} = +-1 rotates the
 *       pair of orbitals (i, N + i) by A(x) = [[cos gx, sin gx], [-sin gx, cos gx]];
 *     the imaginary spin-z channel (AFQMC_SOC_HS_SZ, Eqs. HSspinDecomp, BIOpForHubbard): the pair
 *       takes the phases A(x) = diag(e^{i g x}, e^{-i g x}).  With lam = 0 and a trial state with
 *       P_dn = conj(P_up) this is the paper's attractive Hubbard model (Sec. II.B), sign-free, with
 *       G_dn = conj(G_up) and no spin-mixing block.
 *   B_l = D(x_l) exp(-dtau H0), D(x_l) = (+)_i A(x_{l,i}).
 *   G_ab = <c_a c_b^+>, A = 1 - G.  Updates are rank 2 per site: with S = {i, N + i},
 *   delta = A(-x) A(x)^{-1} - 1 (the flip), the ratio is R = det(1_2 + delta A_SS)
 *   (Eqs. DetRatioSOC, LocalSOC) and G' = G - G[:, S] W (E_S^T - G[S, :]),
 *   W = delta (1 + A_SS delta)^{-1}.
 *
 * Complex matrices crossing the ABI are dense row-major with interleaved (re, im) doubles.
 * Ownership, streams, thread safety and error codes are those of afqmc.h: every call returns
 * 0 or a negative AFQMC_ERR_*; errors other than ARG / STATE are sticky.
 */
#ifndef AFQMC_SOC_H
#define AFQMC_SOC_H

#include <stdint.h>

#include "afqmc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct afqmc_soc_ctx afqmc_soc_ctx;

typedef struct {
    int L;              /* linear lattice size, 2 <= L <= 48 (N = L*L sites, 2N orbitals) */
    int M;              /* imaginary-time slices */
    int n_e;            /* particles: columns of the trial determinant, 1 <= n_e <= 2N */
    int n_walkers;      /* walkers, all on this lattice */
    int precision;      /* AFQMC_PREC_FP64 (parity) or AFQMC_PREC_FP32 (bulk G in complex64) */
    int gemm;           /* FP32 only: AFQMC_GEMM_* engine of the wrap products */
    int stab_every;     /* slices between FP64 re-orthonormalisations / recomputes; divides M */
    double t;           /* nearest-neighbour hopping */
    double lam;         /* Rashba spin-orbit coupling lambda */
    double U;           /* Hubbard U <= 0 (the spin-y decoupling) */
    double dtau;        /* imaginary-time step */
    uint64_t seed;      /* Philox4x64-10 key word 0 (word 1 = walker index) */
    int hs;             /* AFQMC_SOC_HS_SY (0, the default) or AFQMC_SOC_HS_SZ (1) */
} afqmc_soc_params;

#define AFQMC_SOC_HS_SY 0
#define AFQMC_SOC_HS_SZ 1

/* Largest window (sites) of the delayed update, and largest block of the block force-bias
 * update, per bulk precision. */
#define AFQMC_SOC_KMAX_FP32 64
#define AFQMC_SOC_KMAX_FP64 32

/* Create a context and build its constants: exp(-+dtau H0) from the closed-form 2 x 2
 * exponential of h_k, in the bulk precision.  p is copied.  AFQMC_ERR_ARG for sizes out of
 * range, U > 0, an unknown hs, or stab_every not dividing M; AFQMC_ERR_NODEV without an sm_103
 * device. */
int afqmc_soc_create(afqmc_soc_ctx** out, const afqmc_soc_params* p);

/* Free every resource of the context.  NULL is a no-op. */
int afqmc_soc_destroy(afqmc_soc_ctx* ctx);

/* Initialise the walkers (Appendix A, Eq. TrialWvfcCouple; Sec. II.B).
 *   P       host, caller-owned: the 2N x n_e trial determinant (complex, shared by the walkers).
 *   fields  host, nullable: n_walkers x M x N int8 (+-1), concatenated; NULL draws i.i.d. +-1
 *           fields from Philox(seed, walker).
 * Builds the left-factor stack in FP64 (re-orthonormalised every stab_every slices) and G(0),
 * stored in the bulk precision.  Walkers start at slice 0, forward. */
int afqmc_soc_init(afqmc_soc_ctx* ctx, const double* P, const int8_t* fields, void* stream);

/* One slice of the sweep for every walker, in the order of afqmc_sweep_slice:
 *   dir = +1: wrap G(l-1) -> G(l) = B_l G B_l^{-1}, then update slice l;
 *   dir = -1: update slice l, then wrap G(l) -> G(l-1) = B_l^{-1} G B_l.
 *   mode  AFQMC_MODE_LOCAL (rank-2 update of G per accepted site), AFQMC_MODE_DELAYED (windows
 *         of k sites, 1 <= k <= KMAX: decisions on the window's 2k x 2k block, one rank-2m
 *         product per window), AFQMC_MODE_BLOCKFB (blocks of nb sites, 1 <= nb <= KMAX:
 *         stripped force bias of the decoupling channel -- h_i = gamma Re<g_i> with g the field's
 *         generator, spin-y <c+_up c_dn - c+_dn c_up>, spin-z i <n_up - n_dn> -- joint proposal,
 *         one ratio and one rank-2m product per block; Sec. III.B).
 *   replay  host, nullable, 2N bytes per walker: local / delayed replay[i] = accept site i;
 *         block FB replay[i] = propose x'_i = +1 (else -1), replay[N + b] = accept block b.
 * Uniforms: Philox4x64-10, key (seed, walker), counter (j + 1, visit, 0, 0), visit = the number
 * of earlier afqmc_soc_sweep_slice calls; j < N site uniforms (Metropolis test or proposal),
 * j = N + b block acceptance.  Metropolis: accept iff u < |R|.  Returns AFQMC_ERR_STATE when
 * the walkers are not at slice l-1 (forward) / l (backward) or a recompute is due. */
int afqmc_soc_sweep_slice(afqmc_soc_ctx* ctx, int slice, int dir, int mode, int k, int nb, const uint8_t* replay,
                          void* stream);

/* FP64 recompute of G at the current slice (must be a multiple of stab_every):
 * G = 1 - U_R (U_L U_R)^{-1} U_L with the factor of the side just swept propagated from the
 * previous re-orthonormalisation point and re-orthonormalised (pivoted LU of its realified
 * form).  rel_drift (host, nullable, one per walker): ||G_bulk - G_new||_F / ||G_new||_F. */
int afqmc_soc_recompute_G(afqmc_soc_ctx* ctx, double* rel_drift, void* stream);

/* Mixed-estimator energy of every walker with the spin-coupled Wick contraction:
 * E = tr(H0 A) + U sum_i [A_ii A_{N+i,N+i} - A_{N+i,i} A_{i,N+i} - (A_ii + A_{N+i,N+i})/2].
 * energy: host, 2 doubles (re, im) per walker.  Syncs the stream. */
int afqmc_soc_measure_energy(afqmc_soc_ctx* ctx, double* energy, void* stream);

/* Pairing observables of Sec. IV for every walker, mixed estimator at the current slice from the
 * bulk G by the spin-coupled Wick contraction, in FP64 (A = 1 - G, A_ab = <c_b^+ c_a>; u = i, d = N + i):
 *   D = N^{-1} sum_i <n_iu n_id>,  <n_iu n_id> = A_uu A_dd - A_du A_ud (the double occupancy);
 *   <Delta^2> = L^{-2} sum_r P(r), P(r) = L^{-2} sum_i <D+_i D_{i+r} + D_i D+_{i+r}> / 4 (the on-site
 *     pairing correlator), D+_i = c+_iu c+_id, <D+_i D_j> = A_{ju,iu} A_{jd,id} - A_{jd,iu} A_{ju,id},
 *     <D_i D+_j> = G_{iu,ju} G_{id,jd} - G_{id,ju} G_{iu,jd};
 *   in momentum space (c_ks = N^{-1/2} sum_j e^{-i k.r_j} c_js, k = 2 pi (nx, ny) / L, index nx + L ny,
 *   At = F2 A F2^+ with F2 the DFT on each spin block): <n_ku> = At_{ku,ku}, <n_kd> = At_{kd,kd}, and
 *   the pairing matrix Mk[k][k'] = <D+_k D_k'>, D+_k = c+_{k u} c+_{-k d},
 *     = At_{k'u,ku} At_{-k'd,-kd} - At_{-k'd,ku} At_{k'u,-kd}.
 * The condensate fraction n_c is the largest eigenvalue of the Monte Carlo average of
 * Mk[k][k'] - delta_kk' <n_ku> <n_{-k d}>, divided by N_e / 2 (Sec. IV); the averaging is the caller's.
 *   scalars  host, 4 doubles per walker: Re D, Im D, Re <Delta^2>, Im <Delta^2>.
 *   nk       host, nullable: 4N doubles per walker, <n_ku> (N complex) then <n_kd> (N complex).
 *   Mk       host, nullable: N x N complex (re, im interleaved) per walker.
 * The first call allocates the DFT tables (2 x (2 ldz)^2 + 2N 2 ldz doubles, ldz = 2N rounded up to
 * 32) and scratch of the same order.  Syncs the stream.  AFQMC_ERR_ARG before init or for a NULL
 * scalars. */
int afqmc_soc_measure_pairing(afqmc_soc_ctx* ctx, double* scalars, double* nk, double* Mk, void* stream);

/* Accessors (sync the stream of the last call). *//* Accessors (sync the stream of the last call). */
int afqmc_soc_get_G(afqmc_soc_ctx* ctx, int walker, double* host_out);       /* 2N x 2N complex */
int afqmc_soc_set_G(afqmc_soc_ctx* ctx, int walker, const double* host_in);  /* 2N x 2N complex */
int afqmc_soc_get_fields(afqmc_soc_ctx* ctx, int walker, int8_t* host_out);  /* M x N */
int afqmc_soc_get_decisions(afqmc_soc_ctx* ctx, int walker, uint8_t* host_out);  /* 2N, replay layout */
int afqmc_soc_get_ratios(afqmc_soc_ctx* ctx, int walker, double* host_out);  /* 2N complex: site i / N + block */
int afqmc_soc_get_lam_plus(afqmc_soc_ctx* ctx, int walker, double* host_out);  /* N: block FB P(x' = +1) */
int afqmc_soc_get_info(afqmc_soc_ctx* ctx, int* N, int* slice, int* dir);

/* Profiling: per-phase device time with the AFQMC_PHASE_* ids of afqmc.h (WRAP, CHAIN, FLUSH,
 * RECOMPUTE and their sub-phases), as in afqmc_set_profiling / afqmc_get_profile. */
int afqmc_soc_set_profiling(afqmc_soc_ctx* ctx, int on);
int afqmc_soc_get_profile(afqmc_soc_ctx* ctx, double* ms, int64_t* intervals, int64_t* launches);

#ifdef __cplusplus
}
#endif

#endif /* AFQMC_SOC_H */
