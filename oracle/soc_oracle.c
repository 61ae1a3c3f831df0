/*
 * soc_oracle.c -- plain, slow, FP64 complex CPU oracle for the spin-orbit-coupled Hubbard
 * model (Appendix A of the paper): the same PQMC sweep on the 2N x 2N complex G.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference legs of bench.py may load this file.  It shares no code, header, table or
 * constant with the CUDA library.
 *
 * Conventions (Appendix A, Eqs. 2DSocHubbard, HSspinSyDep, A2times2, DetRatioSOC):
 *   orbitals a = i (spin up, site i) and a = N + i (spin down); N = L*L sites, i = x + L*y.
 *   H0 = sum_k c_k^+ h_k c_k with h_k = [[eps_k, conj(L_k)], [L_k, eps_k]] in (up, down),
 *        eps_k = -2t(cos kx + cos ky), L_k = 2 lam (sin ky - i sin kx) the coefficient of
 *        c_{k,down}^+ c_{k,up}.
 *   G_ab = <c_a c_b^+>, A = 1 - G, A_ab = <c_b^+ c_a>.
 *   HS (U < 0, uniform prior 1/2, gamma = arccos(exp(dtau U / 2))): the field x_i = +-1 acts on
 *   the pair (i, N + i) with the 2 x 2 matrix A(gamma x_i), A(t) = exp(t g) for the generator g
 *   of the decoupling channel:
 *     spin-y (hs = 0, Eq. HSspinSyDep):  g = [[0, 1], [-1, 0]],  A(t) = [[cos t, sin t], [-sin t, cos t]];
 *     spin-z (hs = 1, Eqs. HSspinDecomp, BIOpForHubbard, the imaginary s^z channel of the Hubbard
 *             model): g = diag(i, -i),  A(t) = diag(e^{it}, e^{-it}).
 *   Both satisfy A(t) A(t') = A(t + t').  With lam = 0 and hs = 1 this is the paper's attractive
 *   Hubbard model: G stays block diagonal in spin with G_dn = conj(G_up).
 *   B_l = D_l E with D_l = (+)_i A(gamma x_{l,i}) and E = exp(-dtau H0).
 *   Matrices are row-major double complex.
 *
 * G form of the updates (Eq. GrFMatNew: G = 1 - U_R T U_L):
 *   flip at site i, S = {i, N + i}: delta = A(x')A(x)^{-1} - 1 = A(x' - x) - 1 (2 x 2),
 *   R = det(1_2 + delta A_SS)                                      (Eqs. DetRatioSOC, LocalSOC)
 *   G' = G - G[:, S] W (E_S^T - G[S, :]),  W = delta (1_2 + A_SS delta)^{-1}.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

typedef struct {
    int L, N;           /* N sites, 2N orbitals */
    double t, lam, U, dtau;
    double gamma;       /* HS coupling */
    int hs;             /* 0: spin-y channel, 1: spin-z channel (imaginary coupling) */
} soc_params;

/* gamma = arccos(exp(dtau U / 2)) (Eqs. HSspinSyDep, HSspinDecomp); needs U <= 0 (U = 0 gives
 * gamma = 0, the free system) and hs in {0, 1}.  Returns 0 or -1. */
int soc_setup(soc_params* p) {
    p->N = p->L * p->L;
    if (!(p->U <= 0.0) || (p->hs != 0 && p->hs != 1)) return -1;
    p->gamma = acos(exp(p->dtau * p->U / 2.0));
    return 0;
}

/* The 2 x 2 block h_k in (up, down). */
static void soc_hk(const soc_params* p, int nx, int ny, cplx h[2][2]) {
    const double kx = 2.0 * M_PI * nx / p->L, ky = 2.0 * M_PI * ny / p->L;
    const double eps = -2.0 * p->t * (cos(kx) + cos(ky));
    const cplx Lk = 2.0 * p->lam * (sin(ky) - I * sin(kx));
    h[0][0] = eps;
    h[1][1] = eps;
    h[1][0] = Lk;        /* <down| h |up> */
    h[0][1] = conj(Lk);
}

/* exp(-tau h_k) in closed form: h_k = eps + [[0, conj L], [L, 0]], whose off-diagonal part
 * squares to |L|^2, so exp(-tau h_k) = e^{-tau eps} (cosh(tau|L|) - sinh(tau|L|)/|L| offdiag). */
static void soc_expk(const soc_params* p, int nx, int ny, double tau, cplx e[2][2]) {
    cplx h[2][2];
    soc_hk(p, nx, ny, h);
    const double eps = creal(h[0][0]);
    const double a = cabs(h[1][0]);
    const double c = cosh(tau * a), sh = (a > 0.0) ? sinh(tau * a) / a : tau;
    const double f = exp(-tau * eps);
    e[0][0] = f * c;
    e[1][1] = f * c;
    e[1][0] = -f * sh * h[1][0];
    e[0][1] = -f * sh * h[0][1];
}

/* Real-space matrix M_{a b} = N^{-1} sum_k e^{i k.(r_i - r_j)} m_k[s_a][s_b] for a = (s_a, i),
 * b = (s_b, j), from the per-k blocks in mk[(nx + L ny)][2][2]. */
static void soc_from_k(const soc_params* p, const cplx (*mk)[2][2], cplx* M) {
    const int L = p->L, N = p->N, N2 = 2 * N;
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
            const int dx = i % L - j % L, dy = i / L - j / L;
            cplx acc[2][2] = {{0, 0}, {0, 0}};
            for (int ny = 0; ny < L; ny++)
                for (int nx = 0; nx < L; nx++) {
                    const double ph = 2.0 * M_PI * ((double)nx * dx + (double)ny * dy) / L;
                    const cplx e = cos(ph) + I * sin(ph);
                    const cplx(*m)[2] = mk[nx + L * ny];
                    for (int a = 0; a < 2; a++)
                        for (int b = 0; b < 2; b++) acc[a][b] += e * m[a][b];
                }
            for (int a = 0; a < 2; a++)
                for (int b = 0; b < 2; b++) M[(size_t)(a * N + i) * N2 + (b * N + j)] = acc[a][b] / N;
        }
}

/* H0 (2N x 2N), Eq. 2DSocHubbard. */
void soc_H0(const soc_params* p, cplx* H) {
    const int L = p->L;
    cplx(*hk)[2][2] = malloc((size_t)L * L * sizeof(*hk));
    for (int ny = 0; ny < L; ny++)
        for (int nx = 0; nx < L; nx++) soc_hk(p, nx, ny, hk[nx + L * ny]);
    soc_from_k(p, (const cplx(*)[2][2])hk, H);
    free(hk);
}

/* exp(-tau H0) (2N x 2N). */
void soc_expH(const soc_params* p, double tau, cplx* E) {
    const int L = p->L;
    cplx(*ek)[2][2] = malloc((size_t)L * L * sizeof(*ek));
    for (int ny = 0; ny < L; ny++)
        for (int nx = 0; nx < L; nx++) soc_expk(p, nx, ny, tau, ek[nx + L * ny]);
    soc_from_k(p, (const cplx(*)[2][2])ek, E);
    free(ek);
}

/* The decoupling's 2 x 2 matrix A(theta) on the pair (i, N + i), theta = gamma x. */
static void site_mat(const soc_params* p, double theta, cplx r[2][2]) {
    if (p->hs == 1) {
        r[0][0] = cos(theta) + I * sin(theta);
        r[0][1] = 0;
        r[1][0] = 0;
        r[1][1] = cos(theta) - I * sin(theta);
        return;
    }
    r[0][0] = cos(theta);
    r[0][1] = sin(theta);
    r[1][0] = -sin(theta);
    r[1][1] = cos(theta);
}

/* ---------------- small dense complex linear algebra ---------------- */

/* C (n x m) = A (n x k) B (k x m), all row-major. */
static void zgemm(const cplx* A, const cplx* B, cplx* C, int n, int k, int m) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; i++) {
        for (int j = 0; j < m; j++) C[(size_t)i * m + j] = 0;
        for (int q = 0; q < k; q++) {
            const cplx a = A[(size_t)i * k + q];
            for (int j = 0; j < m; j++) C[(size_t)i * m + j] += a * B[(size_t)q * m + j];
        }
    }
}

/* In-place LU with partial pivoting of the n x n a; returns log|det| in *logabs and the phase
 * of det (0 for a singular matrix). */
static cplx zlu_factor(cplx* a, int n, int* piv, double* logabs) {
    cplx ph = 1.0;
    double la = 0.0;
    for (int k = 0; k < n; k++) {
        int pr = k;
        double best = cabs(a[(size_t)k * n + k]);
        for (int r = k + 1; r < n; r++)
            if (cabs(a[(size_t)r * n + k]) > best) { best = cabs(a[(size_t)r * n + k]); pr = r; }
        piv[k] = pr;
        if (best == 0.0) { *logabs = -INFINITY; return 0; }
        if (pr != k) {
            for (int c = 0; c < n; c++) {
                cplx tmp = a[(size_t)k * n + c];
                a[(size_t)k * n + c] = a[(size_t)pr * n + c];
                a[(size_t)pr * n + c] = tmp;
            }
            ph = -ph;
        }
        const cplx d = a[(size_t)k * n + k];
        ph *= d / cabs(d);
        la += log(cabs(d));
#pragma omp parallel for schedule(static)
        for (int r = k + 1; r < n; r++) {
            const cplx l = a[(size_t)r * n + k] / d;
            a[(size_t)r * n + k] = l;
            for (int c = k + 1; c < n; c++) a[(size_t)r * n + c] -= l * a[(size_t)k * n + c];
        }
    }
    *logabs = la;
    return ph;
}

/* Solve a x = b for nrhs right-hand sides (b: n x nrhs row-major, overwritten). */
static void zlu_solve(const cplx* lu, int n, const int* piv, cplx* b, int nrhs) {
    for (int k = 0; k < n; k++)
        if (piv[k] != k)
            for (int c = 0; c < nrhs; c++) {
                cplx tmp = b[(size_t)k * nrhs + c];
                b[(size_t)k * nrhs + c] = b[(size_t)piv[k] * nrhs + c];
                b[(size_t)piv[k] * nrhs + c] = tmp;
            }
#pragma omp parallel for schedule(static)
    for (int c = 0; c < nrhs; c++) {
        for (int r = 0; r < n; r++)
            for (int q = 0; q < r; q++) b[(size_t)r * nrhs + c] -= lu[(size_t)r * n + q] * b[(size_t)q * nrhs + c];
        for (int r = n - 1; r >= 0; r--) {
            for (int q = r + 1; q < n; q++) b[(size_t)r * nrhs + c] -= lu[(size_t)r * n + q] * b[(size_t)q * nrhs + c];
            b[(size_t)r * nrhs + c] /= lu[(size_t)r * n + r];
        }
    }
}

/* Orthonormalise the n columns of the m x n matrix a (element (r, c) at a[r*rs + c*cs]) by
 * modified Gram-Schmidt, twice; *logabs += log|det R| of the discarded triangular factor and the
 * return value is its phase. */
static cplx zorth(cplx* a, int m, int n, size_t rs, size_t cs, double* logabs) {
    cplx ph = 1.0;
    for (int pass = 0; pass < 2; pass++)
        for (int c = 0; c < n; c++) {
            for (int q = 0; q < c; q++) {
                cplx d = 0;
                for (int r = 0; r < m; r++) d += conj(a[r * rs + q * cs]) * a[r * rs + c * cs];
                for (int r = 0; r < m; r++) a[r * rs + c * cs] -= d * a[r * rs + q * cs];
            }
            double nr = 0.0;
            for (int r = 0; r < m; r++) nr += creal(a[r * rs + c * cs] * conj(a[r * rs + c * cs]));
            nr = sqrt(nr);
            *logabs += log(nr);
            for (int r = 0; r < m; r++) a[r * rs + c * cs] /= nr;
        }
    return ph;  /* the factor R of modified Gram-Schmidt has a positive real diagonal */
}

/* v (2N x ncol, row-major) <- D(x) v: rows i and N + i mixed by A(sgn gamma x_i). */
static void rot_rows(const soc_params* p, const int8_t* xl, double sgn, cplx* v, int ncol) {
    const int N = p->N;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; i++) {
        cplx r[2][2];
        site_mat(p, sgn * p->gamma * xl[i], r);
        for (int c = 0; c < ncol; c++) {
            const cplx a = v[(size_t)i * ncol + c], b = v[(size_t)(N + i) * ncol + c];
            v[(size_t)i * ncol + c] = r[0][0] * a + r[0][1] * b;
            v[(size_t)(N + i) * ncol + c] = r[1][0] * a + r[1][1] * b;
        }
    }
}

/* v (nrow x 2N, row-major) <- v D(x): columns i and N + i. */
static void rot_cols(const soc_params* p, const int8_t* xl, double sgn, cplx* v, int nrow) {
    const int N = p->N, N2 = 2 * N;
#pragma omp parallel for schedule(static)
    for (int r0 = 0; r0 < nrow; r0++)
        for (int i = 0; i < N; i++) {
            cplx r[2][2];
            site_mat(p, sgn * p->gamma * xl[i], r);
            const cplx a = v[(size_t)r0 * N2 + i], b = v[(size_t)r0 * N2 + N + i];
            v[(size_t)r0 * N2 + i] = a * r[0][0] + b * r[1][0];
            v[(size_t)r0 * N2 + N + i] = a * r[0][1] + b * r[1][1];
        }
}

/* G(l) from scratch, Eq. GrFMat for spin-coupled systems (Appendix A):
 *   R = B_l ... B_1 P (2N x Ne), L = P^+ B_M ... B_{l+1} (Ne x 2N), G = 1 - R (L R)^{-1} L,
 * with the factors re-orthonormalised every `stab` slices.  Returns log|det(P^+ B_M...B_1 P)|
 * in *logabs and its phase in *phase. */
int soc_green_scratch(const soc_params* p, const cplx* E, const int8_t* x, int M, const cplx* P, int Ne, int ell,
                      int stab, cplx* G, double* logabs, cplx* phase) {
    const int N = p->N, N2 = 2 * N;
    cplx* R = malloc((size_t)N2 * Ne * sizeof(cplx));
    cplx* Lf = malloc((size_t)Ne * N2 * sizeof(cplx));
    cplx* tmp = malloc((size_t)N2 * (N2 > Ne ? N2 : Ne) * sizeof(cplx));
    double la = 0.0;
    cplx ph = 1.0;
    memcpy(R, P, (size_t)N2 * Ne * sizeof(cplx));
    for (int l = 1; l <= ell; l++) {
        zgemm(E, R, tmp, N2, N2, Ne);
        memcpy(R, tmp, (size_t)N2 * Ne * sizeof(cplx));
        rot_rows(p, x + (size_t)(l - 1) * N, 1.0, R, Ne);
        if (stab > 0 && l % stab == 0) ph *= zorth(R, N2, Ne, Ne, 1, &la);
    }
    for (int a = 0; a < Ne; a++)
        for (int b = 0; b < N2; b++) Lf[(size_t)a * N2 + b] = conj(P[(size_t)b * Ne + a]);
    for (int l = M; l > ell; l--) {
        rot_cols(p, x + (size_t)(l - 1) * N, 1.0, Lf, Ne);
        zgemm(Lf, E, tmp, Ne, N2, N2);
        memcpy(Lf, tmp, (size_t)Ne * N2 * sizeof(cplx));
        if (stab > 0 && (M - l + 1) % stab == 0) ph *= zorth(Lf, N2, Ne, 1, N2, &la);
    }
    cplx* O = malloc((size_t)Ne * Ne * sizeof(cplx));
    int* piv = malloc((size_t)Ne * sizeof(int));
    zgemm(Lf, R, O, Ne, N2, Ne);
    double lo = 0.0;
    const cplx pho = zlu_factor(O, Ne, piv, &lo);
    memcpy(tmp, Lf, (size_t)Ne * N2 * sizeof(cplx));
    zlu_solve(O, Ne, piv, tmp, N2);  /* (L R)^{-1} L */
    zgemm(R, tmp, G, N2, Ne, N2);
    for (size_t e = 0; e < (size_t)N2 * N2; e++) G[e] = -G[e];
    for (int a = 0; a < N2; a++) G[(size_t)a * N2 + a] += 1.0;
    if (logabs) *logabs = la + lo;
    if (phase) *phase = ph * pho;
    free(R);
    free(Lf);
    free(tmp);
    free(O);
    free(piv);
    return pho == 0 ? -1 : 0;
}

/* Wrap (Eqs. BlMat, GrFMat): forward G <- D E G E^{-1} D^{-1}; backward G <- E^{-1} D^{-1} G D E,
 * with D = D(x_l), D^{-1} = D(-x_l). */
void soc_wrap(const soc_params* p, const cplx* E, const cplx* Einv, const int8_t* xl, cplx* G, int dir) {
    const int N2 = 2 * p->N;
    cplx* T = malloc((size_t)N2 * N2 * sizeof(cplx));
    if (dir > 0) {
        zgemm(E, G, T, N2, N2, N2);
        zgemm(T, Einv, G, N2, N2, N2);
        rot_rows(p, xl, 1.0, G, N2);
        rot_cols(p, xl, -1.0, G, N2);
    } else {
        rot_rows(p, xl, -1.0, G, N2);
        rot_cols(p, xl, 1.0, G, N2);
        zgemm(Einv, G, T, N2, N2, N2);
        zgemm(T, E, G, N2, N2, N2);
    }
    free(T);
}

/* det of a 2 x 2 and the inverse */
static cplx det2(const cplx m[2][2]) { return m[0][0] * m[1][1] - m[0][1] * m[1][0]; }

/* The flip at site i: delta = A(-2x) - 1, ratio R = det(1 + delta A_SS) and W = delta (1 + A_SS delta)^{-1},
 * from the current 2 x 2 block g of G on (i, N + i). */
static cplx flip_ratio(const soc_params* p, int x, const cplx g[2][2], cplx W[2][2]) {
    cplx r[2][2];
    site_mat(p, -2.0 * p->gamma * x, r);
    const cplx dl[2][2] = {{r[0][0] - 1.0, r[0][1]}, {r[1][0], r[1][1] - 1.0}};
    cplx Ass[2][2];
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) Ass[a][b] = (a == b ? 1.0 : 0.0) - g[a][b];
    cplx m1[2][2], m2[2][2];  /* 1 + delta A, 1 + A delta */
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) {
            m1[a][b] = (a == b ? 1.0 : 0.0) + dl[a][0] * Ass[0][b] + dl[a][1] * Ass[1][b];
            m2[a][b] = (a == b ? 1.0 : 0.0) + Ass[a][0] * dl[0][b] + Ass[a][1] * dl[1][b];
        }
    const cplx R = det2(m1);
    const cplx d2 = det2(m2);
    const cplx inv[2][2] = {{m2[1][1] / d2, -m2[0][1] / d2}, {-m2[1][0] / d2, m2[0][0] / d2}};
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) W[a][b] = dl[a][0] * inv[0][b] + dl[a][1] * inv[1][b];
    return R;
}

/* G <- G - G[:, S] W (E_S^T - G[S, :]), S = (i, N + i). */
static void apply_rank2(int N2, int i, int Ni, const cplx W[2][2], cplx* G) {
    cplx* X = malloc((size_t)N2 * 2 * sizeof(cplx));
    cplx* Y = malloc((size_t)2 * N2 * sizeof(cplx));
    const int S[2] = {i, Ni};
    for (int r = 0; r < N2; r++)
        for (int b = 0; b < 2; b++) X[(size_t)r * 2 + b] = G[(size_t)r * N2 + S[0]] * W[0][b] + G[(size_t)r * N2 + S[1]] * W[1][b];
    for (int a = 0; a < 2; a++)
        for (int c = 0; c < N2; c++) Y[(size_t)a * N2 + c] = (c == S[a] ? 1.0 : 0.0) - G[(size_t)S[a] * N2 + c];
#pragma omp parallel for schedule(static)
    for (int r = 0; r < N2; r++)
        for (int c = 0; c < N2; c++) G[(size_t)r * N2 + c] -= X[(size_t)r * 2] * Y[c] + X[(size_t)r * 2 + 1] * Y[N2 + c];
    free(X);
    free(Y);
}

/* Local update of one slice (Eqs. DetRatioSOC, UpdateLTRSOC, LocalSOC in G form): sites i = 0..N-1
 * in order; accept iff u[i] < |R| (Metropolis, uniform prior); on accept flip x and apply the
 * rank-2 update.  replay (nullable): replay[i] forces the decision at site i.
 * dec[i] = accepted, ratio[2i], ratio[2i+1] = Re, Im of R. */
void soc_local_slice(const soc_params* p, cplx* G, int8_t* xl, const double* u, const uint8_t* replay, uint8_t* dec,
                     double* ratio) {
    const int N = p->N, N2 = 2 * N;
    for (int i = 0; i < N; i++) {
        cplx g[2][2] = {{G[(size_t)i * N2 + i], G[(size_t)i * N2 + N + i]},
                        {G[(size_t)(N + i) * N2 + i], G[(size_t)(N + i) * N2 + N + i]}};
        cplx W[2][2];
        const cplx R = flip_ratio(p, xl[i], g, W);
        ratio[2 * i] = creal(R);
        ratio[2 * i + 1] = cimag(R);
        const int acc = replay ? (replay[i] != 0) : (u[i] < cabs(R));
        dec[i] = (uint8_t)acc;
        if (!acc) continue;
        apply_rank2(N2, i, N + i, W, G);
        xl[i] = (int8_t)(-xl[i]);
    }
}

/* Delayed update of one slice (Appendix A: the delayed scheme with N_e x 2 and 2 x N_e vectors per
 * accepted site, here in G form): windows of k consecutive sites.  Within a window, the current
 * column pair and row pair of site i are those of G0 plus the buffered rank-2 terms a_m b_m; an
 * accepted site appends a_m = -(current G[:, S]) W and b_m = E_S^T - current G[S, :]; the window
 * ends with G0 <- G0 + sum_m a_m b_m.  Same decisions and ratios as the local update. */
void soc_delayed_slice(const soc_params* p, cplx* G, int8_t* xl, const double* u, int k, const uint8_t* replay,
                       uint8_t* dec, double* ratio) {
    const int N = p->N, N2 = 2 * N;
    if (k < 1) k = 1;
    cplx* A = malloc((size_t)N2 * 2 * k * sizeof(cplx));  /* a_m as columns 2m, 2m+1 */
    cplx* B = malloc((size_t)2 * k * N2 * sizeof(cplx));  /* b_m as rows 2m, 2m+1 */
    cplx* col = malloc((size_t)N2 * 2 * sizeof(cplx));
    cplx* row = malloc((size_t)2 * N2 * sizeof(cplx));
    for (int s0 = 0; s0 < N; s0 += k) {
        const int n = (N - s0 < k) ? N - s0 : k;
        int m = 0;
        for (int q = 0; q < n; q++) {
            const int i = s0 + q;
            const int S[2] = {i, N + i};
            for (int r = 0; r < N2; r++)
                for (int b = 0; b < 2; b++) {
                    cplx v = G[(size_t)r * N2 + S[b]];
                    for (int mm = 0; mm < 2 * m; mm++) v += A[(size_t)r * 2 * k + mm] * B[(size_t)mm * N2 + S[b]];
                    col[(size_t)r * 2 + b] = v;
                }
            for (int a = 0; a < 2; a++)
                for (int c = 0; c < N2; c++) {
                    cplx v = G[(size_t)S[a] * N2 + c];
                    for (int mm = 0; mm < 2 * m; mm++) v += A[(size_t)S[a] * 2 * k + mm] * B[(size_t)mm * N2 + c];
                    row[(size_t)a * N2 + c] = v;
                }
            cplx g[2][2] = {{col[(size_t)S[0] * 2], col[(size_t)S[0] * 2 + 1]},
                            {col[(size_t)S[1] * 2], col[(size_t)S[1] * 2 + 1]}};
            cplx W[2][2];
            const cplx R = flip_ratio(p, xl[i], g, W);
            ratio[2 * i] = creal(R);
            ratio[2 * i + 1] = cimag(R);
            const int acc = replay ? (replay[i] != 0) : (u[i] < cabs(R));
            dec[i] = (uint8_t)acc;
            if (!acc) continue;
            for (int r = 0; r < N2; r++)
                for (int b = 0; b < 2; b++)
                    A[(size_t)r * 2 * k + 2 * m + b] = -(col[(size_t)r * 2] * W[0][b] + col[(size_t)r * 2 + 1] * W[1][b]);
            for (int a = 0; a < 2; a++)
                for (int c = 0; c < N2; c++)
                    B[(size_t)(2 * m + a) * N2 + c] = (c == S[a] ? 1.0 : 0.0) - row[(size_t)a * N2 + c];
            xl[i] = (int8_t)(-xl[i]);
            m++;
        }
#pragma omp parallel for schedule(static)
        for (int r = 0; r < N2; r++)
            for (int c = 0; c < N2; c++) {
                cplx v = 0;
                for (int q = 0; q < 2 * m; q++) v += A[(size_t)r * 2 * k + q] * B[(size_t)q * N2 + c];
                G[(size_t)r * N2 + c] += v;
            }
    }
    free(A);
    free(B);
    free(col);
    free(row);
}

/* The orbital list of a set of sites: F = (i_1 .. i_n, N + i_1 .. N + i_n). */
static void orbitals(int N, const int* sites, int n, int* F) {
    for (int a = 0; a < n; a++) {
        F[a] = sites[a];
        F[n + a] = N + sites[a];
    }
}

/* Delta on the orbitals of `sites` for the moves x -> xnew (block diagonal in the site pairs):
 * Delta[(a, n+a) x (a, n+a)] = A(xnew_a) A(x_a)^{-1} - 1 = A(xnew_a - x_a) - 1; dim 2n. */
static void delta_block(const soc_params* p, const int8_t* x, const int8_t* xnew, int n, cplx* D) {
    const int n2 = 2 * n;
    for (int e = 0; e < n2 * n2; e++) D[e] = 0;
    for (int a = 0; a < n; a++) {
        cplx r[2][2];
        site_mat(p, p->gamma * ((double)xnew[a] - (double)x[a]), r);
        const int o[2] = {a, n + a};
        for (int s = 0; s < 2; s++)
            for (int t = 0; t < 2; t++) D[o[s] * n2 + o[t]] = r[s][t] - (s == t ? 1.0 : 0.0);
    }
}

/* Stripped force bias of the block of sites [s0, s0 + n) (Appendix A with Eq. BlkFrcBsTnew1 in G form):
 * with the block's current fields taken out of R, Delta_b = A(-x) - 1 on the block orbitals, the
 * stripped one-body matrix on the block is  Abar = (1 + Delta_b)(1 + A_bb Delta_b)^{-1} A_bb  (A = 1 - G),
 * and obar_i is the stripped expectation of the field's generator g on site i (the field enters
 * as exp(gamma x g)), which sets the bias:
 *   spin-y: obar_i = <c+_{i,up} c_{i,dn}> - <c+_{i,dn} c_{i,up}> = Abar[dn i, up i] - Abar[up i, dn i];
 *   spin-z: obar_i = i (<n_{i,up}> - <n_{i,dn}>) = i (Abar[up i, up i] - Abar[dn i, dn i]).
 * obar holds n complex values. */
void soc_block_force_bias(const soc_params* p, const cplx* G, const int8_t* xl, int s0, int n, cplx* obar) {
    const int N = p->N, N2 = 2 * N, n2 = 2 * n;
    int* sites = malloc((size_t)n * sizeof(int));
    int* F = malloc((size_t)n2 * sizeof(int));
    int8_t* zero = calloc((size_t)n, 1);
    cplx* D = malloc((size_t)n2 * n2 * sizeof(cplx));
    cplx* Abb = malloc((size_t)n2 * n2 * sizeof(cplx));
    cplx* Mx = malloc((size_t)n2 * n2 * sizeof(cplx));
    int* piv = malloc((size_t)n2 * sizeof(int));
    for (int a = 0; a < n; a++) sites[a] = s0 + a;
    orbitals(N, sites, n, F);
    delta_block(p, xl + s0, zero, n, D); /* A(0 - x) - 1 */
    for (int a = 0; a < n2; a++)
        for (int b = 0; b < n2; b++) Abb[a * n2 + b] = (a == b ? 1.0 : 0.0) - G[(size_t)F[a] * N2 + F[b]];
    for (int a = 0; a < n2; a++)
        for (int b = 0; b < n2; b++) {
            cplx v = (a == b ? 1.0 : 0.0);
            for (int q = 0; q < n2; q++) v += Abb[a * n2 + q] * D[q * n2 + b];
            Mx[a * n2 + b] = v;
        }
    double la;
    zlu_factor(Mx, n2, piv, &la);
    zlu_solve(Mx, n2, piv, Abb, n2); /* Abb <- (1 + A Delta)^{-1} A */
    for (int a = 0; a < n; a++) {
        /* rows dn a and up a of (1 + Delta) Abb */
        cplx dn_up = Abb[(n + a) * n2 + a], up_dn = Abb[a * n2 + n + a];
        cplx up_up = Abb[a * n2 + a], dn_dn = Abb[(n + a) * n2 + n + a];
        for (int q = 0; q < n2; q++) {
            dn_up += D[(n + a) * n2 + q] * Abb[q * n2 + a];
            up_dn += D[a * n2 + q] * Abb[q * n2 + n + a];
            up_up += D[a * n2 + q] * Abb[q * n2 + a];
            dn_dn += D[(n + a) * n2 + q] * Abb[q * n2 + n + a];
        }
        obar[a] = p->hs == 1 ? I * (up_up - dn_dn) : dn_up - up_dn;
    }
    free(sites); free(F); free(zero); free(D); free(Abb); free(Mx); free(piv);
}

/* Block force-bias update of one slice (Sec. III.B with the bias of the decoupling channel), blocks of
 * nb consecutive sites (the last one partial).  Per block: h_i = gamma Re(obar_i); proposal
 * lambda(x') = e^{x' h} / (e^{h} + e^{-h}) drawn with u_prop[i] (x' = +1 iff u_prop[i] < lambda(+1));
 * on the flipped set F the Metropolis ratio is
 *   R = det(1 + Delta_F A_FF) * prod_{i in F} e^{(x_i - x'_i) h_i}
 * (uniform prior; the product is the proposal ratio P(X'->X)/P(X->X')), accepted iff u_acc[b] < |R|,
 * and G <- G - G[:, F] W (E_F^T - G[F, :]), W = Delta_F (1 + A_FF Delta_F)^{-1}.
 * replay (nullable): replay[i] = 1 proposes x'_i = +1; replay[N + b] forces block b's decision.
 * Outputs xprop[i], lam_plus[i], dec[b], ratio[2b], ratio[2b+1] (Re, Im of R). */
void soc_blockfb_slice(const soc_params* p, cplx* G, int8_t* xl, const double* u_prop, const double* u_acc, int nb,
                       const uint8_t* replay, int8_t* xprop, double* lam_plus, uint8_t* dec, double* ratio) {
    const int N = p->N, N2 = 2 * N;
    if (nb < 1) nb = 1;
    const int nblocks = (N + nb - 1) / nb;
    cplx* obar = malloc((size_t)nb * sizeof(cplx));
    int* Fs = malloc((size_t)nb * sizeof(int));
    int* F = malloc((size_t)2 * nb * sizeof(int));
    int8_t* xf = malloc((size_t)nb);
    int8_t* xn = malloc((size_t)nb);
    cplx* D = malloc((size_t)4 * nb * nb * sizeof(cplx));
    cplx* Mf = malloc((size_t)4 * nb * nb * sizeof(cplx));
    cplx* Wm = malloc((size_t)4 * nb * nb * sizeof(cplx));
    int* piv = malloc((size_t)2 * nb * sizeof(int));
    cplx* X = malloc((size_t)N2 * 2 * nb * sizeof(cplx));
    cplx* Y = malloc((size_t)2 * nb * N2 * sizeof(cplx));
    cplx* XW = malloc((size_t)N2 * 2 * nb * sizeof(cplx));
    for (int bk = 0; bk < nblocks; bk++) {
        const int s0 = bk * nb, n = (s0 + nb <= N) ? nb : N - s0;
        soc_block_force_bias(p, G, xl, s0, n, obar);
        double logq = 0.0;
        int nF = 0;
        for (int a = 0; a < n; a++) {
            const int i = s0 + a;
            const double h = p->gamma * creal(obar[a]);
            const double lamp = 1.0 / (1.0 + exp(-2.0 * h));
            lam_plus[i] = lamp;
            const int xp = replay ? (replay[i] ? +1 : -1) : (u_prop[i] < lamp ? +1 : -1);
            xprop[i] = (int8_t)xp;
            if (xp != xl[i]) {
                Fs[nF] = i;
                xf[nF] = xl[i];
                xn[nF] = (int8_t)xp;
                nF++;
                logq += (double)(xl[i] - xp) * h;
            }
        }
        if (nF == 0) { /* the proposal is the current state */
            dec[bk] = 1;
            ratio[2 * bk] = 1.0;
            ratio[2 * bk + 1] = 0.0;
            continue;
        }
        const int f2 = 2 * nF;
        orbitals(N, Fs, nF, F);
        delta_block(p, xf, xn, nF, D);
        /* Mf = 1 + A_FF Delta_F */
        for (int a = 0; a < f2; a++)
            for (int b = 0; b < f2; b++) {
                cplx v = (a == b ? 1.0 : 0.0);
                for (int q = 0; q < f2; q++)
                    v += ((a == q ? 1.0 : 0.0) - G[(size_t)F[a] * N2 + F[q]]) * D[q * f2 + b];
                Mf[a * f2 + b] = v;
            }
        double la;
        const cplx ph = zlu_factor(Mf, f2, piv, &la); /* det(1 + A Delta) = det(1 + Delta A) */
        const cplx R = (ph == 0) ? 0 : ph * exp(la + logq);
        ratio[2 * bk] = creal(R);
        ratio[2 * bk + 1] = cimag(R);
        const int acc = replay ? (replay[N + bk] != 0) : (u_acc[bk] < cabs(R));
        dec[bk] = (uint8_t)acc;
        if (!acc) continue;
        /* W = Delta (1 + A Delta)^{-1} */
        for (int a = 0; a < f2; a++)
            for (int b = 0; b < f2; b++) Wm[a * f2 + b] = (a == b ? 1.0 : 0.0);
        zlu_solve(Mf, f2, piv, Wm, f2); /* Wm = Mf^{-1} */
        for (int a = 0; a < f2; a++)
            for (int b = 0; b < f2; b++) {
                cplx v = 0;
                for (int q = 0; q < f2; q++) v += D[a * f2 + q] * Wm[q * f2 + b];
                Mf[a * f2 + b] = v; /* W */
            }
        for (int r = 0; r < N2; r++)
            for (int a = 0; a < f2; a++) X[(size_t)r * f2 + a] = G[(size_t)r * N2 + F[a]];
        for (int a = 0; a < f2; a++)
            for (int c = 0; c < N2; c++) Y[(size_t)a * N2 + c] = (c == F[a] ? 1.0 : 0.0) - G[(size_t)F[a] * N2 + c];
        zgemm(X, Mf, XW, N2, f2, f2);
#pragma omp parallel for schedule(static)
        for (int r = 0; r < N2; r++)
            for (int c = 0; c < N2; c++) {
                cplx v = 0;
                for (int q = 0; q < f2; q++) v += XW[(size_t)r * f2 + q] * Y[(size_t)q * N2 + c];
                G[(size_t)r * N2 + c] -= v;
            }
        for (int a = 0; a < nF; a++) xl[Fs[a]] = xn[a];
    }
    free(obar); free(Fs); free(F); free(xf); free(xn); free(D); free(Mf); free(Wm); free(piv);
    free(X); free(Y); free(XW);
}

/* Energy, Eqs. 2DSocHubbard and Oxformula with the spin-coupled Wick contraction:
 *   E = tr(H0 A) + U sum_i [A_ii A_{N+i,N+i} - A_{N+i,i} A_{i,N+i} - (A_ii + A_{N+i,N+i}) / 2],
 * A = 1 - G, A_ab = <c_b^+ c_a>.  out = (Re E, Im E). */
void soc_energy(const soc_params* p, const cplx* H0, const cplx* G, double* out) {
    const int N = p->N, N2 = 2 * N;
    cplx e = 0;
    for (int a = 0; a < N2; a++)
        for (int b = 0; b < N2; b++) e += H0[(size_t)a * N2 + b] * ((a == b ? 1.0 : 0.0) - G[(size_t)b * N2 + a]);
    for (int i = 0; i < N; i++) {
        const cplx Aii = 1.0 - G[(size_t)i * N2 + i], Add = 1.0 - G[(size_t)(N + i) * N2 + N + i];
        const cplx Adu = -G[(size_t)(N + i) * N2 + i], Aud = -G[(size_t)i * N2 + N + i];
        e += p->U * (Aii * Add - Adu * Aud - 0.5 * (Aii + Add));
    }
    out[0] = creal(e);
    out[1] = cimag(e);
}

/* Pairing observables of Sec. IV (the attractive Hubbard benchmarks), mixed estimator from G by the
 * spin-coupled Wick contraction (A = 1 - G, A_ab = <c_b^+ c_a>, G_ab = <c_a c_b^+>; orbitals
 * u = i, d = N + i):
 *   double occupancy   D = N^{-1} sum_i <n_iu n_id> = N^{-1} sum_i (A_uu A_dd - A_du A_ud);
 *   pairing            <Delta^2> = L^{-2} sum_r P(r), P(r) = L^{-2} sum_i <D+_i D_{i+r} + D_i D+_{i+r}> / 4,
 *                      D+_i = c+_iu c+_id, with
 *                      <D+_i D_j> = A_{ju,iu} A_{jd,id} - A_{jd,iu} A_{ju,id},
 *                      <D_i D+_j> = G_{iu,ju} G_{id,jd} - G_{id,ju} G_{iu,jd};
 *   momentum space     c_{k s} = N^{-1/2} sum_j e^{-i k.r_j} c_{j s}, k = 2 pi (nx, ny) / L, index
 *                      nx + L ny; At_{(p s),(q t)} = <c+_{q t} c_{p s}> = (F A F^+) with
 *                      F_{p j} = N^{-1/2} e^{-i p.r_j} on each spin block;
 *                      nk[k] = <n_{k u}> = At_{ku,ku}, nk[N + k] = <n_{k d}> = At_{kd,kd};
 *                      Mk[k][k'] = <D+_k D_k'>, D+_k = c+_{k u} c+_{-k d}:
 *                                = At_{k'u,ku} At_{-k'd,-kd} - At_{-k'd,ku} At_{k'u,-kd}.
 * The condensate fraction n_c = lambda_max(M) / (N_e / 2) (Sec. IV) takes the Monte Carlo average
 * of Mk minus delta_kk' <n_{ku}> <n_{-kd}>; that average is the caller's.
 * out: Re D, Im D, Re <Delta^2>, Im <Delta^2>; nk: 2N complex; Mk: N x N complex (both nullable). */
void soc_pairing(const soc_params* p, const cplx* G, double* out, cplx* nk, cplx* Mk) {
    const int L = p->L, N = p->N, N2 = 2 * N;
    cplx* A = malloc((size_t)N2 * N2 * sizeof(cplx));
    for (int a = 0; a < N2; a++)
        for (int b = 0; b < N2; b++) A[(size_t)a * N2 + b] = (a == b ? 1.0 : 0.0) - G[(size_t)a * N2 + b];
#define AE(a, b) A[(size_t)(a) * N2 + (b)]
#define GE(a, b) G[(size_t)(a) * N2 + (b)]
    cplx d = 0, pd = 0;
    for (int i = 0; i < N; i++) d += AE(i, i) * AE(N + i, N + i) - AE(N + i, i) * AE(i, N + i);
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
            const cplx dpd = AE(j, i) * AE(N + j, N + i) - AE(N + j, i) * AE(j, N + i);
            const cplx ddp = GE(i, j) * GE(N + i, N + j) - GE(N + i, j) * GE(i, N + j);
            pd += 0.25 * (dpd + ddp);
        }
    out[0] = creal(d) / N;
    out[1] = cimag(d) / N;
    out[2] = creal(pd) / ((double)N * N);
    out[3] = cimag(pd) / ((double)N * N);
    if (nk || Mk) {
        /* F (N x N) and At = F2 A F2^+ with F2 = diag(F, F) */
        cplx* F = malloc((size_t)N * N * sizeof(cplx));
        for (int q = 0; q < N; q++)
            for (int j = 0; j < N; j++) {
                const double ph = -2.0 * M_PI * ((double)(q % L) * (j % L) + (double)(q / L) * (j / L)) / L;
                F[(size_t)q * N + j] = (cos(ph) + I * sin(ph)) / sqrt((double)N);
            }
        cplx* T = malloc((size_t)N2 * N2 * sizeof(cplx));
        cplx* At = malloc((size_t)N2 * N2 * sizeof(cplx));
        /* T = A F2^+ : T[a][(q t)] = sum_j A[a][(j t)] conj(F[q][j]) */
#pragma omp parallel for schedule(static)
        for (int a = 0; a < N2; a++)
            for (int t = 0; t < 2; t++)
                for (int q = 0; q < N; q++) {
                    cplx v = 0;
                    for (int j = 0; j < N; j++) v += AE(a, t * N + j) * conj(F[(size_t)q * N + j]);
                    T[(size_t)a * N2 + t * N + q] = v;
                }
        /* At = F2 T : At[(p s)][b] = sum_i F[p][i] T[(i s)][b] */
#pragma omp parallel for schedule(static)
        for (int s = 0; s < 2; s++)
            for (int pp = 0; pp < N; pp++)
                for (int b = 0; b < N2; b++) {
                    cplx v = 0;
                    for (int i = 0; i < N; i++) v += F[(size_t)pp * N + i] * T[(size_t)(s * N + i) * N2 + b];
                    At[(size_t)(s * N + pp) * N2 + b] = v;
                }
#define AT(a, b) At[(size_t)(a) * N2 + (b)]
        if (nk)
            for (int k = 0; k < N; k++) {
                nk[k] = AT(k, k);
                nk[N + k] = AT(N + k, N + k);
            }
        if (Mk)
            for (int k = 0; k < N; k++) {
                const int mk = (L - k % L) % L + L * ((L - k / L) % L);
                for (int k2 = 0; k2 < N; k2++) {
                    const int mk2 = (L - k2 % L) % L + L * ((L - k2 / L) % L);
                    Mk[(size_t)k * N + k2] = AT(k2, k) * AT(N + mk2, N + mk) - AT(N + mk2, k) * AT(k2, N + mk);
                }
            }
#undef AT
        free(F);
        free(T);
        free(At);
    }
#undef AE
#undef GE
    free(A);
}
