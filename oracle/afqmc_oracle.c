/*
 * afqmc_oracle.c -- plain, slow, FP64 CPU oracle for the ground-state AFQMC
 * (PQMC) auxiliary-field update sweep on the equal-time Green's function G.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this file.  It shares no
 * code, header, table or constant with the CUDA library.
 *
 * Conventions (paper section II, Eqs. GrFMat, BlMat, HSspinDecomp):
 *   sites i = x + Lx*y, N = Lx*Ly; G_ij = <c_i c_j^+>;  A = 1 - G, A_ij = <c_j^+ c_i>.
 *   E = exp(-dtau K), Einv = exp(+dtau K); B_l^s = D_l^s E, D_l^s = diag(exp(c_s x_{l,i})).
 *   All N x N matrices are row-major.  U_R is N x ns row-major, U_L is ns x N row-major.
 *   Slices l = 1..M; the field of slice l, site i is x[(l-1)*N + i] in {-1,+1}.
 *
 * Hubbard-Stratonovich modes (Sec. II.B and Hirsch's real decouplings):
 *   HS_SZ_REAL     (U > 0): cosh(lam) = exp(dtau U / 2), c_up = +lam, c_dn = -lam, s(x) = 1.
 *   HS_CHARGE_REAL (U < 0): cosh(lam) = exp(dtau |U| / 2), c_up = c_dn = +lam, s(x) = exp(-lam x).
 * where e^{-dtau U (n_up n_dn - (n_up+n_dn)/2)} = C * sum_x s(x) e^{x (c_up n_up + c_dn n_dn)} / 2.
 *
 * Loops over independent output rows carry OpenMP pragmas; every output element
 * is still accumulated by one thread in the written order, so results do not
 * depend on the thread count.
 *
 * Every function below follows the paper's equations, restated in the G form
 * (the identity G = 1 - U_R T U_L of Eq. GrFMatNew turns the paper's T-matrix
 * updates into updates of G):
 *   ratio      r_s = det(1 + Delta^s A^s)                       (Eq. DetRatio10 via Sylvester)
 *   update     A' = (1 + Delta)(1 + A Delta)^{-1} A              (Eq. UpdateLTRMat via Woodbury)
 *   local      G' = G - (d/r) G_{:,i} (e_i^T - G_{i,:})          (Eqs. DetRatiolocal, UpdateLTRlocal)
 *   delayed    G_[m] = G_[0] + sum_m a_m b_m^T                   (Eqs. DelayTMat00, DelayRgenk, FinalDelay)
 *   block FB   stripped force bias + joint proposal + det ratio  (Eqs. BlockFrcbsPhiLPhiR .. BlkFrcBsTnew2)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define HS_SZ_REAL 0
#define HS_CHARGE_REAL 1

typedef struct {
    int Lx, Ly, N, M;
    int hs;
    double t, U, dtau;
    double lam;     /* HS coupling */
    double c[2];    /* c_up, c_dn */
} or_params;

/* ------------------------------------------------------------------ */
/* Model: lattice, hopping and exp(-+dtau K)  (Eq. 2DHubbard)          */
/* ------------------------------------------------------------------ */

/* HS coupling constants for the mode in p (Eq. HSspinDecomp and Hirsch's
 * real spin / charge channels).  Returns 0, or -1 on a bad mode / sign of U. */
int or_setup(or_params* p) {
    p->N = p->Lx * p->Ly;
    if (p->hs == HS_SZ_REAL) {
        if (p->U < 0) return -1;
        p->lam = acosh(exp(p->dtau * p->U / 2.0));
        p->c[0] = p->lam;
        p->c[1] = -p->lam;
    } else if (p->hs == HS_CHARGE_REAL) {
        if (p->U > 0) return -1;
        p->lam = acosh(exp(p->dtau * fabs(p->U) / 2.0));
        p->c[0] = p->lam;
        p->c[1] = p->lam;
    } else {
        return -1;
    }
    return 0;
}

/* log of the field-dependent scalar s(x) of the decoupling */
static double hs_log_scalar(const or_params* p, int x) {
    return p->hs == HS_CHARGE_REAL ? -p->lam * (double)x : 0.0;
}

/* Delta^s_ii for the change x -> xp at one site: e^{c_s (xp - x)} - 1  (Sec. II.C) */
static double field_delta(const or_params* p, int s, int x, int xp) {
    return exp(p->c[s] * (double)(xp - x)) - 1.0;
}

/* exp(-tau K) for the periodic nearest-neighbour lattice, as the Fourier sum
 * E_ij = N^{-1} sum_k exp(-tau eps_k) cos(k.(r_i - r_j)),
 * eps_k = -2t(cos kx + cos ky), k in units of 2 pi / L  (Eq. 2DHubbard). */
void or_expK(const or_params* p, double tau, double* E) {
    int Lx = p->Lx, Ly = p->Ly, N = p->N;
    double* f = (double*)calloc((size_t)N, sizeof(double)); /* by displacement */
    for (int dy = 0; dy < Ly; dy++)
        for (int dx = 0; dx < Lx; dx++) {
            double acc = 0.0;
            for (int ny = 0; ny < Ly; ny++)
                for (int nx = 0; nx < Lx; nx++) {
                    double kx = 2.0 * M_PI * nx / Lx, ky = 2.0 * M_PI * ny / Ly;
                    double eps = -2.0 * p->t * (cos(kx) + cos(ky));
                    acc += exp(-tau * eps) * cos(kx * dx + ky * dy);
                }
            f[dx + Lx * dy] = acc / N;
        }
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
            int dx = ((i % Lx) - (j % Lx) + Lx) % Lx;
            int dy = ((i / Lx) - (j / Lx) + Ly) % Ly;
            E[(size_t)i * N + j] = f[dx + Lx * dy];
        }
    free(f);
}

/* ------------------------------------------------------------------ */
/* Small dense linear algebra: LU with partial pivoting, Householder QR */
/* ------------------------------------------------------------------ */

/* In-place LU of the n x n row-major a with partial pivoting.  piv[k] is the
 * row swapped with k.  Returns the sign of the permutation times the sign of
 * prod(diag U); *logabs = log|det a|.  A zero pivot gives sign 0. */
static int lu_factor(double* a, int n, int* piv, double* logabs) {
    int sgn = 1;
    double la = 0.0;
    for (int k = 0; k < n; k++) {
        int pr = k;
        double best = fabs(a[(size_t)k * n + k]);
        for (int r = k + 1; r < n; r++)
            if (fabs(a[(size_t)r * n + k]) > best) { best = fabs(a[(size_t)r * n + k]); pr = r; }
        piv[k] = pr;
        if (best == 0.0) { *logabs = -INFINITY; return 0; }
        if (pr != k) {
            for (int c = 0; c < n; c++) {
                double tmp = a[(size_t)k * n + c];
                a[(size_t)k * n + c] = a[(size_t)pr * n + c];
                a[(size_t)pr * n + c] = tmp;
            }
            sgn = -sgn;
        }
        double d = a[(size_t)k * n + k];
        if (d < 0) sgn = -sgn;
        la += log(fabs(d));
#pragma omp parallel for schedule(static)
        for (int r = k + 1; r < n; r++) {
            double l = a[(size_t)r * n + k] / d;
            a[(size_t)r * n + k] = l;
            for (int c = k + 1; c < n; c++) a[(size_t)r * n + c] -= l * a[(size_t)k * n + c];
        }
    }
    *logabs = la;
    return sgn;
}

/* Solve (LU) X = B in place, B is n x nrhs row-major. */
static void lu_solve(const double* lu, int n, const int* piv, double* b, int nrhs) {
    for (int k = 0; k < n; k++)
        if (piv[k] != k)
            for (int c = 0; c < nrhs; c++) {
                double tmp = b[(size_t)k * nrhs + c];
                b[(size_t)k * nrhs + c] = b[(size_t)piv[k] * nrhs + c];
                b[(size_t)piv[k] * nrhs + c] = tmp;
            }
    for (int r = 0; r < n; r++)
        for (int k = 0; k < r; k++) {
            double l = lu[(size_t)r * n + k];
            for (int c = 0; c < nrhs; c++) b[(size_t)r * nrhs + c] -= l * b[(size_t)k * nrhs + c];
        }
    for (int r = n - 1; r >= 0; r--) {
        for (int k = r + 1; k < n; k++) {
            double u = lu[(size_t)r * n + k];
            for (int c = 0; c < nrhs; c++) b[(size_t)r * nrhs + c] -= u * b[(size_t)k * nrhs + c];
        }
        double d = lu[(size_t)r * n + r];
        for (int c = 0; c < nrhs; c++) b[(size_t)r * nrhs + c] /= d;
    }
}

/* Determinant of the n x n row-major a (copied).  Returns sign, *logabs. */
static int det_sign_log(const double* a, int n, double* logabs) {
    double* w = (double*)malloc(sizeof(double) * (size_t)n * n + 1);
    int* piv = (int*)malloc(sizeof(int) * (size_t)n + 1);
    memcpy(w, a, sizeof(double) * (size_t)n * n);
    int s = lu_factor(w, n, piv, logabs);
    free(w);
    free(piv);
    return s;
}

/* Thin Householder QR of the m x n matrix whose element (r, c) is
 * a[r * rs + c * cs].  On return the same storage holds Q (m x n, orthonormal
 * columns); the function returns sign(det R) and adds log|det R| to *logabs. */
static int qr_orth(double* a, int m, int n, size_t rs, size_t cs, double* logabs) {
    double* v = (double*)malloc(sizeof(double) * (size_t)m * n + 1); /* reflectors, column-major m x n */
    double* beta = (double*)malloc(sizeof(double) * (size_t)n + 1);
    int sgn = 1;
#define A_(r, c) a[(size_t)(r) * rs + (size_t)(c) * cs]
    for (int j = 0; j < n; j++) {
        double nrm = 0.0;
        for (int r = j; r < m; r++) nrm += A_(r, j) * A_(r, j);
        nrm = sqrt(nrm);
        double x0 = A_(j, j);
        double alpha = (x0 >= 0) ? -nrm : nrm; /* R_jj */
        double* vj = v + (size_t)j * m;
        for (int r = 0; r < m; r++) vj[r] = 0.0;
        for (int r = j; r < m; r++) vj[r] = A_(r, j);
        vj[j] -= alpha;
        double vn = 0.0;
        for (int r = j; r < m; r++) vn += vj[r] * vj[r];
        beta[j] = (vn > 0) ? 2.0 / vn : 0.0;
        /* apply H_j = 1 - beta v v^T to columns j..n-1 */
#pragma omp parallel for schedule(static)
        for (int c = j; c < n; c++) {
            double s = 0.0;
            for (int r = j; r < m; r++) s += vj[r] * A_(r, c);
            s *= beta[j];
            for (int r = j; r < m; r++) A_(r, c) -= s * vj[r];
        }
        if (alpha < 0) sgn = -sgn;
        *logabs += log(fabs(alpha));
        if (alpha == 0.0) sgn = 0;
    }
    /* Q = H_0 H_1 ... H_{n-1} [I_n; 0] */
    for (int r = 0; r < m; r++)
        for (int c = 0; c < n; c++) A_(r, c) = (r == c) ? 1.0 : 0.0;
    for (int j = n - 1; j >= 0; j--) {
        double* vj = v + (size_t)j * m;
#pragma omp parallel for schedule(static)
        for (int c = 0; c < n; c++) {
            double s = 0.0;
            for (int r = j; r < m; r++) s += vj[r] * A_(r, c);
            s *= beta[j];
            for (int r = j; r < m; r++) A_(r, c) -= s * vj[r];
        }
    }
    /* Q R with Q from the reflectors: det(H_j) = -1 each; keep the sign of
     * R_true = Q^T A consistent with A = Q R by folding det(Q-part) out:
     * A = (H_0..H_{n-1}) [R;0] and Q above are exactly those columns, so
     * sign(det R) is the product of the alphas' signs computed above. */
#undef A_
    free(v);
    free(beta);
    return sgn;
}

/* ------------------------------------------------------------------ */
/* Propagation and G from scratch  (Eqs. ConfgWeight, GrFMat, GrFMatNew) */
/* ------------------------------------------------------------------ */

/* Y = B_l^s X for X N x ns (row-major): (D E X). */
static void apply_B_left(const or_params* p, const double* E, const int8_t* xl, int s,
                         const double* X, double* Y, int ns) {
    int N = p->N;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; i++) {
        double d = exp(p->c[s] * xl[i]);
        double* y = Y + (size_t)i * ns;
        for (int c = 0; c < ns; c++) y[c] = 0.0;
        for (int k = 0; k < N; k++) {
            double e = E[(size_t)i * N + k];
            for (int c = 0; c < ns; c++) y[c] += e * X[(size_t)k * ns + c];
        }
        for (int c = 0; c < ns; c++) y[c] *= d;
    }
}

/* Y = X B_l^s for X ns x N: (X D) E. */
static void apply_B_right(const or_params* p, const double* E, const int8_t* xl, int s,
                          const double* X, double* Y, int ns) {
    int N = p->N;
    double* XD = (double*)malloc(sizeof(double) * (size_t)ns * N + 1);
    for (int r = 0; r < ns; r++)
        for (int k = 0; k < N; k++) XD[(size_t)r * N + k] = X[(size_t)r * N + k] * exp(p->c[s] * xl[k]);
#pragma omp parallel for schedule(static)
    for (int r = 0; r < ns; r++) {
        double* y = Y + (size_t)r * N;
        for (int j = 0; j < N; j++) y[j] = 0.0;
        for (int k = 0; k < N; k++) {
            double a = XD[(size_t)r * N + k];
            for (int j = 0; j < N; j++) y[j] += a * E[(size_t)k * N + j];
        }
    }
    free(XD);
}

/* Equal-time G at slice l (0 <= l <= M) for spin s, from scratch:
 *   R = B_l ... B_1 P,  L = P^T B_M ... B_{l+1},  G = 1 - R (L R)^{-1} L,
 * with the QR re-orthonormalisation of U_R and U_L every `stab` products
 * (Sec. II.B, Eq. GrFMatNew).  P is N x ns row-major.  If UR_out / UL_out are
 * non-null they receive the final (orthonormal) U_R and U_L.  Returns the sign
 * of det(L R) = det(P^T B_M..B_1 P) and writes log|det| to *logabs. */
int or_green_scratch(const or_params* p, const double* E, const int8_t* x, const double* P, int ns,
                     int s, int l, int stab, double* G, double* logabs, double* UR_out, double* UL_out) {
    int N = p->N;
    size_t nn = (size_t)N * ns;
    double* UR = (double*)malloc(sizeof(double) * nn + 1);
    double* UL = (double*)malloc(sizeof(double) * nn + 1);
    double* tmp = (double*)malloc(sizeof(double) * nn + 1);
    double la = 0.0;
    int sgn = 1;
    memcpy(UR, P, sizeof(double) * nn);
    for (int r = 0; r < ns; r++)
        for (int k = 0; k < N; k++) UL[(size_t)r * N + k] = P[(size_t)k * ns + r];
    if (stab < 1) stab = 1 << 30;
    int cnt = 0;
    for (int j = 1; j <= l; j++) {
        apply_B_left(p, E, x + (size_t)(j - 1) * N, s, UR, tmp, ns);
        memcpy(UR, tmp, sizeof(double) * nn);
        if (++cnt % stab == 0) sgn *= qr_orth(UR, N, ns, (size_t)ns, 1, &la);
    }
    sgn *= qr_orth(UR, N, ns, (size_t)ns, 1, &la);
    cnt = 0;
    for (int j = p->M; j >= l + 1; j--) {
        apply_B_right(p, E, x + (size_t)(j - 1) * N, s, UL, tmp, ns);
        memcpy(UL, tmp, sizeof(double) * nn);
        if (++cnt % stab == 0) sgn *= qr_orth(UL, N, ns, 1, (size_t)N, &la); /* QR of U_L^T */
    }
    sgn *= qr_orth(UL, N, ns, 1, (size_t)N, &la);
    /* O = U_L U_R (ns x ns); T = O^{-1}; G = 1 - U_R T U_L */
    double* O = (double*)malloc(sizeof(double) * (size_t)ns * ns + 1);
#pragma omp parallel for schedule(static)
    for (int a = 0; a < ns; a++) {
        double* o = O + (size_t)a * ns;
        for (int b = 0; b < ns; b++) o[b] = 0.0;
        for (int k = 0; k < N; k++) {
            double l = UL[(size_t)a * N + k];
            for (int b = 0; b < ns; b++) o[b] += l * UR[(size_t)k * ns + b];
        }
    }
    int* piv = (int*)malloc(sizeof(int) * (size_t)ns + 1);
    double lo;
    sgn *= lu_factor(O, ns, piv, &lo);
    la += lo;
    /* Z = O^{-1} U_L  (ns x N) */
    memcpy(tmp, UL, sizeof(double) * nn);
    lu_solve(O, ns, piv, tmp, N);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; i++) {
        double* g = G + (size_t)i * N;
        for (int j = 0; j < N; j++) g[j] = 0.0;
        for (int k = 0; k < ns; k++) {
            double r = UR[(size_t)i * ns + k];
            for (int j = 0; j < N; j++) g[j] += r * tmp[(size_t)k * N + j];
        }
        for (int j = 0; j < N; j++) g[j] = (i == j ? 1.0 : 0.0) - g[j];
    }
    if (UR_out) memcpy(UR_out, UR, sizeof(double) * nn);
    if (UL_out) memcpy(UL_out, UL, sizeof(double) * nn);
    *logabs = la;
    free(UR); free(UL); free(tmp); free(O); free(piv);
    return sgn;
}

/* C = A B for N x N row-major matrices; each C_ij sums k = 0..N-1 in order. */
static void matmul(const double* A, const double* B, double* C, int N) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; i++) {
        double* c = C + (size_t)i * N;
        for (int j = 0; j < N; j++) c[j] = 0.0;
        for (int k = 0; k < N; k++) {
            double a = A[(size_t)i * N + k];
            for (int j = 0; j < N; j++) c[j] += a * B[(size_t)k * N + j];
        }
    }
}

/* ------------------------------------------------------------------ */
/* Wrap  G(l) = B_l G(l-1) B_l^{-1}  (Eqs. BlMat, GrFMat)               */
/* ------------------------------------------------------------------ */

/* dir = +1: G <- D E G Einv D^{-1} with D from slice field xl (forward, l-1 -> l).
 * dir = -1: G <- Einv D^{-1} G D E (backward, l -> l-1). */
void or_wrap(const or_params* p, const double* E, const double* Einv, const int8_t* xl, int s,
             int dir, double* G) {
    int N = p->N;
    double* T = (double*)malloc(sizeof(double) * (size_t)N * N + 1);
    double* d = (double*)malloc(sizeof(double) * (size_t)N + 1);
    for (int i = 0; i < N; i++) d[i] = exp(p->c[s] * xl[i]);
    if (dir > 0) {
        /* T = E G ; G = D (T Einv) D^{-1} */
        matmul(E, G, T, N);
        matmul(T, Einv, G, N);
        for (int i = 0; i < N; i++)
            for (int j = 0; j < N; j++) G[(size_t)i * N + j] = d[i] * G[(size_t)i * N + j] / d[j];
    } else {
        /* T = D^{-1} G D ; G = Einv T E */
        for (int i = 0; i < N; i++)
            for (int j = 0; j < N; j++) T[(size_t)i * N + j] = G[(size_t)i * N + j] * d[j] / d[i];
        double* T2 = (double*)malloc(sizeof(double) * (size_t)N * N + 1);
        matmul(Einv, T, T2, N);
        matmul(T2, E, G, N);
        free(T2);
    }
    free(T);
    free(d);
}

/* ------------------------------------------------------------------ */
/* Local update  (Sec. II.D, Eqs. DetailBalance, DetRatiolocal,        */
/* UpdateLTRlocal) in G form                                           */
/* ------------------------------------------------------------------ */

/* One Metropolis pass over the sites i = 0..N-1 of one slice.
 * G[0], G[1]: spin up / down (N x N).  xl: the slice's fields (modified).
 * u[i]: uniform in [0,1) for site i.  replay (nullable): forced decisions.
 * dec[i] receives the decision, ratio[i] the weight ratio R_i.
 * *sign is multiplied by sign(R) for each accepted flip. */
void or_local_slice(const or_params* p, double* G0, double* G1, int8_t* xl, const double* u,
                    const uint8_t* replay, uint8_t* dec, double* ratio, double* sign) {
    int N = p->N;
    double* G[2] = {G0, G1};
    double* col = (double*)malloc(sizeof(double) * (size_t)N + 1);
    double* row = (double*)malloc(sizeof(double) * (size_t)N + 1);
    for (int i = 0; i < N; i++) {
        int x = xl[i], xp = -x;
        double R = exp(hs_log_scalar(p, xp) - hs_log_scalar(p, x));
        double d[2], r[2];
        for (int s = 0; s < 2; s++) {
            d[s] = field_delta(p, s, x, xp);
            r[s] = 1.0 + d[s] * (1.0 - G[s][(size_t)i * N + i]);
            R *= r[s];
        }
        int acc = replay ? (replay[i] != 0) : (u[i] < fabs(R));
        dec[i] = (uint8_t)acc;
        ratio[i] = R;
        if (!acc) continue;
        for (int s = 0; s < 2; s++) {
            double* g = G[s];
            for (int a = 0; a < N; a++) col[a] = g[(size_t)a * N + i];
            for (int b = 0; b < N; b++) row[b] = (b == i ? 1.0 : 0.0) - g[(size_t)i * N + b];
            double f = d[s] / r[s];
#pragma omp parallel for schedule(static)
            for (int a = 0; a < N; a++)
                for (int b = 0; b < N; b++) g[(size_t)a * N + b] -= f * col[a] * row[b];
        }
        xl[i] = (int8_t)xp;
        if (R < 0) *sign = -*sign;
    }
    free(col);
    free(row);
}

/* ------------------------------------------------------------------ */
/* Delayed update  (Sec. III.A, Eqs. DelayTMat00, DelayRatio,          */
/* DelayRgenk, FinalDelay) in G form                                   */
/* ------------------------------------------------------------------ */

/* Same pass as or_local_slice, but the rank-1 corrections are delayed:
 * after m accepted flips G = G_[0] + sum_{m'<m} a_m' b_m'^T with
 *   a_m = -(d/r) (G_[0] e_i + sum a_m' b_m'[i])      (current column i)
 *   b_m =  e_i - (e_i^T G_[0] + sum a_m'[i] b_m'^T)  (current row i)
 * and the diagonal kept current on the fly.  The buffered update is applied
 * as one matrix product G_[0] += U V^T when k vectors are buffered
 * (strategy = 2: k accepted moves) or after k proposals (strategy = 1), and
 * always at the end of the slice. */
void or_delayed_slice(const or_params* p, double* G0, double* G1, int8_t* xl, const double* u,
                      int k, int strategy, const uint8_t* replay, uint8_t* dec, double* ratio,
                      double* sign, int* nflush) {
    int N = p->N;
    double* G[2] = {G0, G1};
    if (k < 1) k = 1;
    double* Ub[2];
    double* Vb[2];
    double* dg[2];
    for (int s = 0; s < 2; s++) {
        Ub[s] = (double*)calloc((size_t)N * k + 1, sizeof(double)); /* Ub[j*k + m] = a_m[j] */
        Vb[s] = (double*)calloc((size_t)N * k + 1, sizeof(double)); /* Vb[j*k + m] = b_m[j] */
        dg[s] = (double*)malloc(sizeof(double) * (size_t)N + 1);
        for (int j = 0; j < N; j++) dg[s][j] = G[s][(size_t)j * N + j];
    }
    int m = 0, ntry = 0, flushes = 0;
    for (int i = 0; i <= N; i++) {
        int want_flush = (i == N) ? (m > 0) : 0;
        if (i < N) {
            int x = xl[i], xp = -x;
            double R = exp(hs_log_scalar(p, xp) - hs_log_scalar(p, x));
            double d[2], r[2];
            for (int s = 0; s < 2; s++) {
                d[s] = field_delta(p, s, x, xp);
                r[s] = 1.0 + d[s] * (1.0 - dg[s][i]);
                R *= r[s];
            }
            int acc = replay ? (replay[i] != 0) : (u[i] < fabs(R));
            dec[i] = (uint8_t)acc;
            ratio[i] = R;
            ntry++;
            if (acc) {
                for (int s = 0; s < 2; s++) {
                    double* g = G[s];
                    double* U = Ub[s];
                    double* V = Vb[s];
                    double f = -d[s] / r[s];
#pragma omp parallel for schedule(static)
                    for (int j = 0; j < N; j++) {
                        double colj = g[(size_t)j * N + i], rowj = g[(size_t)i * N + j];
                        for (int q = 0; q < m; q++) {
                            colj += U[(size_t)j * k + q] * V[(size_t)i * k + q];
                            rowj += U[(size_t)i * k + q] * V[(size_t)j * k + q];
                        }
                        U[(size_t)j * k + m] = f * colj;
                        V[(size_t)j * k + m] = (j == i ? 1.0 : 0.0) - rowj;
                    }
                    for (int j = 0; j < N; j++) dg[s][j] += U[(size_t)j * k + m] * V[(size_t)j * k + m];
                }
                m++;
                xl[i] = (int8_t)xp;
                if (R < 0) *sign = -*sign;
            }
            if (strategy == 2 && m == k) want_flush = 1;
            if (strategy == 1 && ntry == k && m > 0) want_flush = 1;
            if (strategy == 1 && ntry == k) ntry = 0;
        }
        if (want_flush) {
            for (int s = 0; s < 2; s++) {
                double* g = G[s];
#pragma omp parallel for schedule(static)
                for (int a = 0; a < N; a++)
                    for (int b = 0; b < N; b++) {
                        double acc2 = 0.0;
                        for (int q = 0; q < m; q++) acc2 += Ub[s][(size_t)a * k + q] * Vb[s][(size_t)b * k + q];
                        g[(size_t)a * N + b] += acc2;
                    }
                for (int j = 0; j < N; j++) dg[s][j] = g[(size_t)j * N + j];
            }
            m = 0;
            flushes++;
        }
    }
    if (nflush) *nflush = flushes;
    for (int s = 0; s < 2; s++) { free(Ub[s]); free(Vb[s]); free(dg[s]); }
}

/* ------------------------------------------------------------------ */
/* T form  (Sec. II.C, Eq. GrFMatNew; Sec. II.D, Eqs. DetRatio10,      */
/* UpdateLTRMat; Sec. III.A, Eqs. DelayTMat00, DelayRatio, DelayRgenk, */
/* FinalDelay): the paper's own walker state                           */
/* ------------------------------------------------------------------ */

/* Per spin the walker is U_R (N x ns), U_L (ns x N) and T = (U_L U_R)^{-1} (ns x ns), with
 * G = 1 - U_R T U_L (Eq. GrFMatNew) never formed.  Between slices the factors move and T stays:
 *   forward  (l-1 -> l): U_R <- B_l U_R = D E U_R,           U_L <- U_L B_l^{-1} = U_L Einv D^{-1};
 *   backward (l -> l-1): U_R <- B_l^{-1} U_R = Einv D^{-1} U_R, U_L <- U_L B_l = U_L D E;
 * U_L U_R is unchanged by either. */
void or_tform_wrap(const or_params* p, const double* E, const double* Einv, const int8_t* xl, int s, int dir,
                   int ns, double* UR, double* UL) {
    int N = p->N;
    size_t nn = (size_t)N * ns;
    double* d = (double*)malloc(sizeof(double) * (size_t)N + 1);
    double* tmp = (double*)malloc(sizeof(double) * nn + 1);
    for (int i = 0; i < N; i++) d[i] = exp(p->c[s] * xl[i]);
    const double* ER = (dir > 0) ? E : Einv;  /* left factor of U_R */
    const double* EL = (dir > 0) ? Einv : E;  /* right factor of U_L */
    /* U_R: forward D (E U_R); backward Einv (D^{-1} U_R) */
    if (dir < 0)
        for (int i = 0; i < N; i++)
            for (int c = 0; c < ns; c++) UR[(size_t)i * ns + c] /= d[i];
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; i++) {
        double* t = tmp + (size_t)i * ns;
        for (int c = 0; c < ns; c++) t[c] = 0.0;
        for (int k = 0; k < N; k++) {
            double e = ER[(size_t)i * N + k];
            for (int c = 0; c < ns; c++) t[c] += e * UR[(size_t)k * ns + c];
        }
    }
    for (int i = 0; i < N; i++)
        for (int c = 0; c < ns; c++) UR[(size_t)i * ns + c] = (dir > 0 ? d[i] : 1.0) * tmp[(size_t)i * ns + c];
    /* U_L: forward (U_L Einv) D^{-1}; backward (U_L D) E */
    if (dir < 0)
        for (int r = 0; r < ns; r++)
            for (int k = 0; k < N; k++) UL[(size_t)r * N + k] *= d[k];
#pragma omp parallel for schedule(static)
    for (int r = 0; r < ns; r++) {
        double* t = tmp + (size_t)r * N;
        for (int j = 0; j < N; j++) t[j] = 0.0;
        for (int k = 0; k < N; k++) {
            double a = UL[(size_t)r * N + k];
            for (int j = 0; j < N; j++) t[j] += a * EL[(size_t)k * N + j];
        }
    }
    for (int r = 0; r < ns; r++)
        for (int j = 0; j < N; j++) UL[(size_t)r * N + j] = tmp[(size_t)r * N + j] / (dir > 0 ? d[j] : 1.0);
    free(d);
    free(tmp);
}

/* Delayed update of one slice in the T form.  At a proposed site i, per spin s with
 * Delta = e^{c_s (x' - x)} - 1 the only non-zero element of the Delta matrix of Eq. DetRatio10,
 * u = U_R[i, :] (the row as it is now) and v = Delta U_L[:, i]:
 *   r   = 1 + u T_[0] v - sum_{m<k} (u x_m)(y_m v)                          (Eq. DelayRatio)
 * and, if the move is the k-th acceptance,
 *   x_k = (T_[0] v - sum_{m<k} x_m (y_m v)) / r,
 *   y_k = u T_[0] - sum_{m<k} (u x_m) y_m                                    (Eq. DelayRgenk)
 *   U_R[i, :] <- (1 + Delta) U_R[i, :]                                       (Eq. UpdateLTRMat)
 * T_[0] <- T_[0] - X Y (Eq. FinalDelay) after every k proposed sites (strategy 1, the paper's
 * choice) or every k acceptances (strategy 2), and at the end of the slice.  Decisions and the
 * weight ratio R = (P-ratio) r_up r_dn follow or_local_slice. */
void or_tform_delayed_slice(const or_params* p, double* UR0, double* UR1, const double* UL0, const double* UL1,
                            double* T0, double* T1, int ns0, int ns1, int8_t* xl, const double* u, int k,
                            int strategy, const uint8_t* replay, uint8_t* dec, double* ratio, double* sign,
                            int* nflush) {
    int N = p->N;
    double* UR[2] = {UR0, UR1};
    const double* UL[2] = {UL0, UL1};
    double* T[2] = {T0, T1};
    int ns[2] = {ns0, ns1};
    if (k < 1) k = 1;
    double *X[2], *Y[2], *v[2], *Tv[2], *uT[2], *cm[2], *dm[2];
    for (int s = 0; s < 2; s++) {
        int n = ns[s];
        X[s] = (double*)calloc((size_t)n * k + 1, sizeof(double));  /* X[a*k + m] = x_m[a] */
        Y[s] = (double*)calloc((size_t)k * n + 1, sizeof(double));  /* Y[m*n + b] = y_m[b] */
        v[s] = (double*)malloc(sizeof(double) * (size_t)n + 1);
        Tv[s] = (double*)malloc(sizeof(double) * (size_t)n + 1);
        uT[s] = (double*)malloc(sizeof(double) * (size_t)n + 1);
        cm[s] = (double*)malloc(sizeof(double) * (size_t)k + 1);
        dm[s] = (double*)malloc(sizeof(double) * (size_t)k + 1);
    }
    int m = 0, ntry = 0, flushes = 0;
    for (int i = 0; i <= N; i++) {
        int want_flush = (i == N) ? (m > 0) : 0;
        if (i < N) {
            int x = xl[i], xp = -x;
            double R = exp(hs_log_scalar(p, xp) - hs_log_scalar(p, x));
            double d[2], r[2];
            for (int s = 0; s < 2; s++) {
                int n = ns[s];
                const double* us = UR[s] + (size_t)i * n;
                const double* t = T[s];
                d[s] = field_delta(p, s, x, xp);
                for (int a = 0; a < n; a++) v[s][a] = d[s] * UL[s][(size_t)a * N + i];
                for (int a = 0; a < n; a++) {
                    double acc = 0.0;
                    for (int b = 0; b < n; b++) acc += t[(size_t)a * n + b] * v[s][b];
                    Tv[s][a] = acc;
                }
                for (int b = 0; b < n; b++) {
                    double acc = 0.0;
                    for (int a = 0; a < n; a++) acc += us[a] * t[(size_t)a * n + b];
                    uT[s][b] = acc;
                }
                double uTv = 0.0;
                for (int a = 0; a < n; a++) uTv += us[a] * Tv[s][a];
                double corr = 0.0;
                for (int q = 0; q < m; q++) {
                    double c = 0.0, e = 0.0;
                    for (int a = 0; a < n; a++) c += us[a] * X[s][(size_t)a * k + q];
                    for (int b = 0; b < n; b++) e += Y[s][(size_t)q * n + b] * v[s][b];
                    cm[s][q] = c;
                    dm[s][q] = e;
                    corr += c * e;
                }
                r[s] = 1.0 + uTv - corr;
                R *= r[s];
            }
            int acc = replay ? (replay[i] != 0) : (u[i] < fabs(R));
            dec[i] = (uint8_t)acc;
            ratio[i] = R;
            ntry++;
            if (acc) {
                for (int s = 0; s < 2; s++) {
                    int n = ns[s];
                    double* us = UR[s] + (size_t)i * n;
                    for (int a = 0; a < n; a++) {
                        double xa = Tv[s][a];
                        for (int q = 0; q < m; q++) xa -= X[s][(size_t)a * k + q] * dm[s][q];
                        X[s][(size_t)a * k + m] = xa / r[s];
                    }
                    for (int b = 0; b < n; b++) {
                        double yb = uT[s][b];
                        for (int q = 0; q < m; q++) yb -= cm[s][q] * Y[s][(size_t)q * n + b];
                        Y[s][(size_t)m * n + b] = yb;
                    }
                    for (int a = 0; a < n; a++) us[a] *= 1.0 + d[s];
                }
                m++;
                xl[i] = (int8_t)xp;
                if (R < 0) *sign = -*sign;
            }
            if (strategy == 2 && m == k) want_flush = 1;
            if (strategy == 1 && ntry == k && m > 0) want_flush = 1;
            if (strategy == 1 && ntry == k) ntry = 0;
        }
        if (want_flush) {
            for (int s = 0; s < 2; s++) {
                int n = ns[s];
                double* t = T[s];
#pragma omp parallel for schedule(static)
                for (int a = 0; a < n; a++)
                    for (int b = 0; b < n; b++) {
                        double acc2 = 0.0;
                        for (int q = 0; q < m; q++) acc2 += X[s][(size_t)a * k + q] * Y[s][(size_t)q * n + b];
                        t[(size_t)a * n + b] -= acc2;
                    }
            }
            m = 0;
            flushes++;
        }
    }
    if (nflush) *nflush = flushes;
    for (int s = 0; s < 2; s++) {
        free(X[s]); free(Y[s]); free(v[s]); free(Tv[s]); free(uT[s]); free(cm[s]); free(dm[s]);
    }
}

/* Block force-bias pass over one slice in the T form (Sec. III.B), with the conventions of
 * or_blockfb_slice (blocks, uniforms, replay layout, proposal and acceptance).  Per block S and
 * spin s, with u_i = U_R[i, :] and v_i = d_i U_L[:, i]:
 *   stripped:  Db_ii = e^{-c_s x_i} - 1, U (rows u_i) and V (columns Db_ii U_L[:, i]), i in S,
 *              Ttil = T - (T V)[1 + (U T) V]^{-1}(U T)                    (Eq. BlkFrcBsTnew1)
 *              nbar_i = (1 + Db_ii) u_i Ttil U_L[:, i]   (the diagonal of (1+Db) U_R Ttil U_L);
 *   ratio:     r_s = det[1 + (U' T) V'] over the flipped sites F, V' columns
 *              (e^{c_s (x' - x)} - 1) U_L[:, i]                           (Eq. DetRatio10)
 *   accepted:  T <- T - (T V')[1 + (U' T) V']^{-1}(U' T)                  (Eq. BlkFrcBsTnew2)
 *              U_R[i, :] <- (1 + Delta_i) U_R[i, :] for i in F             (Eq. UpdateLTRMat). */
void or_tform_blockfb_slice(const or_params* p, double* UR0, double* UR1, const double* UL0, const double* UL1,
                            double* T0, double* T1, int ns0, int ns1, int8_t* xl, const double* u_prop,
                            const double* u_acc, int nb, const uint8_t* replay, int8_t* xprop, double* lam_plus,
                            uint8_t* dec, double* ratio, double* sign) {
    int N = p->N;
    double* UR[2] = {UR0, UR1};
    const double* UL[2] = {UL0, UL1};
    double* T[2] = {T0, T1};
    int ns[2] = {ns0, ns1};
    if (nb < 1) nb = 1;
    int nsx = ns0 > ns1 ? ns0 : ns1;
    double* nbar[2];
    nbar[0] = (double*)malloc(sizeof(double) * (size_t)nb + 1);
    nbar[1] = (double*)malloc(sizeof(double) * (size_t)nb + 1);
    int* F = (int*)malloc(sizeof(int) * (size_t)nb + 1);
    int* piv = (int*)malloc(sizeof(int) * (size_t)nb + 1);
    double* TV = (double*)malloc(sizeof(double) * (size_t)nsx * nb + 1);  /* ns x n   */
    double* UT = (double*)malloc(sizeof(double) * (size_t)nb * nsx + 1);  /* n x ns   */
    double* Mx = (double*)malloc(sizeof(double) * (size_t)nb * nb + 1);   /* n x n    */
    double* Tt = (double*)malloc(sizeof(double) * (size_t)nsx * nsx + 1); /* ns x ns  */
    double* dv = (double*)malloc(sizeof(double) * (size_t)nb + 1);
    int nblocks = (N + nb - 1) / nb;
    for (int bk = 0; bk < nblocks; bk++) {
        int s0 = bk * nb, n = (s0 + nb <= N) ? nb : N - s0;
        /* (a) stripped force bias */
        for (int s = 0; s < 2; s++) {
            int m = ns[s];
            const double* t = T[s];
            for (int a = 0; a < n; a++) dv[a] = exp(-p->c[s] * xl[s0 + a]) - 1.0;
            for (int c = 0; c < m; c++)
                for (int a = 0; a < n; a++) {
                    double acc = 0.0;
                    for (int e = 0; e < m; e++) acc += t[(size_t)c * m + e] * dv[a] * UL[s][(size_t)e * N + s0 + a];
                    TV[(size_t)c * n + a] = acc;
                }
            for (int a = 0; a < n; a++)
                for (int c = 0; c < m; c++) {
                    double acc = 0.0;
                    for (int e = 0; e < m; e++) acc += UR[s][(size_t)(s0 + a) * m + e] * t[(size_t)e * m + c];
                    UT[(size_t)a * m + c] = acc;
                }
            for (int a = 0; a < n; a++)
                for (int b = 0; b < n; b++) {
                    double acc = (a == b ? 1.0 : 0.0);
                    for (int c = 0; c < m; c++) acc += UT[(size_t)a * m + c] * dv[b] * UL[s][(size_t)c * N + s0 + b];
                    Mx[(size_t)a * n + b] = acc;
                }
            double la;
            lu_factor(Mx, n, piv, &la);
            lu_solve(Mx, n, piv, UT, m); /* UT <- [1 + (U T) V]^{-1} (U T) */
            for (int c = 0; c < m; c++)
                for (int e = 0; e < m; e++) {
                    double acc = t[(size_t)c * m + e];
                    for (int a = 0; a < n; a++) acc -= TV[(size_t)c * n + a] * UT[(size_t)a * m + e];
                    Tt[(size_t)c * m + e] = acc;
                }
            for (int a = 0; a < n; a++) {
                int i = s0 + a;
                double acc = 0.0;
                for (int c = 0; c < m; c++) {
                    double w = 0.0;
                    for (int e = 0; e < m; e++) w += Tt[(size_t)c * m + e] * UL[s][(size_t)e * N + i];
                    acc += UR[s][(size_t)i * m + c] * w;
                }
                nbar[s][a] = (1.0 + dv[a]) * acc;
            }
        }
        /* (b) proposals, as or_blockfb_slice */
        double logprior = 0.0;
        int nF = 0;
        for (int a = 0; a < n; a++) {
            int i = s0 + a;
            double h = p->c[0] * nbar[0][a] + p->c[1] * nbar[1][a];
            double lp = hs_log_scalar(p, +1) + h, lm = hs_log_scalar(p, -1) - h;
            double lamp = 1.0 / (1.0 + exp(lm - lp));
            lam_plus[i] = lamp;
            int xp = replay ? (replay[i] ? +1 : -1) : (u_prop[i] < lamp ? +1 : -1);
            xprop[i] = (int8_t)xp;
            if (xp != xl[i]) {
                F[nF++] = i;
                double lbx = hs_log_scalar(p, xl[i]) + xl[i] * h;
                double lbxp = hs_log_scalar(p, xp) + xp * h;
                logprior += (hs_log_scalar(p, xp) - hs_log_scalar(p, xl[i])) + (lbx - lbxp);
            }
        }
        if (nF == 0) {
            dec[bk] = 1;
            ratio[bk] = 1.0;
            continue;
        }
        /* (c) r_s = det[1 + (U' T) V'] over the flipped sites */
        double R = exp(logprior);
        for (int s = 0; s < 2; s++) {
            int m = ns[s];
            const double* t = T[s];
            for (int a = 0; a < nF; a++) dv[a] = field_delta(p, s, xl[F[a]], -xl[F[a]]);
            for (int a = 0; a < nF; a++)
                for (int c = 0; c < m; c++) {
                    double acc = 0.0;
                    for (int e = 0; e < m; e++) acc += UR[s][(size_t)F[a] * m + e] * t[(size_t)e * m + c];
                    UT[(size_t)a * m + c] = acc;
                }
            for (int a = 0; a < nF; a++)
                for (int b = 0; b < nF; b++) {
                    double acc = (a == b ? 1.0 : 0.0);
                    for (int c = 0; c < m; c++) acc += UT[(size_t)a * m + c] * dv[b] * UL[s][(size_t)c * N + F[b]];
                    Mx[(size_t)a * nF + b] = acc;
                }
            double la;
            int sg = det_sign_log(Mx, nF, &la);
            R *= sg * exp(la);
        }
        int acc = replay ? (replay[N + bk] != 0) : (u_acc[bk] < fabs(R));
        dec[bk] = (uint8_t)acc;
        ratio[bk] = R;
        if (!acc) continue;
        /* (d) T <- T - (T V')[1 + (U' T) V']^{-1}(U' T);  U_R rows of F scaled by 1 + Delta */
        for (int s = 0; s < 2; s++) {
            int m = ns[s];
            double* t = T[s];
            for (int a = 0; a < nF; a++) dv[a] = field_delta(p, s, xl[F[a]], -xl[F[a]]);
            for (int c = 0; c < m; c++)
                for (int a = 0; a < nF; a++) {
                    double acc2 = 0.0;
                    for (int e = 0; e < m; e++) acc2 += t[(size_t)c * m + e] * dv[a] * UL[s][(size_t)e * N + F[a]];
                    TV[(size_t)c * nF + a] = acc2;
                }
            for (int a = 0; a < nF; a++)
                for (int c = 0; c < m; c++) {
                    double acc2 = 0.0;
                    for (int e = 0; e < m; e++) acc2 += UR[s][(size_t)F[a] * m + e] * t[(size_t)e * m + c];
                    UT[(size_t)a * m + c] = acc2;
                }
            for (int a = 0; a < nF; a++)
                for (int b = 0; b < nF; b++) {
                    double acc2 = (a == b ? 1.0 : 0.0);
                    for (int c = 0; c < m; c++) acc2 += UT[(size_t)a * m + c] * dv[b] * UL[s][(size_t)c * N + F[b]];
                    Mx[(size_t)a * nF + b] = acc2;
                }
            double la;
            lu_factor(Mx, nF, piv, &la);
            lu_solve(Mx, nF, piv, UT, m);
            for (int c = 0; c < m; c++)
                for (int e = 0; e < m; e++) {
                    double acc2 = 0.0;
                    for (int a = 0; a < nF; a++) acc2 += TV[(size_t)c * nF + a] * UT[(size_t)a * m + e];
                    t[(size_t)c * m + e] -= acc2;
                }
            for (int a = 0; a < nF; a++)
                for (int c = 0; c < m; c++) UR[s][(size_t)F[a] * m + c] *= 1.0 + dv[a];
        }
        for (int a = 0; a < nF; a++) xl[F[a]] = (int8_t)(-xl[F[a]]);
        if (R < 0) *sign = -*sign;
    }
    free(nbar[0]); free(nbar[1]); free(F); free(piv); free(TV); free(UT); free(Mx); free(Tt); free(dv);
}

/* ------------------------------------------------------------------ */
/* Block force-bias update  (Sec. III.B, Eqs. BlockFrcbsPhiLPhiR,      */
/* BlockFrcbsRatio, BlkFrcBsErr, BlkFrcBsTnew1, BlkFrcBsTnew2)          */
/* ------------------------------------------------------------------ */

/* Stripped force bias of one block S = [s0, s0+n) for spin s:
 *   Abar_SS = (1 + Db)(1 + A_SS Db)^{-1} A_SS,  Db_ii = e^{-c_s x_i} - 1,
 * the block of R~(L R~)^{-1} L with R~ = (1 + Db) R (the block's fields
 * removed); nbar_i = (Abar_SS)_ii.  A = 1 - G. */
void or_block_force_bias(const or_params* p, const double* g, const int8_t* xl, int s, int s0, int n,
                         double* nbar) {
    int N = p->N;
    double* A = (double*)malloc(sizeof(double) * (size_t)n * n + 1);
    double* Mx = (double*)malloc(sizeof(double) * (size_t)n * n + 1);
    double* db = (double*)malloc(sizeof(double) * (size_t)n + 1);
    int* piv = (int*)malloc(sizeof(int) * (size_t)n + 1);
    for (int a = 0; a < n; a++) db[a] = exp(-p->c[s] * xl[s0 + a]) - 1.0;
    for (int a = 0; a < n; a++)
        for (int b = 0; b < n; b++) {
            A[(size_t)a * n + b] = (a == b ? 1.0 : 0.0) - g[(size_t)(s0 + a) * N + (s0 + b)];
            Mx[(size_t)a * n + b] = (a == b ? 1.0 : 0.0) + A[(size_t)a * n + b] * db[b];
        }
    double la;
    lu_factor(Mx, n, piv, &la);
    lu_solve(Mx, n, piv, A, n); /* A <- (1 + A Db)^{-1} A */
    for (int a = 0; a < n; a++) nbar[a] = (1.0 + db[a]) * A[(size_t)a * n + a];
    free(A); free(Mx); free(db); free(piv);
}

/* Block force-bias pass over one slice, blocks of nb consecutive sites
 * (the last block is partial when nb does not divide N).
 * u_prop[i]: uniform for the proposal at site i; u_acc[b]: for block b's
 * Metropolis test.  replay (nullable): replay[i] = 1 proposes x'_i = +1,
 * replay[N + b] forces block b's decision.  Outputs: xprop[i] the proposed
 * field, lam_plus[i] the proposal probability of x' = +1, dec[b], ratio[b]
 * (the full Metropolis ratio including the prior ratio). */
void or_blockfb_slice(const or_params* p, double* G0, double* G1, int8_t* xl, const double* u_prop,
                      const double* u_acc, int nb, const uint8_t* replay, int8_t* xprop, double* lam_plus,
                      uint8_t* dec, double* ratio, double* sign) {
    int N = p->N;
    double* G[2] = {G0, G1};
    if (nb < 1) nb = 1;
    double* nbar[2];
    nbar[0] = (double*)malloc(sizeof(double) * (size_t)nb + 1);
    nbar[1] = (double*)malloc(sizeof(double) * (size_t)nb + 1);
    int* F = (int*)malloc(sizeof(int) * (size_t)nb + 1);
    double* Mf = (double*)malloc(sizeof(double) * (size_t)nb * nb + 1);
    double* W = (double*)malloc(sizeof(double) * (size_t)nb * nb + 1);
    double* Df = (double*)malloc(sizeof(double) * (size_t)nb + 1);
    int* piv = (int*)malloc(sizeof(int) * (size_t)nb + 1);
    double* X = (double*)malloc(sizeof(double) * (size_t)N * nb + 1);
    double* Y = (double*)malloc(sizeof(double) * (size_t)N * nb + 1);
    double* XW = (double*)malloc(sizeof(double) * (size_t)N * nb + 1);
    int nblocks = (N + nb - 1) / nb;
    for (int bk = 0; bk < nblocks; bk++) {
        int s0 = bk * nb, n = (s0 + nb <= N) ? nb : N - s0;
        for (int s = 0; s < 2; s++) or_block_force_bias(p, G[s], xl, s, s0, n, nbar[s]);
        /* proposals from lambda(x') = bbar(x') / sum_x bbar(x), bbar(x) = s(x) e^{x h} */
        double logprior = 0.0;
        int nF = 0;
        for (int a = 0; a < n; a++) {
            int i = s0 + a;
            double h = p->c[0] * nbar[0][a] + p->c[1] * nbar[1][a];
            double lp = hs_log_scalar(p, +1) + h, lm = hs_log_scalar(p, -1) - h;
            double lamp = 1.0 / (1.0 + exp(lm - lp));
            lam_plus[i] = lamp;
            int xp = replay ? (replay[i] ? +1 : -1) : (u_prop[i] < lamp ? +1 : -1);
            xprop[i] = (int8_t)xp;
            if (xp != xl[i]) {
                F[nF++] = i;
                /* W'/W prior part s(x')/s(x) times P(X'->X)/P(X->X') = bbar(x)/bbar(x') */
                double lbx = hs_log_scalar(p, xl[i]) + xl[i] * h;
                double lbxp = hs_log_scalar(p, xp) + xp * h;
                logprior += (hs_log_scalar(p, xp) - hs_log_scalar(p, xl[i])) + (lbx - lbxp);
            }
        }
        if (nF == 0) { /* proposal equals the current state: nothing changes */
            dec[bk] = 1;
            ratio[bk] = 1.0;
            continue;
        }
        double R = exp(logprior), rs[2];
        for (int s = 0; s < 2; s++) {
            for (int a = 0; a < nF; a++) Df[a] = field_delta(p, s, xl[F[a]], -xl[F[a]]);
            for (int a = 0; a < nF; a++)
                for (int b = 0; b < nF; b++) {
                    double Aab = (a == b ? 1.0 : 0.0) - G[s][(size_t)F[a] * N + F[b]];
                    Mf[(size_t)a * nF + b] = (a == b ? 1.0 : 0.0) + Aab * Df[b];
                }
            double la;
            int sg = det_sign_log(Mf, nF, &la);
            rs[s] = sg * exp(la);
            R *= rs[s];
        }
        int acc = replay ? (replay[N + bk] != 0) : (u_acc[bk] < fabs(R));
        dec[bk] = (uint8_t)acc;
        ratio[bk] = R;
        if (!acc) continue;
        for (int s = 0; s < 2; s++) {
            double* g = G[s];
            /* W = Df (1 + A_FF Df)^{-1} ; G <- G - G[:,F] W (E_F^T - G[F,:]) */
            for (int a = 0; a < nF; a++) Df[a] = field_delta(p, s, xl[F[a]], -xl[F[a]]);
            for (int a = 0; a < nF; a++)
                for (int b = 0; b < nF; b++) {
                    double Aab = (a == b ? 1.0 : 0.0) - g[(size_t)F[a] * N + F[b]];
                    Mf[(size_t)a * nF + b] = (a == b ? 1.0 : 0.0) + Aab * Df[b];
                }
            double la;
            lu_factor(Mf, nF, piv, &la);
            for (int a = 0; a < nF; a++)
                for (int b = 0; b < nF; b++) W[(size_t)a * nF + b] = (a == b ? 1.0 : 0.0);
            lu_solve(Mf, nF, piv, W, nF); /* W <- Mf^{-1} */
            for (int a = 0; a < nF; a++)
                for (int b = 0; b < nF; b++) W[(size_t)a * nF + b] *= Df[a];
            for (int j = 0; j < N; j++)
                for (int a = 0; a < nF; a++) {
                    X[(size_t)j * nF + a] = g[(size_t)j * N + F[a]];
                    Y[(size_t)a * N + j] = (j == F[a] ? 1.0 : 0.0) - g[(size_t)F[a] * N + j];
                }
            for (int j = 0; j < N; j++)
                for (int b = 0; b < nF; b++) {
                    double acc2 = 0.0;
                    for (int a = 0; a < nF; a++) acc2 += X[(size_t)j * nF + a] * W[(size_t)a * nF + b];
                    XW[(size_t)j * nF + b] = acc2;
                }
#pragma omp parallel for schedule(static)
            for (int a = 0; a < N; a++)
                for (int b = 0; b < N; b++) {
                    double acc2 = 0.0;
                    for (int q = 0; q < nF; q++) acc2 += XW[(size_t)a * nF + q] * Y[(size_t)q * N + b];
                    g[(size_t)a * N + b] -= acc2;
                }
        }
        for (int a = 0; a < nF; a++) xl[F[a]] = (int8_t)(-xl[F[a]]);
        if (R < 0) *sign = -*sign;
    }
    free(nbar[0]); free(nbar[1]); free(F); free(Mf); free(W); free(Df); free(piv);
    free(X); free(Y); free(XW);
}

/* ------------------------------------------------------------------ */
/* Energy  (Eqs. 2DHubbard, Oxformula): spin-decoupled Wick contraction */
/* ------------------------------------------------------------------ */

/* E = sum_s tr(K A^s) + U sum_i [A^up_ii A^dn_ii - (A^up_ii + A^dn_ii)/2], A = 1 - G,
 * with K the hopping matrix (row-major N x N). */
double or_energy(const or_params* p, const double* K, const double* G0, const double* G1) {
    int N = p->N;
    const double* G[2] = {G0, G1};
    double ekin = 0.0, epot = 0.0;
    for (int s = 0; s < 2; s++)
        for (int i = 0; i < N; i++)
            for (int j = 0; j < N; j++) {
                double Aji = (i == j ? 1.0 : 0.0) - G[s][(size_t)j * N + i];
                ekin += K[(size_t)i * N + j] * Aji;
            }
    for (int i = 0; i < N; i++) {
        double nu = 1.0 - G0[(size_t)i * N + i], nd = 1.0 - G1[(size_t)i * N + i];
        epot += nu * nd - 0.5 * (nu + nd);
    }
    return ekin + p->U * epot;
}

/* The hopping matrix K of the periodic nearest-neighbour lattice: K_ij = -t for
 * every bond (i, j) (bonds that wrap onto the same pair add up). */
void or_hopping(const or_params* p, double* K) {
    int Lx = p->Lx, Ly = p->Ly, N = p->N;
    memset(K, 0, sizeof(double) * (size_t)N * N);
    for (int y = 0; y < Ly; y++)
        for (int x = 0; x < Lx; x++) {
            int i = x + Lx * y;
            int nb[4] = {((x + 1) % Lx) + Lx * y, ((x - 1 + Lx) % Lx) + Lx * y,
                         x + Lx * ((y + 1) % Ly), x + Lx * ((y - 1 + Ly) % Ly)};
            for (int q = 0; q < 4; q++) K[(size_t)i * N + nb[q]] -= p->t;
        }
}
