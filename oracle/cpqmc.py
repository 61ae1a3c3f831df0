"""cpqmc.py -- plain FP64 numpy oracle of one projection step of ground-state constrained-path AFQMC
(CPQMC, Sec. IV.D) on the Hubbard model with the real decouplings of the Hubbard oracle.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the cpu_baseline / reference legs
of bench.py may import this module.  It shares no code with the CUDA library.

The walker ensemble represents |Psi> = sum_k w_k |phi_k> / <psi_T|phi_k> (Eq. CPWvfct1).  One step
applies e^{-dtau K} to every walker (w times <psi_T|e^{-dtau K} phi> / <psi_T|phi>) and then samples
the slice's fields from p~(x) = p(x) <psi_T|B(x)|phi> / <psi_T|phi> (Eqs. CPWvfct2, ptilde), with the
walker's weight multiplied by the normalisation, so that the expectation over the sampled fields
reproduces Eq. CPWvfct2.  Notation: per spin s the walker is U_R = phi_s (N x n_s), the trial enters as
U_L = psi_T,s^+ (n_s x N), T = (U_L U_R)^{-1}, and the mixed one-body matrix A = U_R T U_L
(A_ij = <c_j^+ c_i> between <psi_T| and |phi>; G = 1 - A).  The field of site i enters B(x) as
s(x) e^{c_s x} on the spin-s orbital i (s(x) = e^{-lam x} for the charge channel, 1 for the spin
channel; c_s the per-spin couplings of the model), so with Delta_s(x) = e^{c_s x} - 1:
  <psi_T| b_i(x) |phi> / <psi_T|phi> = s(x) prod_s (1 + Delta_s(x) A_s[i][i]).
Schemes (Sec. IV.D):
  local    sites in order, heat bath: lambda(x) = p(x) s(x) prod_s r_s(x), p = 1/2, constrained path
           lambda(x) <- max(lambda(x), 0); x = +1 iff u_i < lambda(+1) / N_i, N_i = lambda(+1) +
           lambda(-1); w <- w N_i; a walker with N_i = 0 is removed (w = 0).  The delayed update
           reorganises the same sequence (same fields and weights).
  blockfb  blocks of n_b sites: the force bias F_i = sum_s c_s A_s[i][i] (spin channel) or
           lam (A_up[i][i] + A_dn[i][i] - 1) (charge channel) of the block's sites before any of
           them is set; each x_i drawn from q(x_i) = p(x_i) e^{x_i F_i} / Nbar_i, Nbar_i = cosh F_i;
           then w <- w prod_i (s(x_i) Nbar_i e^{-x_i F_i}) prod_s det(1 + Delta_s A_s[S][S])
           (the exact overlap ratio over the proposal), removed if that factor is <= 0.  n_b = N
           is the full force-bias scheme.
Population control (the comb): positions (j + u0) W / n_w of the cumulative weights W select the new
walkers, each with weight W / n_w.
"""
import numpy as np


class CPEnsemble:
    """n_w walkers of the Hubbard model `model` (oracle.Model, real decoupling) guided by the trial
    determinant P (N x n_s, real, the same for both spins)."""

    def __init__(self, model, P, n_w, phi0=None):
        self.m = model
        self.P = np.ascontiguousarray(P, dtype=np.float64)
        self.UL = self.P.T.copy()
        phi = self.P if phi0 is None else np.asarray(phi0, dtype=np.float64)
        self.UR = [[phi.copy(), phi.copy()] for _ in range(n_w)]
        self.w = np.ones(n_w)
        self.charge = model.p.hs == 1

    def s(self, x):
        return np.exp(-self.m.lam * x) if self.charge else 1.0

    def A(self, k, s):
        """Mixed one-body matrix of walker k, spin s: U_R (U_L U_R)^{-1} U_L."""
        UR = self.UR[k][s]
        return UR @ np.linalg.solve(self.UL @ UR, self.UL)

    def overlap(self, k):
        return np.prod([np.linalg.det(self.UL @ self.UR[k][s]) for s in range(2)])

    def kinetic(self):
        """phi <- e^{-dtau K} phi with w <- w <psi_T|e^{-dtau K} phi> / <psi_T|phi>: the part of the
        normalisation of p~ (Eq. ptilde) that the kinetic factor of B(x) carries; a walker whose
        overlap would turn non-positive is removed (the constraint)."""
        for k in range(len(self.w)):
            if self.w[k] == 0.0:
                continue
            before = self.overlap(k)
            for s in range(2):
                self.UR[k][s] = self.m.E @ self.UR[k][s]
            ratio = self.overlap(k) / before
            self.w[k] = self.w[k] * ratio if ratio > 0.0 else 0.0

    def _set_field(self, k, i, x):
        c = self.m.c
        for s in range(2):
            self.UR[k][s][i, :] *= np.exp(c[s] * x)

    def local_fields(self, k, u):
        """Heat-bath fields of one slice for walker k (after the kinetic step); returns the fields,
        per site the normalisation N_i and P(x_i = +1)."""
        N, c = self.m.N, self.m.c
        x = np.zeros(N, np.int8)
        norm = np.zeros(N)
        pplus = np.zeros(N)
        for i in range(N):
            lam = {}
            for xv in (+1, -1):
                r = 1.0
                for s in range(2):
                    r *= 1.0 + (np.exp(c[s] * xv) - 1.0) * self.A(k, s)[i, i]
                lam[xv] = max(0.5 * self.s(xv) * r, 0.0)
            Ni = lam[+1] + lam[-1]
            norm[i] = Ni
            if Ni <= 0.0:
                self.w[k] = 0.0
                return x, norm, pplus
            pplus[i] = lam[+1] / Ni
            x[i] = 1 if u[i] < pplus[i] else -1
            self.w[k] *= Ni
            self._set_field(k, i, x[i])
        return x, norm, pplus

    def block_fields(self, k, u, nb):
        """Block force-bias fields of one slice for walker k; returns the fields, per block the
        weight factor, and per site P(x_i = +1) of the proposal."""
        N, c, lamc = self.m.N, self.m.c, self.m.lam
        x = np.zeros(N, np.int8)
        pplus = np.zeros(N)
        nblocks = (N + nb - 1) // nb
        fac = np.zeros(nblocks)
        for b in range(nblocks):
            S = np.arange(b * nb, min(N, (b + 1) * nb))
            A = [self.A(k, s) for s in range(2)]
            if self.charge:
                F = lamc * (A[0][S, S] + A[1][S, S] - 1.0)
            else:
                F = c[0] * A[0][S, S] + c[1] * A[1][S, S]
            pp = np.exp(F) / (np.exp(F) + np.exp(-F))
            pplus[S] = pp
            xs = np.where(u[S] < pp, 1, -1)
            x[S] = xs
            f = np.prod(self.s(xs) * np.cosh(F) * np.exp(-xs * F))
            for s in range(2):
                D = np.diag(np.exp(c[s] * xs) - 1.0)
                f *= np.linalg.det(np.eye(len(S)) + D @ A[s][np.ix_(S, S)])
            fac[b] = f
            if not f > 0.0:
                self.w[k] = 0.0
                return x, fac, pplus
            self.w[k] *= f
            for a, i in enumerate(S):
                self._set_field(k, i, xs[a])
        return x, fac, pplus

    def step(self, mode, u, nb=4):
        """One projection step for every live walker: e^{-dtau K}, then the slice's fields.
        u: n_w x N uniforms.  Returns per walker (fields, factors, P(x = +1))."""
        self.kinetic()
        out = []
        for k in range(len(self.w)):
            if self.w[k] == 0.0:
                out.append((np.zeros(self.m.N, np.int8), None, None))
                continue
            out.append(self.local_fields(k, u[k]) if mode == "local" else self.block_fields(k, u[k], nb))
        return out

    def reorthonormalise(self):
        """QR of every walker's factors: |phi> changes by a scale only, which Eq. CPWvfct1 divides out."""
        for k in range(len(self.w)):
            for s in range(2):
                self.UR[k][s] = np.linalg.qr(self.UR[k][s])[0]

    def comb(self, u0):
        """Population control: returns the indices of the walkers kept (with repetition)."""
        n = len(self.w)
        W = self.w.sum()
        cum = np.cumsum(self.w)
        pos = (np.arange(n) + u0) * W / n
        idx = np.searchsorted(cum, pos, side="right")
        idx = np.minimum(idx, n - 1)
        self.UR = [[self.UR[j][0].copy(), self.UR[j][1].copy()] for j in idx]
        self.w = np.full(n, W / n)
        return idx

    def local_energy(self, k):
        """Mixed estimator <psi_T|H|phi_k> / <psi_T|phi_k> (Eqs. 2DHubbard, Oxformula)."""
        A = [self.A(k, s) for s in range(2)]
        e = sum(np.sum(self.m.K * A[s].T) for s in range(2))
        d = np.diag(A[0]) * np.diag(A[1]) - 0.5 * (np.diag(A[0]) + np.diag(A[1]))
        return float(e + self.m.p.U * d.sum())

    def energy(self):
        live = self.w > 0
        el = np.array([self.local_energy(k) if live[k] else 0.0 for k in range(len(self.w))])
        return float(np.sum(self.w * el) / np.sum(self.w))
