"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test compares the oracle with something that is not the oracle: scipy's
matrix exponential, numpy determinants of the walker overlap (Eq. ConfgWeight),
the closed-form free-fermion energy, the Fock-space expectation value, or the
exact transition kernel of an enumerable toy chain.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2506_09611_gb300 import inputs
from tests import bruteforce as bf

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _model(Lx, Ly, U=4.0, dtau=0.05, M=8, hs=oracle.HS_SZ_REAL, t=1.0):
    return oracle.Model(Lx, Ly, t, U, dtau, M, hs)


def _log_scalar(m):
    if m.p.hs == oracle.HS_CHARGE_REAL:
        return lambda v: -m.lam * v
    return None


# ---------------------------------------------------------------- model (Eq. 2DHubbard)

@pytest.mark.parametrize("Lx,Ly", [(4, 4), (5, 3), (2, 3), (3, 1)])
def test_expK_matches_expm(Lx, Ly):
    m = _model(Lx, Ly, dtau=0.07)
    K = inputs.hopping_matrix(Lx, Ly)
    np.testing.assert_allclose(m.K, K, atol=0)
    np.testing.assert_allclose(m.E, bf.expK(K, 0.07), atol=1e-13)
    np.testing.assert_allclose(m.Einv, bf.expK(K, -0.07), atol=1e-13)
    np.testing.assert_allclose(m.E @ m.Einv, np.eye(Lx * Ly), atol=1e-13)


def test_hopping_spectrum_is_dispersion():
    Lx, Ly = 6, 4
    m = _model(Lx, Ly)
    eps = sorted(-2 * (np.cos(2 * np.pi * nx / Lx) + np.cos(2 * np.pi * ny / Ly))
                 for nx in range(Lx) for ny in range(Ly))
    np.testing.assert_allclose(np.linalg.eigvalsh(m.K), eps, atol=1e-12)


@pytest.mark.parametrize("hs,U", [(oracle.HS_SZ_REAL, 4.0), (oracle.HS_SZ_REAL, 6.0),
                                  (oracle.HS_CHARGE_REAL, -4.0)])
def test_hs_identity_all_occupations(hs, U):
    """(1/2) sum_x s(x) exp(x (c_up n_up + c_dn n_dn)) = C exp(-dtau U (n_up n_dn - (n_up+n_dn)/2))
    with one occupation-independent constant C (C = 1 for the spin channel)."""
    dtau = 0.05
    m = _model(2, 2, U=U, dtau=dtau, hs=hs)
    ls = _log_scalar(m) or (lambda v: 0.0)
    ratios = []
    for nu, nd in itertools.product((0, 1), repeat=2):
        rhs = 0.5 * sum(np.exp(ls(x) + x * (m.c[0] * nu + m.c[1] * nd)) for x in (-1, 1))
        lhs = np.exp(-dtau * U * (nu * nd - 0.5 * (nu + nd)))
        ratios.append(rhs / lhs)
    np.testing.assert_allclose(ratios, ratios[0], rtol=1e-14)
    if hs == oracle.HS_SZ_REAL:
        assert abs(ratios[0] - 1.0) < 1e-14


# ---------------------------------------------------------------- G (Eqs. GrFMat, GrFMatNew)

def _setup(Lx, Ly, ns, M, seed=3, U=4.0, hs=oracle.HS_SZ_REAL, dtau=0.1):
    m = _model(Lx, Ly, U=U, M=M, hs=hs, dtau=dtau)
    P = inputs.trial_state(Lx, Ly, ns)
    X = inputs.initial_fields(M, Lx * Ly, seed=seed)
    return m, P, X


@pytest.mark.parametrize("ell", [0, 3, 8])
def test_green_scratch_matches_plain_products(ell):
    m, P, X = _setup(3, 3, 4, 8)
    for s in range(2):
        G, sg, la = m.green_scratch(X, P, s, ell, stab=2)
        np.testing.assert_allclose(G, bf.green(m.E, m.c[s], X, P, ell), atol=1e-12)
        det = bf.overlap(m.E, m.c[s], X, P)
        assert sg == np.sign(det)
        assert abs(la - np.log(abs(det))) < 1e-10


def test_projector_invariants():
    """A = 1 - G is a rank-n_sigma projector: G^2 = G and tr(1 - G) = n_sigma."""
    m, P, X = _setup(4, 4, 7, 12)
    for ell in (0, 5, 12):
        for s in range(2):
            G, _, _ = m.green_scratch(X, P, s, ell, stab=3)
            np.testing.assert_allclose(G @ G, G, atol=1e-11)
            assert abs(np.trace(np.eye(16) - G) - 7) < 1e-11


def test_wrap_matches_scratch():
    m, P, X = _setup(3, 3, 4, 8)
    for s in range(2):
        G3 = bf.green(m.E, m.c[s], X, P, 3)
        np.testing.assert_allclose(m.wrap(G3, X[3], s, +1), bf.green(m.E, m.c[s], X, P, 4), atol=1e-12)
        np.testing.assert_allclose(m.wrap(G3, X[2], s, -1), bf.green(m.E, m.c[s], X, P, 2), atol=1e-12)


# ---------------------------------------------------------------- local update

@pytest.mark.parametrize("hs,U", [(oracle.HS_SZ_REAL, 4.0), (oracle.HS_CHARGE_REAL, -4.0)])
def test_local_ratio_is_bruteforce_weight_ratio(hs, U):
    """R_i = W(X with x_{l,i} flipped) / W(X)  (Eqs. DetailBalance, DetRatio00, DetRatiolocal)."""
    m, P, X = _setup(3, 2, 2, 6, U=U, hs=hs)
    ell = 3
    Gs = [bf.green(m.E, m.c[s], X, P, ell) for s in range(2)]
    ls = _log_scalar(m)
    W0 = bf.weight(m.E, m.c, X, P, P, ls)
    # forced decisions: accept sites 1 and 4 only; every ratio is checked against brute force
    forced = np.zeros(m.N, np.uint8)
    forced[[1, 4]] = 1
    u = np.zeros(m.N)
    Gu, Gd, xl, dec, ratio, sg = m.local_slice(Gs[0], Gs[1], X[ell - 1], u, replay=forced)
    Xc = X.copy()
    Wc = W0
    for i in range(m.N):
        Xf = Xc.copy()
        Xf[ell - 1, i] *= -1
        Wf = bf.weight(m.E, m.c, Xf, P, P, ls)
        assert abs(ratio[i] - Wf / Wc) < 1e-10 * max(1, abs(Wf / Wc))
        if forced[i]:
            Xc, Wc = Xf, Wf
    np.testing.assert_array_equal(xl, Xc[ell - 1])
    np.testing.assert_allclose(Gu, bf.green(m.E, m.c[0], Xc, P, ell), atol=1e-11)
    np.testing.assert_allclose(Gd, bf.green(m.E, m.c[1], Xc, P, ell), atol=1e-11)
    assert sg == np.sign(Wc / W0)


def test_local_free_running_sweep_tracks_scratch_and_weight():
    """A forward sweep of local updates: after every slice G equals the from-scratch G of the
    current fields, and the product of accepted ratios telescopes to W(X_end)/W(X_start)."""
    Lx, Ly, ns, M = 4, 4, 7, 6
    m, P, X = _setup(Lx, Ly, ns, M, dtau=0.05)
    w = oracle.Walker(m, P, P, X)
    logprod = 0.0
    W0 = bf.weight(m.E, m.c, X, P, P)
    for ell in range(1, M + 1):
        u = inputs.uniforms(1, 0, ell, 2 * m.N)
        dec, ratio, _ = w.sweep_slice(ell, +1, "local", u)
        logprod += np.sum(np.log(np.abs(ratio[dec == 1])))
        for s in range(2):
            np.testing.assert_allclose(w.G[s], bf.green(m.E, m.c[s], w.x, P, ell), atol=1e-10)
    W1 = bf.weight(m.E, m.c, w.x, P, P)
    assert abs(logprod - np.log(abs(W1 / W0))) < 1e-9
    assert w.sign == np.sign(W1 / W0)


def _negative_weight_case():
    """A seeded 3 x 2 case (2 particles per spin, U = 8, dtau = 0.1) where flipping every field of
    slice 3 takes the weight W(X) = prod_s det(P^T B_M..B_1 P) (Eq. ConfgWeight) to the opposite
    sign: the real spin decoupling has a sign problem away from half filling."""
    m, P, X = _setup(3, 2, 2, 6, seed=4, U=8.0, dtau=0.1)
    ell = 3
    Xf = X.copy()
    Xf[ell - 1] *= -1
    W0, W1 = bf.weight(m.E, m.c, X, P, P), bf.weight(m.E, m.c, Xf, P, P)
    assert W1 / W0 < 0  # the case really crosses a sign change
    return m, P, X, Xf, ell


@pytest.mark.parametrize("scheme", ["local", "delayed-k2", "delayed-k4", "delayed-s1-k3", "blockfb-1", "blockfb-2",
                                    "blockfb-6", "tform-delayed-k2", "tform-blockfb-2"])
def test_sign_follows_the_weight_through_negative_ratios(scheme):
    """Every scheme multiplies the walker sign by sign(R) of each accepted move (Eq. DetailBalance
    with |R|): forcing every flip of a slice whose weight changes sign gives sign -1, with the
    final G (or the T-form factors) equal to the from-scratch result."""
    m, P, X, Xf, ell = _negative_weight_case()
    N = m.N
    Gs = [bf.green(m.E, m.c[s], X, P, ell) for s in range(2)]
    zeros = np.zeros(N)
    if scheme == "local" or scheme.startswith("delayed"):
        forced = np.ones(N, np.uint8)
        if scheme == "local":
            Gu, Gd, xl, dec, ratio, sg = m.local_slice(Gs[0], Gs[1], X[ell - 1], zeros, replay=forced)
        else:
            k = int(scheme.split("k")[-1])
            strategy = 1 if "-s1-" in scheme else 2
            Gu, Gd, xl, dec, ratio, sg, _ = m.delayed_slice(Gs[0], Gs[1], X[ell - 1], zeros, k, strategy, forced)
        assert (ratio < 0).any()
    elif scheme.startswith("blockfb"):
        nb = int(scheme.split("-")[1])
        nblk = (N + nb - 1) // nb
        rep = np.concatenate([(Xf[ell - 1] > 0).astype(np.uint8), np.ones(nblk, np.uint8)])
        Gu, Gd, xl, xprop, _, dec, ratio, sg = m.blockfb_slice(Gs[0], Gs[1], X[ell - 1], zeros, np.zeros(nblk),
                                                              nb, replay=rep)
        np.testing.assert_array_equal(xprop, Xf[ell - 1])
    else:
        UR, UL, T = [], [], []
        for s in range(2):
            _, _, _, ur, ul = m.green_scratch(X, P, s, ell, stab=2, want_factors=True)
            UR.append(ur)
            UL.append(ul)
            T.append(np.linalg.inv(ul @ ur))
        if scheme == "tform-delayed-k2":
            URn, Tn, xl, dec, ratio, sg, _ = m.tform_delayed_slice(UR, UL, T, X[ell - 1], zeros, 2, 2,
                                                                   np.ones(N, np.uint8))
        else:
            nblk = (N + 1) // 2
            rep = np.concatenate([(Xf[ell - 1] > 0).astype(np.uint8), np.ones(nblk, np.uint8)])
            URn, Tn, xl, _, _, dec, ratio, sg = m.tform_blockfb_slice(UR, UL, T, X[ell - 1], zeros, np.zeros(nblk),
                                                                      2, replay=rep)
        Gu, Gd = (np.eye(N) - URn[s] @ Tn[s] @ UL[s] for s in range(2))
    assert dec.all()
    np.testing.assert_array_equal(xl, Xf[ell - 1])
    assert sg == -1.0
    np.testing.assert_allclose(Gu, bf.green(m.E, m.c[0], Xf, P, ell), atol=1e-9)
    np.testing.assert_allclose(Gd, bf.green(m.E, m.c[1], Xf, P, ell), atol=1e-9)


@pytest.mark.parametrize("nb", [1, 3, 16])
def test_block_proposals_equal_to_the_current_fields_are_accepted_unchanged(nb):
    """A block whose proposal repeats its current fields is the null move: no site flips, R = 1
    and u < min(1, |R|) holds for every u in [0, 1).  It is accepted, with ratio 1, and G, the
    fields and the sign stay exactly as they were."""
    m, P, X = _setup(4, 4, 7, 6)
    N, ell = m.N, 2
    Gs = [bf.green(m.E, m.c[s], X, P, ell) for s in range(2)]
    xl = X[ell - 1]
    top = 1.0 - 2.0 ** -53  # the largest uniform below 1
    u_prop = np.where(xl > 0, 0.0, top)  # x' = +1 iff u_prop < lambda(+1), which lies strictly inside (0, 1)
    nblk = (N + nb - 1) // nb
    Gu, Gd, x1, xprop, lamp, dec, ratio, sg = m.blockfb_slice(Gs[0], Gs[1], xl, u_prop, np.full(nblk, top), nb)
    assert np.all((lamp > 0) & (lamp < top))
    np.testing.assert_array_equal(xprop, xl)
    assert dec.all() and sg == 1.0
    np.testing.assert_array_equal(ratio, np.ones(nblk))
    np.testing.assert_array_equal(x1, xl)
    np.testing.assert_array_equal(Gu, Gs[0])
    np.testing.assert_array_equal(Gd, Gs[1])


def test_local_acceptance_is_high_and_falls_with_the_coupling():
    """The paper reports local-update acceptance ratios above 0.8 for its Hubbard runs with a
    two-component discrete decoupling (Sec. III.A; Sec. IV.B.1, independent of L).  Seeded 6 x 6
    chains (15 per spin, dtau = 0.05, 8 slices, 3 seeds) accept 88% of the flips at U = 4, and
    fewer at U = 6, where the field couples more strongly."""
    def acceptance(U):
        acc = []
        for seed in range(3):
            m, P, X = _setup(6, 6, 15, 8, seed=seed, U=U, dtau=0.05)
            w = oracle.Walker(m, P, P, X)
            for ell in range(1, 9):
                dec, _, _ = w.sweep_slice(ell, +1, "local", inputs.uniforms(seed, 0, ell, 2 * m.N))
                acc.append(dec.mean())
        return float(np.mean(acc))

    a4, a6 = acceptance(4.0), acceptance(6.0)
    assert a4 > 0.85 and a6 < a4


@pytest.mark.parametrize("F", [[3], [1, 5, 6, 11], [0, 2, 7, 8, 9, 13, 15]])
def test_t_form_update_with_the_g_form_w(F):
    """The T-form window update a GPU path would apply with the window kernel's (G-form) W:
    W = Delta_F (1 + A_FF Delta_F)^{-1} (Eq. BlkFrcBsTnew2), T' = T - (T U_L[:, F]) W (U_R[F, :] T)
    and U_R's rows F scaled by 1 + Delta_F give 1 - U_R' T' U_L = the from-scratch G after the
    flips at F, which is also the G-form update G - G[:, F] W (E_F^T - G[F, :])."""
    m, P, X = _setup(4, 4, 7, 4)
    ell, N = 2, m.N
    Xf = X.copy()
    Xf[ell - 1, F] *= -1
    for s in range(2):
        _, _, _, UR, UL = m.green_scratch(X, P, s, ell, stab=2, want_factors=True)
        T = np.linalg.inv(UL @ UR)
        G = np.eye(N) - UR @ T @ UL
        dF = np.exp(-2.0 * m.c[s] * X[ell - 1, F]) - 1.0
        AFF = np.eye(len(F)) - G[np.ix_(F, F)]
        W = np.diag(dF) @ np.linalg.inv(np.eye(len(F)) + AFF @ np.diag(dF))
        V, Y = T @ UL[:, F], UR[F, :] @ T
        T1 = T - V @ W @ Y
        UR1 = UR.copy()
        UR1[F, :] *= (1.0 + dF)[:, None]
        G_t = np.eye(N) - UR1 @ T1 @ UL
        E_F = np.eye(N)[:, F]
        G_g = G - G[:, F] @ W @ (E_F.T - G[F, :])
        G_bf = bf.green(m.E, m.c[s], Xf, P, ell)
        np.testing.assert_allclose(G_t, G_bf, atol=1e-10)
        np.testing.assert_allclose(G_g, G_bf, atol=1e-10)


# ---------------------------------------------------------------- delayed update

@pytest.mark.parametrize("k,strategy", [(1, 2), (3, 2), (8, 2), (5, 1), (16, 1)])
def test_delayed_equals_local(k, strategy):
    """Same uniforms -> identical decisions; G agrees with the local update to 1e-12."""
    Lx, Ly, ns, M = 4, 4, 7, 4
    m, P, X = _setup(Lx, Ly, ns, M, dtau=0.05)
    wl = oracle.Walker(m, P, P, X)
    wd = oracle.Walker(m, P, P, X)
    for ell in range(1, M + 1):
        u = inputs.uniforms(7, 0, ell, 2 * m.N)
        dl, rl, _ = wl.sweep_slice(ell, +1, "local", u)
        dd, rd, ex = wd.sweep_slice(ell, +1, "delayed", u, k=k, strategy=strategy)
        np.testing.assert_array_equal(dl, dd)
        np.testing.assert_allclose(rd, rl, rtol=1e-11)
        for s in range(2):
            assert np.linalg.norm(wd.G[s] - wl.G[s]) / np.linalg.norm(wl.G[s]) < 1e-12
            np.testing.assert_allclose(wd.G[s], bf.green(m.E, m.c[s], wd.x, P, ell), atol=1e-10)
    assert wl.sign == wd.sign


# ---------------------------------------------------------------- block force-bias update

def test_block_force_bias_is_bruteforce_stripped_density():
    """nbar_i = [R~ (L R~)^{-1} L]_ii with R~ = B_I^(b)(x_l)^{-1} R  (Eq. BlockFrcbsPhiLPhiR)."""
    m, P, X = _setup(3, 3, 4, 6)
    ell, s0, n = 4, 2, 4
    for s in range(2):
        G = bf.green(m.E, m.c[s], X, P, ell)
        R, L = bf.products(m.E, m.c[s], X, P, ell)
        strip = np.ones(m.N)
        strip[s0:s0 + n] = np.exp(-m.c[s] * X[ell - 1, s0:s0 + n])
        Rt = np.diag(strip) @ R
        At = Rt @ np.linalg.solve(L @ Rt, L)
        np.testing.assert_allclose(m.block_force_bias(G, X[ell - 1], s, s0, n), np.diag(At)[s0:s0 + n],
                                   atol=1e-12)


def test_blockfb_ratio_and_update_bruteforce():
    """Forced proposals: the Metropolis ratio equals W(X')/W(X) times the prior ratio
    prod bbar(x)/bbar(x'); accepted blocks give the from-scratch G (Eq. BlkFrcBsTnew2)."""
    m, P, X = _setup(3, 3, 4, 6)
    ell, nb = 3, 4
    N = m.N
    nblocks = (N + nb - 1) // nb
    Gs = [bf.green(m.E, m.c[s], X, P, ell) for s in range(2)]
    rng = np.random.default_rng(11)
    rep = np.zeros(N + nblocks, np.uint8)
    rep[:N] = rng.integers(0, 2, N)
    rep[N:] = [1, 0, 1]
    Gu, Gd, xl, xprop, lamp, dec, ratio, sg = m.blockfb_slice(Gs[0], Gs[1], X[ell - 1], np.zeros(N),
                                                             np.zeros(nblocks), nb, replay=rep)
    Xc = X.copy()
    for b in range(nblocks):
        S = list(range(b * nb, min(N, b * nb + nb)))
        Xp = Xc.copy()
        Xp[ell - 1, S] = xprop[S]
        W = bf.weight(m.E, m.c, Xc, P, P)
        Wp = bf.weight(m.E, m.c, Xp, P, P)
        # proposal probabilities: lambda_i(x') from the oracle, lambda_i(x) = complement
        q_fwd = np.prod([lamp[i] if xprop[i] > 0 else 1 - lamp[i] for i in S])
        q_bwd = np.prod([lamp[i] if Xc[ell - 1, i] > 0 else 1 - lamp[i] for i in S])
        assert abs(ratio[b] - (Wp / W) * (q_bwd / q_fwd)) < 1e-10 * max(1.0, abs(ratio[b]))
        if rep[N + b]:
            Xc = Xp
    np.testing.assert_array_equal(xl, Xc[ell - 1])
    np.testing.assert_allclose(Gu, bf.green(m.E, m.c[0], Xc, P, ell), atol=1e-11)
    np.testing.assert_allclose(Gd, bf.green(m.E, m.c[1], Xc, P, ell), atol=1e-11)


def test_blockfb_exact_detailed_balance():
    """Exact enumeration on a 2-site, 2-slice toy (16 configurations): the block move's
    kernel T(X->X') = q(X->X') min(1, |R|) satisfies |W(X)| T(X->X') = |W(X')| T(X'->X)."""
    Lx, Ly, M, nb = 2, 1, 2, 2
    m = _model(Lx, Ly, U=6.0, M=M, dtau=0.3)
    P = inputs.trial_state(Lx, Ly, 1)
    N = m.N
    ell = 2
    configs = [np.array(c, np.int8).reshape(M, N) for c in itertools.product((-1, 1), repeat=M * N)]
    key = lambda X: tuple(X.ravel())
    W = {key(X): bf.weight(m.E, m.c, X, P, P) for X in configs}
    T = {}
    for X in configs:
        Gs = [bf.green(m.E, m.c[s], X, P, ell) for s in range(2)]
        for xp in itertools.product((-1, 1), repeat=N):
            rep = np.zeros(N + 1, np.uint8)
            rep[:N] = [1 if v > 0 else 0 for v in xp]
            _, _, _, xprop, lamp, dec, ratio, _ = m.blockfb_slice(Gs[0], Gs[1], X[ell - 1], np.zeros(N),
                                                                 np.zeros(1), nb, replay=rep)
            q = np.prod([lamp[i] if xp[i] > 0 else 1 - lamp[i] for i in range(N)])
            Xp = X.copy()
            Xp[ell - 1] = xp
            T[(key(X), key(Xp))] = q * min(1.0, abs(ratio[0]))
    checked = 0
    for (a, b), tab in T.items():
        if a == b:
            continue
        lhs = abs(W[a]) * tab
        rhs = abs(W[b]) * T[(b, a)]
        assert abs(lhs - rhs) < 1e-12 * max(abs(lhs), abs(rhs), 1e-300)
        checked += 1
    assert checked == 16 * 3


def test_blockfb_nb1_is_heatbath_local_move():
    """With n_b = 1 the block move proposes x' from lambda and its ratio for a flip is the
    local ratio times the prior ratio bbar(x)/bbar(-x)."""
    m, P, X = _setup(3, 3, 4, 6)
    ell = 2
    N = m.N
    Gs = [bf.green(m.E, m.c[s], X, P, ell) for s in range(2)]
    rep = np.zeros(2 * N, np.uint8)
    rep[:N] = (X[ell - 1] < 0).astype(np.uint8)  # propose the flip everywhere, reject all
    _, _, _, xprop, lamp, dec, ratio, _ = m.blockfb_slice(Gs[0], Gs[1], X[ell - 1], np.zeros(N),
                                                         np.zeros(N), 1, replay=rep)
    _, _, _, _, rl, _ = m.local_slice(Gs[0], Gs[1], X[ell - 1], np.zeros(N), replay=np.zeros(N, np.uint8))
    for i in range(N):
        x = X[ell - 1, i]
        lam_x = lamp[i] if x > 0 else 1 - lamp[i]
        assert abs(ratio[i] - rl[i] * lam_x / (1 - lam_x)) < 1e-12 * max(1, abs(ratio[i]))


# ---------------------------------------------------------------- energy (Eq. Oxformula)

@pytest.mark.parametrize("L,ns,expect", [(4, 7, -24.0), (6, 13, None)])
def test_energy_free_fermion_closed_form(L, ns, expect):
    """U = 0: E = 2 * (sum of the lowest n_sigma single-particle energies eps_k)."""
    m = _model(L, L, U=0.0, M=10)
    P = inputs.trial_state(L, L, ns)
    X = inputs.initial_fields(10, L * L)
    Gs = [m.green_scratch(X, P, s, 5)[0] for s in range(2)]
    eps = sorted(-2 * (np.cos(2 * np.pi * a / L) + np.cos(2 * np.pi * b / L)) for a in range(L) for b in range(L))
    closed = 2 * sum(eps[:ns])
    if expect is not None:
        assert abs(closed - expect) < 1e-12
    assert abs(m.energy(Gs[0], Gs[1]) - closed) < 1e-10


@pytest.mark.parametrize("U", [4.0, -3.0])
def test_energy_matches_fock_space(U):
    """Wick-contracted mixed estimator = <psi_l|H|psi_r>/<psi_l|psi_r> on the Fock space (3 sites)."""
    Lx, Ly = 3, 1
    hs = oracle.HS_SZ_REAL if U >= 0 else oracle.HS_CHARGE_REAL
    m = _model(Lx, Ly, U=U, hs=hs)
    rng = np.random.default_rng(5)
    Ru, Rd = rng.standard_normal((3, 1)), rng.standard_normal((3, 2))
    Lu, Ld = rng.standard_normal((1, 3)), rng.standard_normal((2, 3))
    Gu = np.eye(3) - Ru @ np.linalg.solve(Lu @ Ru, Lu)
    Gd = np.eye(3) - Rd @ np.linalg.solve(Ld @ Rd, Ld)
    e_fock = bf.fock_energy(m.K, U, Ru, Lu, Rd, Ld)
    assert abs(m.energy(Gu, Gd) - e_fock) < 1e-10


# ---------------------------------------------------------------- T form (Sec. II.C, Sec. III.A)

def test_tform_wrap_keeps_overlap_and_moves_G():
    """Forward and backward T-form wraps leave U_L U_R (hence T) unchanged, and 1 - U_R T U_L of the
    moved factors is the from-scratch G of the new slice (Eqs. BlMat, GrFMatNew)."""
    m, P, X = _setup(3, 3, 4, 6)
    ell = 2
    for s in range(2):
        _, _, _, UR, UL = m.green_scratch(X, P, s, ell, stab=2, want_factors=True)
        T = np.linalg.inv(UL @ UR)
        for direction, xl, target in ((+1, X[ell], ell + 1), (-1, X[ell - 1], ell - 1)):
            URw, ULw = m.tform_wrap(UR, UL, xl, s, direction)
            np.testing.assert_allclose(ULw @ URw, UL @ UR, atol=1e-12)
            G = np.eye(m.N) - URw @ T @ ULw
            np.testing.assert_allclose(G, bf.green(m.E, m.c[s], X, P, target), atol=1e-11)


def test_tform_local_ratio_is_bruteforce_weight_ratio():
    """k = 1 T-form steps (Eqs. DetRatiolocal, UpdateLTRlocal): every r_up r_dn equals the brute-force
    weight ratio of the flip, with forced acceptances changing U_R and T along the way; T stays the
    inverse overlap and 1 - U_R T U_L the from-scratch G."""
    m, P, X = _setup(3, 2, 2, 6)
    ell = 3
    UR, UL, T = [], [], []
    for s in range(2):
        _, _, _, ur, ul = m.green_scratch(X, P, s, ell, stab=2, want_factors=True)
        UR.append(ur)
        UL.append(ul)
        T.append(np.linalg.inv(ul @ ur))
    W0 = bf.weight(m.E, m.c, X, P, P)
    forced = np.zeros(m.N, np.uint8)
    forced[[0, 3, 4]] = 1
    URn, Tn, xl, dec, ratio, sg, nfl = m.tform_delayed_slice(UR, UL, T, X[ell - 1], np.zeros(m.N), 1, 1,
                                                             replay=forced)
    Xc, Wc = X.copy(), W0
    for i in range(m.N):
        Xf = Xc.copy()
        Xf[ell - 1, i] *= -1
        Wf = bf.weight(m.E, m.c, Xf, P, P)
        assert abs(ratio[i] - Wf / Wc) < 1e-10 * max(1, abs(Wf / Wc))
        if forced[i]:
            Xc, Wc = Xf, Wf
    np.testing.assert_array_equal(xl, Xc[ell - 1])
    assert sg == np.sign(Wc / W0)
    for s in range(2):
        np.testing.assert_allclose(Tn[s], np.linalg.inv(UL[s] @ URn[s]), atol=1e-10)
        np.testing.assert_allclose(np.eye(m.N) - URn[s] @ Tn[s] @ UL[s], bf.green(m.E, m.c[s], Xc, P, ell),
                                   atol=1e-11)


@pytest.mark.parametrize("k,strategy", [(1, 1), (5, 1), (16, 1), (3, 2), (8, 2)])
def test_tform_delayed_equals_gform(k, strategy):
    """The paper's T-form delayed update and the G-form oracle, driven by the same uniforms over a
    forward and part of a backward sweep with FP64 recomputes: identical decisions, fields and sign,
    ratios to 1e-12, G = 1 - U_R T U_L to 1e-11, and T = (U_L U_R)^{-1} after every slice."""
    Lx, Ly, ns, M, stab = 4, 4, 7, 6, 3
    m, P, X = _setup(Lx, Ly, ns, M, dtau=0.05)
    w = oracle.Walker(m, P, P, X)
    tw = oracle.TWalker(m, P, P, X, stab=stab)
    order = [(ell, +1) for ell in range(1, M + 1)] + [(ell, -1) for ell in range(M, M - 3, -1)]
    for visit, (ell, d) in enumerate(order):
        u = inputs.uniforms(7, 0, visit, 2 * m.N)
        d1, r1, _ = w.sweep_slice(ell, d, "delayed", u, k=k, strategy=strategy)
        d2, r2, _ = tw.sweep_slice(ell, d, "delayed", u, k=k, strategy=strategy)
        np.testing.assert_array_equal(d1, d2)
        np.testing.assert_allclose(r2, r1, rtol=1e-12, atol=1e-14)
        np.testing.assert_array_equal(tw.x, w.x)
        assert tw.sign == w.sign
        for s in range(2):
            np.testing.assert_allclose(tw.G(s), w.G[s], atol=1e-11)
            np.testing.assert_allclose(tw.T[s], np.linalg.inv(tw.UL[s] @ tw.UR[s]), atol=1e-10)
        if w.pos % stab == 0:
            w.recompute(stab)
            tw.recompute(stab)


@pytest.mark.parametrize("nb", [1, 4, 7, 16])
def test_tform_blockfb_equals_gform(nb):
    """The T-form block force bias (Eqs. BlkFrcBsTnew1, DetRatio10, BlkFrcBsTnew2) and the G-form oracle
    on the same uniforms: the same stripped-bias proposal probabilities, proposals, decisions and
    ratios, G = 1 - U_R T U_L to 1e-11 and T = (U_L U_R)^{-1} after every slice, over a forward and
    part of a backward sweep with recomputes; nb = 7 leaves a ragged last block."""
    Lx, Ly, ns, M, stab = 4, 4, 7, 6, 3
    m, P, X = _setup(Lx, Ly, ns, M, dtau=0.05)
    w = oracle.Walker(m, P, P, X)
    tw = oracle.TWalker(m, P, P, X, stab=stab)
    order = [(ell, +1) for ell in range(1, M + 1)] + [(ell, -1) for ell in range(M, M - 3, -1)]
    for visit, (ell, d) in enumerate(order):
        u = inputs.uniforms(11, 0, visit, 2 * m.N)
        d1, r1, e1 = w.sweep_slice(ell, d, "blockfb", u, nb=nb)
        d2, r2, e2 = tw.sweep_slice(ell, d, "blockfb", u, nb=nb)
        np.testing.assert_allclose(e2["lam_plus"], e1["lam_plus"], rtol=1e-12, atol=1e-14)
        np.testing.assert_array_equal(e2["xprop"], e1["xprop"])
        np.testing.assert_array_equal(d1, d2)
        np.testing.assert_allclose(r2, r1, rtol=1e-12, atol=1e-14)
        np.testing.assert_array_equal(tw.x, w.x)
        assert tw.sign == w.sign
        for s in range(2):
            np.testing.assert_allclose(tw.G(s), w.G[s], atol=1e-11)
            np.testing.assert_allclose(tw.T[s], np.linalg.inv(tw.UL[s] @ tw.UR[s]), atol=1e-10)
        if w.pos % stab == 0:
            w.recompute(stab)
            tw.recompute(stab)


# ---------------------------------------------------------------- momentum-space wrap (§8(f) F2)

@pytest.mark.parametrize("Lx,Ly", [(4, 4), (6, 4), (5, 3)])
def test_fft_wrap_equals_dense_wrap(Lx, Ly):
    """The wrap with exp(-+dtau K) applied through the 2D lattice DFT equals the dense-matrix wrap
    in both directions and both spins, and moves the from-scratch G to the next slice."""
    m, P, X = _setup(Lx, Ly, 3, 4, dtau=0.08)
    ell = 1
    for s in range(2):
        G = bf.green(m.E, m.c[s], X, P, ell)
        for d, xl in ((+1, X[ell]), (-1, X[ell - 1])):
            np.testing.assert_allclose(m.wrap_fft(G, xl, s, d), m.wrap(G, xl, s, d), atol=1e-12)
        np.testing.assert_allclose(m.wrap_fft(G, X[ell], s, +1), bf.green(m.E, m.c[s], X, P, ell + 1), atol=1e-11)


@pytest.mark.parametrize("k", [4, 5, 16])
def test_tform_window_update_is_block_update_of_its_accepts(k):
    """A delayed window's accumulated change of T and U_R (Eqs. DelayRgenk, FinalDelay) equals one
    rank-n_F block update over the window's accepted sites (Eq. BlkFrcBsTnew2 with F = the accepts):
    the T-form block force-bias pass, forced to propose exactly the final fields window by window and
    to accept every block, reproduces the delayed pass's T and U_R.  This is the window flush of a
    T-form GPU path."""
    Lx, Ly, ns, M = 4, 4, 7, 4
    m, P, X = _setup(Lx, Ly, ns, M, dtau=0.05)
    tw = oracle.TWalker(m, P, P, X)
    ell = 1
    for s in range(2):
        tw.UR[s], tw.UL[s] = m.tform_wrap(tw.UR[s], tw.UL[s], X[ell - 1], s, +1)
    u = inputs.uniforms(5, 0, 0, 2 * m.N)
    UR1, T1, x1, dec, ratio, sg, nfl = m.tform_delayed_slice(tw.UR, tw.UL, tw.T, X[ell - 1], u[:m.N], k, 1)
    nblocks = (m.N + k - 1) // k
    rep = np.zeros(m.N + nblocks, np.uint8)
    rep[:m.N] = x1 > 0  # propose the delayed pass's final fields
    rep[m.N:] = 1       # accept every block
    UR2, T2, x2, xprop, lamp, bdec, bratio, bsg = m.tform_blockfb_slice(tw.UR, tw.UL, tw.T, X[ell - 1], u[:m.N],
                                                                       np.zeros(nblocks), k, replay=rep)
    np.testing.assert_array_equal(x2, x1)
    assert dec.sum() > 0 and sg == bsg
    for s in range(2):
        np.testing.assert_allclose(T2[s], T1[s], atol=1e-12)
        np.testing.assert_allclose(UR2[s], UR1[s], atol=1e-12)
    # the product of a window's accepted local ratios is its block ratio (without the proposal factor)
    for b in range(nblocks):
        sl = slice(b * k, min(m.N, (b + 1) * k))
        acc = dec[sl] == 1
        if acc.any():
            lam_x = np.where(X[ell - 1, sl] > 0, lamp[sl], 1 - lamp[sl])[acc]
            lam_xp = np.where(x1[sl] > 0, lamp[sl], 1 - lamp[sl])[acc]
            assert bratio[b] == pytest.approx(np.prod(ratio[sl][acc]) * np.prod(lam_x / lam_xp), rel=1e-10)


def test_full_force_bias_rejection_is_linear_in_dtau():
    """The full force-bias update (n_b = N) accepts with probability 1 - O(dtau U f_x) (Eqs.
    RatioApprox, AcceptRatio): over seeded 4 x 4 chains the mean rejection probability
    1 - <min(1, |R|)> falls linearly with dtau (log-log slope near 1) and stays below 0.1 at
    dtau = 0.08.  A force bias of the wrong sign or size breaks this scaling."""
    L, ns, U, M = 4, 7, 4.0, 8
    N = L * L
    dtaus = (0.01, 0.02, 0.04, 0.08)
    rej = []
    for dtau in dtaus:
        probs = []
        for seed in range(1, 7):
            m = _model(L, L, U=U, M=M, dtau=dtau)
            P = inputs.trial_state(L, L, ns)
            X = inputs.initial_fields(M, N, seed=seed)
            w = oracle.Walker(m, P, P, X)
            for visit, ell in enumerate(range(1, M + 1)):
                u = inputs.uniforms(seed, 0, visit, 2 * N)
                dec, ratio, _ = w.sweep_slice(ell, +1, "blockfb", u, nb=N)
                probs.append(min(1.0, abs(ratio[0])))
                if w.pos % 4 == 0:
                    w.recompute(4)
        rej.append(1.0 - np.mean(probs))
    slope = np.polyfit(np.log(dtaus), np.log(rej), 1)[0]
    assert 0.8 < slope < 1.2, (rej, slope)
    assert rej[-1] < 0.1


def test_block_force_bias_rejection_set_by_block_size_not_lattice():
    """The block force bias's rejection grows with the block size n_b and, at fixed n_b, hardly
    depends on the lattice size (Sec. III.B): seeded chains at 6 x 6 and 8 x 8 (filling ~0.44,
    U = 4, dtau = 0.1)."""
    U, M, dtau = 4.0, 4, 0.1
    rej = {}
    for L, ns in ((6, 16), (8, 28)):
        N = L * L
        for nb in (2, 4, 8):
            probs = []
            for seed in (1, 2, 3):
                m = _model(L, L, U=U, M=M, dtau=dtau)
                P = inputs.trial_state(L, L, ns)
                X = inputs.initial_fields(M, N, seed=seed)
                w = oracle.Walker(m, P, P, X)
                for visit, ell in enumerate(range(1, M + 1)):
                    u = inputs.uniforms(seed, 0, visit, 2 * N)
                    _, ratio, _ = w.sweep_slice(ell, +1, "blockfb", u, nb=nb)
                    probs.extend(np.minimum(1.0, np.abs(ratio)))
            rej[(L, nb)] = 1.0 - np.mean(probs)
    for L in (6, 8):
        assert rej[(L, 2)] < rej[(L, 4)] < rej[(L, 8)], rej
    for nb in (2, 4, 8):
        assert 0.7 < rej[(8, nb)] / rej[(6, nb)] < 1.4, rej
