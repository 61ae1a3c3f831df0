"""Pins of the spin-orbit-coupled oracle (Appendix A) against what the paper and the mathematics fix.

Independent references: the real-space bond-by-bond H0 of the input module, scipy's expm of the
HS exponent matrix (Eq. BIOpForSy) and of H0, plain numpy products and dets of the walker overlap,
and Fock-space brute force.  Nothing here uses the CUDA library.
"""
import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_2506_09611_gb300 import inputs
from tests import bruteforce as bf


def _model(L=3, U=-4.0, dtau=0.1, M=6, lam=0.5, t=1.0):
    return oracle.SocModel(L, t, lam, U, dtau, M)


def _setup(L=3, n_e=8, M=6, seed=7, U=-4.0, dtau=0.1, lam=0.5):
    m = _model(L, U, dtau, M, lam)
    P = inputs.soc_trial_state(L, n_e, lam=lam)
    X = inputs.initial_fields(M, L * L, seed=seed)
    return m, P, X


@pytest.mark.parametrize("L", [3, 4, 6])
def test_H0_matches_real_space_bonds(L):
    m = _model(L)
    H = inputs.soc_hamiltonian(L, 1.0, 0.5)
    assert np.abs(m.H0 - H).max() < 1e-12


def test_H0_spectrum_is_split_dispersion():
    L = 6
    m = _model(L)
    k = 2 * np.pi * np.arange(L) / L
    kx, ky = np.meshgrid(k, k)
    eps = -2 * (np.cos(kx) + np.cos(ky))
    Lk = 2 * 0.5 * np.abs(np.sin(ky) - 1j * np.sin(kx))
    expect = np.sort(np.concatenate([(eps - Lk).ravel(), (eps + Lk).ravel()]))
    assert np.allclose(np.linalg.eigvalsh(m.H0), expect, atol=1e-12)


@pytest.mark.parametrize("L", [3, 4])
def test_expH_matches_expm(L):
    m = _model(L)
    H = inputs.soc_hamiltonian(L, 1.0, 0.5)
    assert np.abs(m.E - scipy.linalg.expm(-m.p.dtau * H)).max() < 1e-13
    assert np.abs(m.E @ m.Einv - np.eye(2 * L * L)).max() < 1e-13


@pytest.mark.parametrize("U", [-1.0, -4.0, -6.0])
def test_hs_spin_y_identity_on_one_site(U):
    """exp(-dtau U (n_u n_d - (n_u + n_d)/2)) = 1/2 sum_x exp(gamma x (c+_u c_d - c+_d c_u)) (Eq. HSspinSyDep)."""
    m = _model(2, U=U, dtau=0.05)
    cu, cd = bf.fock_ops(2)
    nu, nd = cu.T @ cu, cd.T @ cd
    lhs = scipy.linalg.expm(-0.05 * U * (nu @ nd - 0.5 * (nu + nd)))
    O = cu.T @ cd - cd.T @ cu
    rhs = 0.5 * sum(scipy.linalg.expm(m.gamma * x * O) for x in (+1, -1))
    assert np.abs(lhs - rhs).max() < 1e-13


def test_one_body_rotation_convention():
    """exp(gamma x O), O = c+_u c_d - c+_d c_u, maps c+_a|0> to sum_b A(x)_{ba} c+_b|0>: the one-body
    matrix of the spin-y field is A(x) = [[cos, sin], [-sin, cos]] (Eq. A2times2).  The brute-force
    propagator of these tests exponentiates that exponent matrix, so this pins its convention; the
    oracle's own rotation is then pinned by the from-scratch G below."""
    m = _model(2)
    cu, cd = bf.fock_ops(2)
    O = cu.T @ cd - cd.T @ cu
    vac = np.zeros(4)
    vac[0] = 1
    for x in (+1, -1):
        U = scipy.linalg.expm(m.gamma * x * O)
        A = np.zeros((2, 2))
        for a, ca in enumerate((cu, cd)):
            v = U @ (ca.T @ vac)
            A[0, a] = (cu.T @ vac) @ v
            A[1, a] = (cd.T @ vac) @ v
        g = m.gamma * x
        assert np.abs(A - np.array([[np.cos(g), np.sin(g)], [-np.sin(g), np.cos(g)]])).max() < 1e-14
        H = bf.soc_HI(m.gamma, np.array([x, 0, 0, 0]))
        assert np.abs(scipy.linalg.expm(H)[np.ix_([0, 4], [0, 4])] - A).max() < 1e-14


@pytest.mark.parametrize("ell", [0, 2, 5, 6])
def test_green_scratch_matches_plain_products(ell):
    m, P, X = _setup()
    G, la, ph = m.green_scratch(X, P, ell, stab=2)
    Gb = bf.soc_green(m.E, m.gamma, X, P, ell)
    assert np.linalg.norm(G - Gb) / np.linalg.norm(Gb) < 1e-11
    w = bf.soc_overlap(m.E, m.gamma, X, P)
    assert abs(la - np.log(abs(w))) < 1e-10
    assert abs(ph - w / abs(w)) < 1e-10


def test_projector_invariants_and_sign_free_weight():
    m, P, X = _setup(L=4, n_e=12, M=8)
    for ell in (0, 3, 8):
        G, _, ph = m.green_scratch(X, P, ell, stab=3)
        A = np.eye(G.shape[0]) - G
        assert np.abs(A @ A - A).max() < 1e-10
        assert abs(np.trace(A) - 12) < 1e-10
        # time-reversal-invariant trial state and real spin-y rotations: the weight is real positive
        assert abs(ph - 1) < 1e-10


def test_wrap_matches_scratch():
    m, P, X = _setup()
    for ell in (1, 3):
        G0, _, _ = m.green_scratch(X, P, ell - 1)
        G1, _, _ = m.green_scratch(X, P, ell)
        assert np.linalg.norm(m.wrap(G0, X[ell - 1], +1) - G1) / np.linalg.norm(G1) < 1e-11
        assert np.linalg.norm(m.wrap(G1, X[ell - 1], -1) - G0) / np.linalg.norm(G0) < 1e-11


def test_local_ratio_is_bruteforce_weight_ratio():
    """Every ratio of a free-running local slice equals W(X')/W(X) of the plain overlap, and the
    updated G equals the from-scratch G (Eqs. DetRatioSOC, LocalSOC)."""
    m, P, X = _setup()
    ell = 3
    G, _, _ = m.green_scratch(X, P, ell)
    u = inputs.uniforms(11, 0, 0, m.N) * 0.5 + 0.5  # in [0.5, 1): some ratios below and some above
    Gn, xn, dec, ratio = m.local_slice(G, X[ell - 1], u)
    # replay the decisions one site at a time against the brute-force weights
    Xc = X.copy()
    for i in range(m.N):
        w0 = bf.soc_overlap(m.E, m.gamma, Xc, P)
        Xf = Xc.copy()
        Xf[ell - 1, i] = -Xf[ell - 1, i]
        w1 = bf.soc_overlap(m.E, m.gamma, Xf, P)
        assert abs(ratio[i] - w1 / w0) < 1e-9 * max(1.0, abs(w1 / w0))
        assert abs(ratio[i].imag) < 1e-9 and ratio[i].real > 0
        if dec[i]:
            Xc = Xf
        assert bool(dec[i]) == (u[i] < abs(ratio[i]))
    assert np.array_equal(Xc[ell - 1], xn)
    Gs = bf.soc_green(m.E, m.gamma, Xc, P, ell)
    assert np.linalg.norm(Gn - Gs) / np.linalg.norm(Gs) < 1e-10
    assert dec.sum() > 0 and dec.sum() < m.N


@pytest.mark.parametrize("k", [1, 2, 4, 5, 9])
def test_delayed_equals_local(k):
    m, P, X = _setup(L=4, n_e=12)
    G, _, _ = m.green_scratch(X, P, 2)
    u = inputs.uniforms(3, 0, 1, m.N)
    Gl, xl, dl, rl = m.local_slice(G, X[1], u)
    Gd, xd, dd, rd = m.delayed_slice(G, X[1], u, k)
    assert np.array_equal(dl, dd) and np.array_equal(xl, xd)
    assert np.abs(rl - rd).max() < 1e-10
    assert np.linalg.norm(Gl - Gd) / np.linalg.norm(Gl) < 1e-11


def test_replay_forces_decisions():
    m, P, X = _setup()
    G, _, _ = m.green_scratch(X, P, 1)
    rep = (np.arange(m.N) % 3 == 0).astype(np.uint8)
    Gn, xn, dec, _ = m.local_slice(G, X[0], np.ones(m.N), replay=rep)
    assert np.array_equal(dec, rep)
    Xc = X.copy()
    Xc[0] = np.where(rep == 1, -X[0], X[0])
    assert np.array_equal(xn, Xc[0])
    Gs = bf.soc_green(m.E, m.gamma, Xc, P, 1)
    assert np.linalg.norm(Gn - Gs) / np.linalg.norm(Gs) < 1e-10
    Gd, xd, dd, _ = m.delayed_slice(G, X[0], np.ones(m.N), 4, replay=rep)
    assert np.array_equal(dd, rep) and np.linalg.norm(Gd - Gs) / np.linalg.norm(Gs) < 1e-10


def test_block_force_bias_is_finite_difference_of_stripped_overlap():
    """obar_i = d/de log <psi_l| e^{e O_i} |psi_r~> at e = 0, with |psi_r~> the right state whose block
    fields are taken out (x = 0 on the block: A(0) = 1) and O_i = c+_{i,up} c_{i,dn} - c+_{i,dn} c_{i,up};
    this fixes the index order of the spin-flip expectation."""
    m, P, X = _setup()
    ell, s0, n = 3, 2, 4
    G, _, _ = m.green_scratch(X, P, ell)
    ob = m.block_force_bias(G, X[ell - 1], s0, n)
    Xs = X.astype(np.float64).copy()
    Xs[ell - 1, s0:s0 + n] = 0.0
    R, Lm = bf.soc_products(m.E, m.gamma, Xs, P, ell)
    N = m.N
    for a in range(n):
        i = s0 + a
        O = np.zeros((2 * N, 2 * N))
        O[i, N + i] = 1.0
        O[N + i, i] = -1.0
        h = 1e-5
        lp = np.log(np.linalg.det(Lm @ scipy.linalg.expm(h * O) @ R))
        lm = np.log(np.linalg.det(Lm @ scipy.linalg.expm(-h * O) @ R))
        fd = (lp - lm) / (2 * h)
        assert abs(ob[a] - fd) < 1e-7


def test_blockfb_ratio_and_update_bruteforce():
    m, P, X = _setup()
    ell, nb = 2, 4
    G, _, _ = m.green_scratch(X, P, ell)
    nblocks = (m.N + nb - 1) // nb
    up = inputs.uniforms(5, 0, 0, m.N)
    ua = np.zeros(nblocks)  # accept every block whose ratio is not zero
    Gn, xn, xprop, lamp, dec, ratio = m.blockfb_slice(G, X[ell - 1], up, ua, nb)
    Xc = X.copy()
    for b in range(nblocks):
        s0, n = b * nb, min(nb, m.N - b * nb)
        xl = Xc[ell - 1].copy()
        Gc = bf.soc_green(m.E, m.gamma, Xc, P, ell)
        ob = m.block_force_bias(Gc, xl, s0, n)
        h = m.gamma * ob.real
        assert np.allclose(lamp[s0:s0 + n], 1 / (1 + np.exp(-2 * h)), atol=1e-12)
        xp = np.where(up[s0:s0 + n] < lamp[s0:s0 + n], 1, -1)
        assert np.array_equal(xprop[s0:s0 + n], xp)
        Xf = Xc.copy()
        Xf[ell - 1, s0:s0 + n] = xp
        flipped = xp != xl[s0:s0 + n]
        q = np.exp(np.sum((xl[s0:s0 + n] - xp)[flipped] * h[flipped]))
        expect = bf.soc_overlap(m.E, m.gamma, Xf, P) / bf.soc_overlap(m.E, m.gamma, Xc, P) * q
        assert abs(ratio[b] - expect) < 1e-9 * max(1.0, abs(expect))
        assert dec[b] == 1
        Xc = Xf
    assert np.array_equal(Xc[ell - 1], xn)
    Gs = bf.soc_green(m.E, m.gamma, Xc, P, ell)
    assert np.linalg.norm(Gn - Gs) / np.linalg.norm(Gs) < 1e-10


def test_blockfb_exact_detailed_balance():
    """On a 2 x 2 lattice with one slice the chain of a single block covering all sites can be
    enumerated: the transition matrix T(X -> X') = q(X'|X) min(1, |R|) satisfies W(X) T(X->X') = W(X') T(X'->X)."""
    L, M = 2, 1
    m = _model(L, M=M, U=-4.0, dtau=0.2, lam=0.5)
    N = m.N
    P = inputs.soc_trial_state(L, 4)
    confs = [np.array([[1 if (c >> i) & 1 else -1 for i in range(N)]], np.int8) for c in range(1 << N)]
    W = np.array([bf.soc_overlap(m.E, m.gamma, x, P).real for x in confs])
    assert np.all(W > 0)
    T = np.zeros((len(confs), len(confs)))
    for a, x in enumerate(confs):
        G, _, _ = m.green_scratch(x, P, 1)
        for b, xp in enumerate(confs):
            rep = np.zeros(2 * N, np.uint8)
            rep[:N] = (xp[0] > 0)
            rep[N] = 1
            _, _, _, lamp, dec, ratio = m.blockfb_slice(G, x[0], np.zeros(N), np.zeros(1), N, replay=rep)
            qprop = np.prod(np.where(xp[0] > 0, lamp, 1 - lamp))
            T[a, b] = qprop * min(1.0, abs(ratio[0]))
    F = W[:, None] * T
    offdiag = ~np.eye(len(confs), dtype=bool)
    assert np.abs(F - F.T)[offdiag].max() < 1e-12 * W.max()


def test_energy_free_fermion_closed_form():
    """U = 0: gamma = 0, G = 1 - P P^+ and E = sum of the lowest N_e levels of H0."""
    for L, n_e in ((4, 12), (6, 36)):
        m = _model(L, U=0.0)
        P = inputs.soc_trial_state(L, n_e)
        X = inputs.initial_fields(m.M, m.N)
        G, _, _ = m.green_scratch(X, P, 3)
        w = np.linalg.eigvalsh(inputs.soc_hamiltonian(L))
        # the 1e-6 perturbation of the trial state mixes in other levels at O(1e-5): an energy
        # error of second order, O(1e-10)
        assert abs(m.energy(G) - w[:n_e].sum()) < 1e-8


@pytest.mark.parametrize("U", [0.0, -3.0])
def test_energy_matches_fock_space(U):
    """The spin-coupled Wick contraction equals the Fock-space mixed expectation for a random
    spin-mixing H0 and random complex Slater determinants on 2 x 2 sites (8 orbitals)."""
    m = _model(2, U=U)
    rng = np.random.default_rng(3)
    H0 = rng.standard_normal((8, 8)) + 1j * rng.standard_normal((8, 8))
    H0 = 0.5 * (H0 + H0.conj().T)
    R = rng.standard_normal((8, 3)) + 1j * rng.standard_normal((8, 3))
    Lm = rng.standard_normal((3, 8)) + 1j * rng.standard_normal((3, 8))
    G = np.eye(8) - R @ np.linalg.solve(Lm @ R, Lm)
    assert abs(m.energy(G, H0) - bf.soc_fock_energy(H0, U, R, Lm)) < 1e-10


def test_free_running_sweep_tracks_scratch():
    """A few slice-steps of the walker in all three modes keep G equal to the from-scratch G."""
    m, P, X = _setup(L=3, n_e=8, M=4)
    for mode in ("local", "delayed", "blockfb"):
        w = oracle.SocWalker(m, P, X)
        for ell in (1, 2, 3):
            u = inputs.uniforms(9, 0, ell, 2 * m.N)
            w.sweep_slice(ell, +1, mode, u, k=4, nb=3)
        Gs = bf.soc_green(m.E, m.gamma, w.x, P, w.pos)
        assert np.linalg.norm(w.G - Gs) / np.linalg.norm(Gs) < 1e-10


def test_full_force_bias_rejection_is_linear_in_dtau():
    """The full spin-flip force bias (n_b = N, Appendix A with Eqs. RatioApprox, AcceptRatio): over
    seeded 4 x 4 chains at half filling the mean rejection probability 1 - <min(1, |R|)> falls
    linearly with dtau for small dtau (log-log slope near 1).  A Metropolis ratio without the
    proposal factor breaks this scaling.  The spin-flip bias itself is weak on this workload
    (P(x' = +1) within 0.42-0.54), so its index order is pinned by the finite-difference test,
    not by this one."""
    L, ne, M = 4, 16, 8
    N = L * L
    dtaus = (0.01, 0.02, 0.04)
    rej = []
    for dtau in dtaus:
        probs = []
        for seed in range(1, 5):
            m = oracle.SocModel(L, 1.0, 0.5, -4.0, dtau, M)
            w = oracle.SocWalker(m, inputs.soc_trial_state(L, ne), inputs.initial_fields(M, N, seed=seed))
            for visit, ell in enumerate(range(1, M + 1)):
                _, ratio, _ = w.sweep_slice(ell, +1, "blockfb", inputs.uniforms(seed, 0, visit, 2 * N), nb=N)
                probs.append(min(1.0, abs(ratio[0])))
                if w.pos % 4 == 0:
                    w.recompute(4)
        rej.append(1.0 - np.mean(probs))
    slope = np.polyfit(np.log(dtaus), np.log(rej), 1)[0]
    assert 0.75 < slope < 1.25, (rej, slope)


@pytest.mark.parametrize("nb", [1, 4, 9])
def test_block_proposals_equal_to_the_current_fields_are_accepted_unchanged(nb):
    """A block whose proposal repeats its current fields is the null move: Delta_F is empty, so
    R = 1 and u < min(1, |R|) holds for every u in [0, 1).  It is accepted, with ratio 1, and G and
    the fields stay exactly as they were."""
    m, P, X = _setup()
    N, ell = m.N, 2
    G, _, _ = m.green_scratch(X, P, ell)
    xl = X[ell - 1]
    top = 1.0 - 2.0 ** -53  # the largest uniform below 1
    u_prop = np.where(xl > 0, 0.0, top)  # x' = +1 iff u_prop < lambda(+1), which lies strictly inside (0, 1)
    nblk = (N + nb - 1) // nb
    G1, x1, xprop, lamp, dec, ratio = m.blockfb_slice(G, xl, u_prop, np.full(nblk, top), nb)
    assert np.all((lamp > 0) & (lamp < top))
    np.testing.assert_array_equal(xprop, xl)
    assert dec.all()
    np.testing.assert_array_equal(ratio, np.ones(nblk))
    np.testing.assert_array_equal(x1, xl)
    np.testing.assert_array_equal(G1, G)


@pytest.mark.parametrize("L", [3, 4, 6])
@pytest.mark.parametrize("direction", [+1, -1])
def test_momentum_space_wrap_equals_the_dense_wrap(L, direction):
    """SocModel.wrap_fft (exp(-dtau h_k) per momentum on FFT'd columns; the paper's FFT
    propagation) equals the dense wrap with the real-space exp(-dtau H0), for the from-scratch G
    and for an arbitrary complex matrix, forward and backward; and moves G(l-1) to G(l)."""
    m, P, X = _setup(L=L, n_e=2 * (L * L // 2), M=4)
    rng = np.random.default_rng(L)
    ell = 2
    G, _, _ = m.green_scratch(X, P, ell - 1 if direction > 0 else ell)
    Z = rng.standard_normal(G.shape) + 1j * rng.standard_normal(G.shape)
    for A in (G, Z):
        ref = m.wrap(A, X[ell - 1], direction)
        got = m.wrap_fft(A, X[ell - 1], direction)
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
    G1, _, _ = m.green_scratch(X, P, ell if direction > 0 else ell - 1)
    np.testing.assert_allclose(m.wrap_fft(G, X[ell - 1], direction), G1, atol=1e-10)
