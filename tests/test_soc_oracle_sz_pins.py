"""Pins of the oracle's imaginary spin-z decoupling (Sec. II.B, Eqs. HSspinDecomp, BIOpForHubbard) in
the spin-coupled oracle (soc_oracle.c with hs = 1): the paper's own decoupling of the attractive
Hubbard model, where the field acts on the pair (i, N + i) as diag(e^{i gamma x}, e^{-i gamma x}).

Independent references: scipy's expm of the Fock-space exponent, plain numpy products and dets of
the walker overlap (tests/bruteforce.py with the spin-z exponent matrix), finite differences of the
stripped overlap, and an exact enumeration of every field configuration of a 2 x 2 lattice against
the Fock-space projection.  Nothing here uses the CUDA library.
"""
import itertools

import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_2506_09611_gb300 import inputs
from tests import bruteforce as bf


def _model(L=3, U=-4.0, dtau=0.1, M=6, lam=0.0, t=1.0):
    return oracle.SocModel(L, t, lam, U, dtau, M, hs="sz")


def _setup(L=3, ns=4, M=6, seed=7, U=-4.0, dtau=0.1, lam=0.0):
    m = _model(L, U, dtau, M, lam)
    P = inputs.sz_trial_state(L, ns) if lam == 0.0 else inputs.soc_trial_state(L, 2 * ns, lam=lam)
    X = inputs.initial_fields(M, L * L, seed=seed)
    return m, P, X


@pytest.mark.parametrize("U", [-1.0, -4.0, -6.0])
def test_hs_spin_z_identity_on_one_site(U):
    """exp(-dtau U (n_u n_d - (n_u + n_d)/2)) = 1/2 sum_x exp(i gamma x (n_u - n_d)) with
    gamma = arccos(exp(dtau U / 2)) (Eq. HSspinDecomp), as operators on the 4-state Fock space."""
    m = _model(2, U=U, dtau=0.05)
    assert m.gamma == pytest.approx(np.arccos(np.exp(0.05 * U / 2)), abs=1e-15)
    cu, cd = bf.fock_ops(2)
    nu, nd = cu.T @ cu, cd.T @ cd
    lhs = scipy.linalg.expm(-0.05 * U * (nu @ nd - 0.5 * (nu + nd)))
    rhs = 0.5 * sum(scipy.linalg.expm(1j * m.gamma * x * (nu - nd)) for x in (+1, -1))
    assert np.abs(lhs - rhs).max() < 1e-13


def test_one_body_phase_convention():
    """exp(i gamma x (n_u - n_d)) maps c+_a|0> to sum_b A_{ba} c+_b|0> with
    A = diag(e^{i gamma x}, e^{-i gamma x}); the brute-force exponent matrix has that exponential."""
    m = _model(2)
    cu, cd = bf.fock_ops(2)
    nu, nd = cu.T @ cu, cd.T @ cd
    vac = np.zeros(4)
    vac[0] = 1
    for x in (+1, -1):
        U = scipy.linalg.expm(1j * m.gamma * x * (nu - nd))
        A = np.zeros((2, 2), np.complex128)
        for a, ca in enumerate((cu, cd)):
            v = U @ (ca.T @ vac)
            A[0, a] = (cu.T @ vac) @ v
            A[1, a] = (cd.T @ vac) @ v
        g = m.gamma * x
        assert np.abs(A - np.diag([np.exp(1j * g), np.exp(-1j * g)])).max() < 1e-14
        H = bf.soc_HI(m.gamma, np.array([x, 0, 0, 0]), "sz")
        assert np.abs(scipy.linalg.expm(H)[np.ix_([0, 4], [0, 4])] - A).max() < 1e-14


@pytest.mark.parametrize("lam", [0.0, 0.5])
@pytest.mark.parametrize("ell", [0, 2, 5, 6])
def test_green_scratch_matches_plain_products(ell, lam):
    m, P, X = _setup(lam=lam)
    G, la, ph = m.green_scratch(X, P, ell, stab=2)
    Gb = bf.soc_green(m.E, m.gamma, X, P, ell, "sz")
    assert np.linalg.norm(G - Gb) / np.linalg.norm(Gb) < 1e-11
    w = bf.soc_overlap(m.E, m.gamma, X, P, "sz")
    assert abs(la - np.log(abs(w))) < 1e-10
    assert abs(ph - w / abs(w)) < 1e-10


def test_spin_blocks_and_sign_free_weight():
    """lam = 0, P_dn = conj(P_up): B_dn = conj(B_up), so G has no spin-mixing block, G_dn = conj(G_up),
    and the weight det(...) = |det_up|^2 is real and positive (Sec. II.B)."""
    m, P, X = _setup(L=4, ns=6, M=8)
    N = m.N
    for ell in (0, 3, 8):
        G, _, ph = m.green_scratch(X, P, ell, stab=3)
        assert np.abs(G[:N, N:]).max() < 1e-12 and np.abs(G[N:, :N]).max() < 1e-12
        assert np.abs(G[N:, N:] - G[:N, :N].conj()).max() < 1e-11
        assert np.abs(G[:N, :N].imag).max() > 1e-3  # genuinely complex
        assert abs(ph - 1) < 1e-10


def test_wrap_matches_scratch_and_the_momentum_space_wrap():
    m, P, X = _setup()
    for ell in (1, 3):
        G0, _, _ = m.green_scratch(X, P, ell - 1)
        G1, _, _ = m.green_scratch(X, P, ell)
        assert np.linalg.norm(m.wrap(G0, X[ell - 1], +1) - G1) / np.linalg.norm(G1) < 1e-11
        assert np.linalg.norm(m.wrap(G1, X[ell - 1], -1) - G0) / np.linalg.norm(G0) < 1e-11
        assert np.linalg.norm(m.wrap_fft(G0, X[ell - 1], +1) - G1) / np.linalg.norm(G1) < 1e-11


def test_local_ratio_is_bruteforce_weight_ratio():
    """Every ratio of a free-running local slice equals W(X')/W(X) of the plain overlap, real and
    positive (|r_up|^2), and the updated G equals the from-scratch G."""
    m, P, X = _setup()
    ell = 3
    G, _, _ = m.green_scratch(X, P, ell)
    u = inputs.uniforms(11, 0, 0, m.N) * 0.5 + 0.5
    Gn, xn, dec, ratio = m.local_slice(G, X[ell - 1], u)
    Xc = X.copy()
    for i in range(m.N):
        w0 = bf.soc_overlap(m.E, m.gamma, Xc, P, "sz")
        Xf = Xc.copy()
        Xf[ell - 1, i] = -Xf[ell - 1, i]
        w1 = bf.soc_overlap(m.E, m.gamma, Xf, P, "sz")
        assert abs(ratio[i] - w1 / w0) < 1e-9 * max(1.0, abs(w1 / w0))
        assert abs(ratio[i].imag) < 1e-9 and ratio[i].real > 0
        if dec[i]:
            Xc = Xf
        assert bool(dec[i]) == (u[i] < abs(ratio[i]))
    assert np.array_equal(Xc[ell - 1], xn)
    Gs = bf.soc_green(m.E, m.gamma, Xc, P, ell, "sz")
    assert np.linalg.norm(Gn - Gs) / np.linalg.norm(Gs) < 1e-10
    assert 0 < dec.sum() < m.N


@pytest.mark.parametrize("k", [1, 2, 4, 5, 9])
def test_delayed_equals_local(k):
    m, P, X = _setup(L=4, ns=6)
    G, _, _ = m.green_scratch(X, P, 2)
    u = inputs.uniforms(3, 0, 1, m.N)
    Gl, xl, dl, rl = m.local_slice(G, X[1], u)
    Gd, xd, dd, rd = m.delayed_slice(G, X[1], u, k)
    assert np.array_equal(dl, dd) and np.array_equal(xl, xd)
    assert np.abs(rl - rd).max() < 1e-10
    assert np.linalg.norm(Gl - Gd) / np.linalg.norm(Gl) < 1e-11


def test_block_force_bias_is_finite_difference_of_stripped_overlap():
    """obar_i = d/de log <psi_l| e^{e O_i} |psi_r~> at e = 0, with |psi_r~> the right state whose block
    fields are taken out and O_i = i (n_{i,up} - n_{i,dn}), the generator of the spin-z field; the
    bias exponent gamma Re(obar_i) is then -gamma Im(<n_up> - <n_dn>)."""
    m, P, X = _setup()
    ell, s0, n = 3, 2, 4
    G, _, _ = m.green_scratch(X, P, ell)
    ob = m.block_force_bias(G, X[ell - 1], s0, n)
    Xs = X.astype(np.float64).copy()
    Xs[ell - 1, s0:s0 + n] = 0.0
    R, Lm = bf.soc_products(m.E, m.gamma, Xs, P, ell, "sz")
    N = m.N
    for a in range(n):
        i = s0 + a
        O = np.zeros((2 * N, 2 * N), np.complex128)
        O[i, i] = 1j
        O[N + i, N + i] = -1j
        h = 1e-5
        lp = np.log(np.linalg.det(Lm @ scipy.linalg.expm(h * O) @ R))
        lm = np.log(np.linalg.det(Lm @ scipy.linalg.expm(-h * O) @ R))
        fd = (lp - lm) / (2 * h)
        assert abs(ob[a] - fd) < 1e-7
    assert np.abs(ob.real).max() > 1e-3  # a bias that is not trivially zero


def test_blockfb_ratio_and_update_bruteforce():
    m, P, X = _setup()
    ell, nb = 2, 4
    G, _, _ = m.green_scratch(X, P, ell)
    nblocks = (m.N + nb - 1) // nb
    up = inputs.uniforms(5, 0, 0, m.N)
    ua = np.zeros(nblocks)
    Gn, xn, xprop, lamp, dec, ratio = m.blockfb_slice(G, X[ell - 1], up, ua, nb)
    Xc = X.copy()
    for b in range(nblocks):
        s0, n = b * nb, min(nb, m.N - b * nb)
        xl = Xc[ell - 1].copy()
        Gc = bf.soc_green(m.E, m.gamma, Xc, P, ell, "sz")
        ob = m.block_force_bias(Gc, xl, s0, n)
        h = m.gamma * ob.real
        assert np.allclose(lamp[s0:s0 + n], 1 / (1 + np.exp(-2 * h)), atol=1e-12)
        xp = np.where(up[s0:s0 + n] < lamp[s0:s0 + n], 1, -1)
        assert np.array_equal(xprop[s0:s0 + n], xp)
        Xf = Xc.copy()
        Xf[ell - 1, s0:s0 + n] = xp
        flipped = xp != xl[s0:s0 + n]
        q = np.exp(np.sum((xl[s0:s0 + n] - xp)[flipped] * h[flipped]))
        expect = bf.soc_overlap(m.E, m.gamma, Xf, P, "sz") / bf.soc_overlap(m.E, m.gamma, Xc, P, "sz") * q
        assert abs(ratio[b] - expect) < 1e-9 * max(1.0, abs(expect))
        assert dec[b] == 1
        Xc = Xf
    assert np.array_equal(Xc[ell - 1], xn)
    Gs = bf.soc_green(m.E, m.gamma, Xc, P, ell, "sz")
    assert np.linalg.norm(Gn - Gs) / np.linalg.norm(Gs) < 1e-10


def test_blockfb_exact_detailed_balance():
    """2 x 2 lattice, one slice, one block over all sites: the enumerated transition matrix
    T(X -> X') = q(X'|X) min(1, |R|) satisfies W(X) T(X->X') = W(X') T(X'->X)."""
    L, M = 2, 1
    m = _model(L, M=M, U=-4.0, dtau=0.2)
    N = m.N
    P = inputs.sz_trial_state(L, 2)
    confs = [np.array([[1 if (c >> i) & 1 else -1 for i in range(N)]], np.int8) for c in range(1 << N)]
    W = np.array([bf.soc_overlap(m.E, m.gamma, x, P, "sz").real for x in confs])
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


def _fock_hubbard(L, t, U):
    """H = K + U sum_i (n_iu n_id - (n_iu + n_id)/2) on the Fock space of the 2N spin orbitals, and
    the one-body operator map M -> c+ M c."""
    N = L * L
    cs = bf.fock_ops(2 * N)
    cd = [C.T for C in cs]

    def one_body(Mat):
        out = np.zeros((1 << (2 * N), 1 << (2 * N)), np.complex128)
        for a in range(2 * N):
            for b in range(2 * N):
                if Mat[a, b] != 0:
                    out += Mat[a, b] * cd[a] @ cs[b]
        return out

    K = inputs.hopping_matrix(L, L, t)
    HI = np.zeros((1 << (2 * N), 1 << (2 * N)))
    for i in range(N):
        nu, nd = cd[i] @ cs[i], cd[N + i] @ cs[N + i]
        HI += U * (nu @ nd - 0.5 * (nu + nd))
    return one_body, one_body(np.kron(np.eye(2), K)), HI, cd


def test_enumerated_estimator_equals_the_fock_space_projection():
    """Every field configuration of a 2 x 2 lattice with M = 2 slices (2^8 of them), weighted by
    det(P^+ B_M ... B_1 P) / 2^{NM}, gives sum_X W E_X / sum_X W equal to the Fock-space
    <psi_T| T^{M - l} H T^l |psi_T> / <psi_T| T^M |psi_T>, T = e^{-dtau H_I} e^{-dtau K}: the spin-z
    decoupling is exact for every Trotter factor, so this pins gamma, the phase convention, the
    order of D and E in B_l and the mixed-estimator energy together (Eqs. HSspinDecomp, GSObsQMC)."""
    L, M, U, dtau, t, ns, ell = 2, 2, -4.0, 0.2, 1.0, 1, 1
    N = L * L
    m = _model(L, U=U, dtau=dtau, M=M)
    P = inputs.sz_trial_state(L, ns)
    num = den = 0.0
    for bits in itertools.product((1, -1), repeat=N * M):
        X = np.array(bits, np.int8).reshape(M, N)
        G, la, ph = m.green_scratch(X, P, ell, stab=0)
        w = ph * np.exp(la)
        num += w * m.energy(G)
        den += w
    est = num / den
    one_body, Kf, HI, cd = _fock_hubbard(L, t, U)
    Tm = scipy.linalg.expm(-dtau * HI) @ scipy.linalg.expm(-dtau * Kf)
    vac = np.zeros(1 << (2 * N), np.complex128)
    vac[0] = 1.0
    psi = vac
    for col in range(P.shape[1]):
        psi = sum(P[a, col] * cd[a] for a in range(2 * N)) @ psi
    H = Kf + HI
    right = np.linalg.matrix_power(Tm, ell) @ psi
    left = psi.conj() @ np.linalg.matrix_power(Tm, M - ell)
    exact = (left @ H @ right) / (left @ right)
    assert abs(est - exact) < 1e-10 * abs(exact)
    assert abs(np.imag(den)) < 1e-12 * abs(den)
