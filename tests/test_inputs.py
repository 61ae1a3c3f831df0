"""The seeded input module against the recipe it states: trial states are orthonormal bases of the
lowest single-particle levels (the ground state of the non-interacting part), the SOC perturbation
is time-reversal invariant, the twisted spin-z trial is a set of plane waves and a pseudospin singlet
at half filling, fields are +-1 with probability 1/2, uniforms have 53 random bits in [0, 1), and the
configured lattices get the particle numbers of their fillings."""
import numpy as np
import pytest

from paper_2506_09611_gb300 import inputs


def _shells(H, P, n):
    """(levels below the Fermi level, levels up to and including its shell, weight of P outside
    those levels, deviation of P's projector on the levels below it from the identity)."""
    w, V = np.linalg.eigh(H)
    ef, tol = w[n - 1], 1e-9
    below, upto = w < ef - tol, w <= ef + tol
    leak = np.linalg.norm(V[:, ~upto].conj().T @ P)
    Vb = V[:, below]
    cover = np.linalg.norm(Vb.conj().T @ P @ P.conj().T @ Vb - np.eye(below.sum()))
    return int(below.sum()), int(upto.sum()), leak, cover


@pytest.mark.parametrize("L,ns,closed,shell", [(4, 7, 5, 11), (6, 13, 9, 13), (16, 112, 109, 113), (40, 700, 693, 701)])
def test_trial_state_spans_the_lowest_levels(L, ns, closed, shell):
    """P is the ground state of the non-interacting part: every level below the Fermi level is in
    its span, and it has no weight beyond the Fermi shell, up to first order in the 1e-6 tie-break
    that picks the open shell's filled part (4 x 4 fills 5 levels + 2 of the 6 at zero energy;
    16 x 16: 109 + 3 of 4; 40 x 40: 693 + 7 of 8)."""
    P = inputs.trial_state(L, L, ns)
    assert P.shape == (L * L, ns)
    np.testing.assert_allclose(P.T @ P, np.eye(ns), atol=1e-12)
    b, u, leak, cover = _shells(inputs.hopping_matrix(L, L), P, ns)
    assert (b, u) == (closed, shell)
    assert leak < 1e-5 * np.sqrt(ns * L * L) and cover < 1e-6
    np.testing.assert_array_equal(P, inputs.trial_state(L, L, ns))  # seeded


def test_hopping_matrix_is_the_periodic_nearest_neighbour_lattice():
    K = inputs.hopping_matrix(5, 3, t=1.5)
    assert np.allclose(K, K.T)
    np.testing.assert_allclose(K.sum(axis=1), -4 * 1.5)  # four neighbours each
    assert K[0, 1] == -1.5 and K[0, 4] == -1.5 and K[0, 5] == -1.5 and K[0, 10] == -1.5 and K[0, 6] == 0


@pytest.mark.parametrize("L,ne,closed,shell", [(3, 8, 6, 10), (4, 16, 14, 18), (6, 36, 34, 38), (24, 576, 574, 578)])
def test_soc_trial_state_spans_the_lowest_levels_and_respects_time_reversal(L, ne, closed, shell):
    N = L * L
    H = inputs.soc_hamiltonian(L)
    assert np.allclose(H, H.conj().T)
    theta = np.block([[np.zeros((N, N)), -np.eye(N)], [np.eye(N), np.zeros((N, N))]])  # i sigma_y, then conj
    S = inputs.soc_trs_perturbation(N)
    np.testing.assert_allclose(theta @ S.conj() @ theta.T, S, atol=1e-12)
    np.testing.assert_allclose(theta @ H.conj() @ theta.T, H, atol=1e-12)
    P = inputs.soc_trial_state(L, ne)
    np.testing.assert_allclose(P.conj().T @ P, np.eye(ne), atol=1e-12)
    b, u, leak, cover = _shells(H, P, ne)
    assert (b, u) == (closed, shell)  # half filling at 24 x 24: 574 + 2 of 4
    assert leak < 1e-5 * np.sqrt(ne * 2 * N) and cover < 1e-6


def test_fields_are_fair_signs_and_differ_between_walkers():
    X = inputs.initial_fields(80, 1600, seed=1)
    assert X.dtype == np.int8 and set(np.unique(X)) == {-1, 1}
    p = (X > 0).mean()
    assert abs(p - 0.5) < 5 * np.sqrt(0.25 / X.size)
    np.testing.assert_array_equal(X, inputs.initial_fields(80, 1600, seed=1))
    assert (X != inputs.initial_fields(80, 1600, seed=1, walker=1)).mean() > 0.4
    assert (X != inputs.initial_fields(80, 1600, seed=2)).mean() > 0.4


def test_uniforms_have_53_bits_in_the_unit_interval():
    u = inputs.uniforms(3, 1, 7, 100000)
    assert u.min() >= 0.0 and u.max() < 1.0
    k = u * 2.0 ** 53
    np.testing.assert_array_equal(k, np.floor(k))  # multiples of 2^-53
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / u.size)
    hist = np.histogram(u, bins=10, range=(0, 1))[0]
    assert hist.min() > 9500 and hist.max() < 10500
    np.testing.assert_array_equal(u, inputs.uniforms(3, 1, 7, 100000))
    assert not np.array_equal(u[:100], inputs.uniforms(3, 1, 8, 100))  # the visit is part of the counter


def test_population_and_fillings():
    Ls = inputs.batch_lattices(256, seed=5)
    assert Ls.shape == (256,) and set(np.unique(Ls)) == {8, 12, 16, 24}
    np.testing.assert_array_equal(Ls, inputs.batch_lattices(256, seed=5))
    assert [inputs.n_sigma_for(L, 0.875) for L in (8, 12, 16, 24, 40)] == [28, 63, 112, 252, 700]
    assert inputs.n_sigma_for(4, 0.875) == 7


def _eta2_wick(P, L, ns):
    """<eta^2> of the product determinant P (2N x 2ns, blocks up/down) at half filling (eta_z = 0):
    <eta+ eta-> = sum_ij (-1)^{i+j} <c+_iup c_jup> <c+_idn c_jdn> by Wick's theorem."""
    N = L * L
    ru = P[:N, :ns].conj() @ P[:N, :ns].T  # <c+_i c_j> = sum_m conj(P_im) P_jm
    rd = P[N:, ns:].conj() @ P[N:, ns:].T
    s = np.array([(-1) ** (i % L + i // L) for i in range(N)])
    return float(np.real(np.sum(np.outer(s, s) * ru * rd)))


def test_twisted_hopping_is_the_flux_threaded_lattice():
    """K(0) is the plain hopping; with a flux its spectrum is the shifted dispersion
    -2t (cos(kx + theta_x/L) + cos(ky + theta_y/L)), Hermitian, with every level split."""
    np.testing.assert_allclose(inputs.twisted_hopping_matrix(5, (0.0, 0.0), 1.5), inputs.hopping_matrix(5, 5, 1.5))
    L, tw = 6, (0.1, 0.07)
    K = inputs.twisted_hopping_matrix(L, tw)
    assert np.allclose(K, K.conj().T)
    k = 2 * np.pi * np.arange(L) / L
    e = np.sort((-2 * (np.cos(k[:, None] + tw[0] / L) + np.cos(k[None, :] + tw[1] / L))).ravel())
    w = np.linalg.eigvalsh(K)
    np.testing.assert_allclose(w, e, atol=1e-12)
    assert np.min(np.diff(w)) > 1e-4


@pytest.mark.parametrize("L", [4, 6, 8])
def test_twisted_sz_trial_is_plane_waves_and_a_pseudospin_singlet(L):
    """The twisted trial (the pairing runs' default) fills the n_s plane waves of lowest twisted energy
    for spin up and the opposite momenta for spin down (P_dn = conj(P_up)); at half filling it has
    <eta^2> = 0, while the randomly tie-broken real trial does not."""
    N, ns = L * L, L * L // 2
    P = inputs.sz_trial_state(L, ns, twist=(0.1, 0.07))
    np.testing.assert_allclose(P.conj().T @ P, np.eye(2 * ns), atol=1e-12)
    np.testing.assert_allclose(P[N:, ns:], P[:N, :ns].conj(), atol=0)
    assert np.all(P[:N, ns:] == 0) and np.all(P[N:, :ns] == 0)
    # the up projector commutes with the lattice translations (a set of plane waves)
    Tx = np.zeros((N, N))
    for i in range(N):
        Tx[(i % L + 1) % L + L * (i // L), i] = 1.0
    Pr = P[:N, :ns] @ P[:N, :ns].conj().T
    np.testing.assert_allclose(Tx @ Pr, Pr @ Tx, atol=1e-10)
    assert abs(_eta2_wick(P, L, ns)) < 1e-10
    assert _eta2_wick(inputs.sz_trial_state(L, ns), L, ns) > 0.5


def test_eta2_wick_matches_the_fock_space_casimir():
    """The Wick form of <eta^2> used above against the Fock-space eta+ eta- on 2 x 2 (8 orbitals)
    for a random complex product determinant with two electrons per spin."""
    from tests import bruteforce as bf
    L, ns, N = 2, 2, 4
    rng = np.random.default_rng(5)
    Pu = np.linalg.qr(rng.standard_normal((N, ns)) + 1j * rng.standard_normal((N, ns)))[0]
    Pd = np.linalg.qr(rng.standard_normal((N, ns)) + 1j * rng.standard_normal((N, ns)))[0]
    P = np.zeros((2 * N, 2 * ns), np.complex128)
    P[:N, :ns], P[N:, ns:] = Pu, Pd
    cs = [C.astype(np.complex128) for C in bf.fock_ops(2 * N)]
    cd = [C.T for C in cs]
    psi = np.zeros(1 << (2 * N), np.complex128)
    psi[0] = 1.0
    for col in range(2 * ns):
        psi = sum(P[a, col] * cd[a] for a in range(2 * N)) @ psi
    sgn = [(-1) ** (i % L + i // L) for i in range(N)]
    eta_p = sum(sgn[i] * cd[i] @ cd[N + i] for i in range(N))
    e2 = (psi.conj() @ eta_p @ eta_p.conj().T @ psi) / (psi.conj() @ psi)
    assert abs(e2 - _eta2_wick(P, L, ns)) < 1e-12
