"""Pins of the CPQMC oracle (oracle/cpqmc.py; Sec. IV.D, Eqs. CPWvfct1, CPWvfct2, ptilde) against what the
mathematics fixes, by numpy brute force that shares nothing with it:

* the heat-bath normalisation N_i of a site is sum_x p(x) <psi_T|B_i(x)|phi> / <psi_T|phi> from plain
  determinants, for both decouplings;
* one projection step is unbiased: enumerating every field outcome of a 2 x 2 lattice with its
  sampling probability, sum prob * w' <chi|phi'> / <psi_T|phi'> equals the exact
  sum_x p(x) <chi|B(x) e^{-dtau K}|phi> / <psi_T|phi> (Eq. CPWvfct2) for random test determinants chi,
  for the local heat bath and for block force bias with n_b = 1, 2 and N (the full scheme);
* the comb keeps the total weight and gives walker k floor or ceil of n_w w_k / W copies;
* the mixed energy equals the Fock-space <psi_T|H|phi> / <psi_T|phi>.
Nothing here uses the CUDA library.
"""
import itertools

import numpy as np
import pytest

import oracle
from oracle.cpqmc import CPEnsemble
from paper_2506_09611_gb300 import inputs
from tests import bruteforce as bf


def _ens(L=2, ns=1, U=2.0, dtau=0.05, hs=oracle.HS_SZ_REAL, n_w=1, seed=3):
    m = oracle.Model(L, L, 1.0, U, dtau, 4, hs=hs)
    P = inputs.trial_state(L, L, ns)
    rng = np.random.default_rng(seed)
    phi = P + 0.3 * rng.standard_normal(P.shape)  # a walker away from the trial
    return m, P, CPEnsemble(m, P, n_w, phi0=phi)


def _ratio(e, k, i, x):
    """<psi_T| b_i(x) |phi_k> / <psi_T|phi_k> from determinants (including the scalar s(x))."""
    c = e.m.c
    num = den = 1.0
    for s in range(2):
        D = np.eye(e.m.N)
        D[i, i] = np.exp(c[s] * x)
        num *= np.linalg.det(e.UL @ D @ e.UR[k][s])
        den *= np.linalg.det(e.UL @ e.UR[k][s])
    return e.s(x) * num / den


@pytest.mark.parametrize("hs,U", [(oracle.HS_SZ_REAL, 2.0), (oracle.HS_CHARGE_REAL, -2.0)])
def test_heat_bath_normalisation_is_the_overlap_ratio_sum(hs, U):
    m, P, e = _ens(L=3, ns=3, U=U, hs=hs)
    e.kinetic()
    ref = []
    for i in range(m.N):
        ref.append(0.5 * (_ratio(e, 0, i, +1) + _ratio(e, 0, i, -1)))
        # set the field the sampler would set with u = 0.3, to follow the same sequence
        r_plus = 0.5 * _ratio(e, 0, i, +1)
        x = 1 if 0.3 < r_plus / ref[-1] else -1
        e._set_field(0, i, x)
    m2, P2, e2 = _ens(L=3, ns=3, U=U, hs=hs)
    e2.kinetic()
    _, norm, _ = e2.local_fields(0, np.full(m.N, 0.3))
    np.testing.assert_allclose(norm, ref, rtol=1e-12)


def _overlap_with(e, chi, k):
    return np.prod([np.linalg.det(chi[s].T @ e.UR[k][s]) for s in range(2)])


def _exact_step(m, P, phi, chi):
    """sum_x p(x) s(x) <chi| D(x) E |phi> / <psi_T|phi> over all 2^N fields."""
    N, c = m.N, m.c
    den = np.prod([np.linalg.det(P.T @ phi) for _ in range(2)])
    tot = 0.0
    charge = m.p.hs == 1
    for bits in itertools.product((1, -1), repeat=N):
        x = np.array(bits, dtype=np.float64)
        sx = np.prod(np.exp(-m.lam * x)) if charge else 1.0
        num = np.prod([np.linalg.det(chi[s].T @ bf.B_mat(m.E, c[s], x.astype(np.int8)) @ phi) for s in range(2)])
        tot += 0.5 ** N * sx * num
    return tot / den


@pytest.mark.parametrize("mode,nb", [("local", 1), ("blockfb", 1), ("blockfb", 2), ("blockfb", 4)])
@pytest.mark.parametrize("hs,U", [(oracle.HS_SZ_REAL, 1.0), (oracle.HS_CHARGE_REAL, -1.5)])
def test_one_step_is_unbiased(mode, nb, hs, U):
    L, ns = 2, 1
    m, P, e0 = _ens(L, ns, U, 0.1, hs)
    phi = e0.UR[0][0].copy()
    rng = np.random.default_rng(11)
    chis = [[rng.standard_normal((m.N, ns)) for _ in range(2)] for _ in range(3)]
    N = m.N
    got = np.zeros(len(chis))
    total_prob = 0.0
    for bits in itertools.product((0, 1), repeat=N):
        e = CPEnsemble(m, P, 1, phi0=phi)
        u = np.where(np.array(bits) == 0, 0.0, 1.0 - 1e-15)  # 0 -> x = +1, else x = -1
        (x, fac, pp), = e.step(mode, u[None, :], nb=nb)
        prob = np.prod(np.where(x > 0, pp, 1.0 - pp))
        assert e.w[0] > 0  # no constraint hit on this workload: the step is exact
        total_prob += prob
        for j, chi in enumerate(chis):
            got[j] += prob * e.w[0] * _overlap_with(e, chi, 0) / e.overlap(0)
    assert abs(total_prob - 1.0) < 1e-12
    for j, chi in enumerate(chis):
        ref = _exact_step(m, P, phi, chi)
        assert abs(got[j] - ref) < 1e-11 * max(1.0, abs(ref)), (j, got[j], ref)


def test_comb_keeps_the_total_weight_and_the_expected_copies():
    m, P, e = _ens(L=2, ns=1, n_w=7)
    rng = np.random.default_rng(2)
    e.w = rng.uniform(0.1, 3.0, 7)
    W = e.w.sum()
    expect = 7 * e.w / W
    tags = [k for k in range(7)]
    for k in range(7):
        e.UR[k][0][0, 0] = 1000.0 + k  # tag each walker
    idx = e.comb(0.37)
    assert abs(e.w.sum() - W) < 1e-12 and np.allclose(e.w, W / 7)
    counts = np.bincount(idx, minlength=7)
    assert np.all((counts == np.floor(expect)) | (counts == np.ceil(expect)))
    assert [int(e.UR[j][0][0, 0] - 1000) for j in range(7)] == [tags[i] for i in idx]


def test_mixed_energy_equals_fock_space():
    m, P, e = _ens(L=2, ns=1, U=3.0)
    ref = bf.fock_energy(m.K, 3.0, e.UR[0][0], e.UL, e.UR[0][1], e.UL)
    assert abs(e.local_energy(0) - ref) < 1e-11 * max(1.0, abs(ref))


def test_free_walker_weight_and_energy():
    """U = 0: every field leaves the walker unchanged (c = 0, N_i = 1), so one step multiplies the
    weight by the kinetic overlap ratio alone, e^{-dtau E_0} for the trial's levels (E_0 = -24 on
    4 x 4 with 7 per spin, up to the trial's 1e-6 perturbation), and the mixed energy is E_0."""
    m = oracle.Model(4, 4, 1.0, 0.0, 0.05, 4)
    P = inputs.trial_state(4, 4, 7)
    e = CPEnsemble(m, P, 2)
    assert abs(e.energy() - (-24.0)) < 1e-5
    out = e.step("local", inputs.uniforms(1, 0, 0, 2 * 16).reshape(2, 16))
    assert all(np.allclose(o[1], 1.0) for o in out)
    assert np.allclose(e.w, np.exp(0.05 * 24.0), rtol=1e-5)
    assert abs(e.energy() - (-24.0)) < 1e-5


@pytest.mark.parametrize("hs,U", [(oracle.HS_SZ_REAL, 2.0), (oracle.HS_CHARGE_REAL, -2.0)])
def test_force_bias_is_the_derivative_of_the_log_overlap(hs, U):
    """The block proposal q(x_i) = e^{x_i F_i} / (2 cosh F_i) carries the force bias
    F_i = d/de log <psi_T| e^{e v_i} |phi> at e = 0, v_i the field's one-body exponent per unit x
    (sum_s c_s n_is, plus -lam for the charge channel's scalar): a finite difference of plain
    determinants.  (Any proposal keeps the step unbiased, so only this pins the bias itself.)"""
    m, P, e = _ens(L=3, ns=3, U=U, hs=hs)
    e.kinetic()
    phi = [e.UR[0][0].copy(), e.UR[0][1].copy()]
    (x, fac, pp), = [e.block_fields(0, np.full(m.N, 0.5), m.N)]
    F = 0.5 * np.log(pp / (1.0 - pp))
    h = 1e-6
    for i in range(m.N):
        def logov(eps):
            v = -m.lam * eps if hs == oracle.HS_CHARGE_REAL else 0.0
            for s in range(2):
                D = np.eye(m.N)
                D[i, i] = np.exp(eps * m.c[s])
                v += np.log(abs(np.linalg.det(e.UL @ D @ phi[s])))
            return v
        fd = (logov(h) - logov(-h)) / (2 * h)
        assert abs(F[i] - fd) < 1e-7, (i, F[i], fd)
