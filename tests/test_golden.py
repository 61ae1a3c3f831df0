"""Stored U = 0 energies (tests/golden/free_fermion_energies.txt, written from the dispersion
relations of Eqs. 2DHubbard and 2DSocHubbard by tests/golden/make_free_fermion_energies.py): the
file regenerates exactly, and the FP64 oracle's mixed-estimator energy at U = 0 reproduces the
stored values on the lattices it evaluates in seconds."""
import importlib.util
import os

import numpy as np
import pytest

import oracle
from paper_2506_09611_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _generator():
    spec = importlib.util.spec_from_file_location("make_ffe", os.path.join(GOLDEN, "make_free_fermion_energies.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _table():
    rows = {}
    with open(os.path.join(GOLDEN, "free_fermion_energies.txt")) as f:
        for line in f:
            if line.startswith("#"):
                continue
            name, kind, L, n, t, lam, e = line.split("#")[0].split()
            rows[name] = (kind, int(L), int(n), float(t), float(lam), float(e))
    return rows


def test_golden_file_regenerates():
    with open(os.path.join(GOLDEN, "free_fermion_energies.txt")) as f:
        assert f.read().splitlines() == _generator().lines()


@pytest.mark.parametrize("name", ["hubbard_4x4", "hubbard_16x16"])
def test_oracle_reproduces_hubbard_energy(name):
    kind, L, ns, t, lam, e = _table()[name]
    M = 4
    m = oracle.Model(L, L, t, 0.0, 0.05, M)
    P = inputs.trial_state(L, L, ns)
    X = inputs.initial_fields(M, L * L)
    Gs = [m.green_scratch(X, P, s, 2)[0] for s in range(2)]
    assert abs(m.energy(Gs[0], Gs[1]) - e) < 1e-8


def test_oracle_reproduces_soc_energy():
    kind, L, ne, t, lam, e = _table()["soc_4x4"]
    M = 4
    m = oracle.SocModel(L, t, lam, 0.0, 0.05, M)
    P = inputs.soc_trial_state(L, ne, t=t, lam=lam)
    X = inputs.initial_fields(M, L * L)
    G, _, _ = m.green_scratch(X, P, 2)
    assert abs(m.energy(G).real - e) < 1e-8
