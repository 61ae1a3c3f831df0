"""The C-ABI library builds, loads and exports every entry point include/afqmc.h and
include/afqmc_soc.h declare (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2506_09611_gb300 import afqmc, build, soc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols(header=None):
    names = [header] if header else ["afqmc.h", "afqmc_soc.h"]
    syms = set()
    for h in names:
        src = open(os.path.join(ROOT, "include", h)).read()
        syms |= set(re.findall(r"\b(afqmc_[a-z_A-Z]+)\s*\(", src))
    return sorted(syms)


def test_header_declares_the_boundary():
    syms = declared_symbols("afqmc.h")
    for name in ("afqmc_create", "afqmc_destroy", "afqmc_init_walkers", "afqmc_sweep_slice",
                 "afqmc_recompute_G", "afqmc_measure_energy", "afqmc_strerror"):
        assert name in syms
    assert set(syms) == set(afqmc.EXPORTS)
    soc_syms = declared_symbols("afqmc_soc.h")
    assert set(soc_syms) - set(syms) == set(soc.EXPORTS)


def test_library_builds_and_exports_every_symbol():
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    for name in declared_symbols():
        assert re.search(rf"\bT {name}\b", out), name


def test_strerror_without_gpu():
    afqmc.load()
    assert afqmc.strerror(-6) == "call out of sequence"
    assert afqmc.strerror(0) == "ok"


def test_create_rejects_bad_arguments_before_touching_the_device():
    lib = afqmc.load()
    h = ctypes.c_void_p()
    bad = afqmc.afqmc_params(hs=0, precision=1, M=10, stab_every=3, t=1.0, U=4.0, dtau=0.05, seed=1)
    assert lib.afqmc_create(ctypes.byref(h), ctypes.byref(bad)) == -1  # M not a multiple of stab_every
    bad2 = afqmc.afqmc_params(hs=0, precision=1, M=10, stab_every=5, t=1.0, U=-4.0, dtau=0.05, seed=1)
    assert lib.afqmc_create(ctypes.byref(h), ctypes.byref(bad2)) == -1  # spin channel needs U >= 0
    bad3 = afqmc.afqmc_params(hs=7, precision=1, M=10, stab_every=5, t=1.0, U=4.0, dtau=0.05, seed=1)
    assert lib.afqmc_create(ctypes.byref(h), ctypes.byref(bad3)) == -1
    assert lib.afqmc_destroy(None) == 0


def test_dgemm_hook_rejects_bad_arguments_before_touching_the_device():
    lib = afqmc.load()
    p = ctypes.c_void_p(16)  # never dereferenced: the checks come first
    assert lib.afqmc_debug_dgemm(2, 4, 4, 4, p, 4, p, 4, p, 4, None) == -1   # unknown engine
    assert lib.afqmc_debug_dgemm(1, 0, 4, 4, p, 4, p, 4, p, 4, None) == -1   # empty M
    assert lib.afqmc_debug_dgemm(1, 4, 4, 8, p, 4, p, 4, p, 4, None) == -1   # lda < K
    assert lib.afqmc_debug_dgemm(0, 4, 8, 4, p, 4, p, 4, p, 8, None) == -1   # ldb < N
    assert lib.afqmc_debug_dgemm(1, 4, 4, 4, None, 4, p, 4, p, 4, None) == -1  # null operand


def test_gemm_hook_rejects_bad_arguments_before_touching_the_device():
    lib = afqmc.load()
    p = ctypes.c_void_p(16)  # never dereferenced: the checks come first
    assert lib.afqmc_debug_gemm(3, 8, 8, 8, p, 8, p, 8, p, 8, 0, None) == -1   # unknown engine
    assert lib.afqmc_debug_gemm(2, 8, 0, 8, p, 8, p, 8, p, 8, 0, None) == -1   # empty N
    assert lib.afqmc_debug_gemm(2, 8, 8, 16, p, 8, p, 16, p, 8, 0, None) == -1  # lda < K
    assert lib.afqmc_debug_gemm(2, 8, 8, 16, p, 16, p, 8, p, 8, 0, None) == -1  # ldb < K
    assert lib.afqmc_debug_gemm(2, 16, 8, 8, p, 8, p, 8, p, 8, 1, None) == -1   # ldc < M for C^T
    assert lib.afqmc_debug_gemm(1, 8, 8, 8, p, 8, None, 8, p, 8, 0, None) == -1  # null operand


def test_wait_probe_rejects_a_limit_out_of_range_before_touching_the_device():
    lib = afqmc.load()
    assert lib.afqmc_debug_wait_timeout(0, None) == -1
    assert lib.afqmc_debug_wait_timeout(999, None) == -1
    assert lib.afqmc_debug_wait_timeout(2_000_000_001, None) == -1


def test_soc_create_rejects_bad_arguments_before_touching_the_device():
    lib = soc.load()
    h = ctypes.c_void_p()
    good = dict(L=4, M=10, n_e=8, n_walkers=1, precision=0, gemm=0, stab_every=5, t=1.0, lam=0.5, U=-4.0,
                dtau=0.05, seed=1)
    for bad in (dict(U=4.0), dict(stab_every=3), dict(L=1), dict(n_e=33), dict(precision=7), dict(n_walkers=0),
                dict(hs=2), dict(hs=-1)):
        p = soc.afqmc_soc_params(**{**good, **bad})
        assert lib.afqmc_soc_create(ctypes.byref(h), ctypes.byref(p)) == -1, bad
    assert lib.afqmc_soc_destroy(None) == 0


def test_every_entry_point_rejects_a_null_context_without_the_device():
    """Each stateful call of both headers returns AFQMC_ERR_ARG for a NULL context before any CUDA
    call (destroy of NULL is a no-op)."""
    lib = afqmc.load()
    soc.load()
    ARG = -1
    ip = ctypes.c_int()
    d = ctypes.c_double()
    i8 = ctypes.c_int8()
    u8 = ctypes.c_uint8()
    i64 = ctypes.c_int64()
    one = ctypes.c_int(1)
    p = ctypes.byref
    assert lib.afqmc_destroy(None) == 0
    assert lib.afqmc_init_walkers(None, 1, p(one), p(one), p(one), p(d), None, None) == ARG
    assert lib.afqmc_sweep_slice(None, 1, 1, 1, 8, 4, None, None, None) == ARG
    assert lib.afqmc_recompute_G(None, None, None) == ARG
    assert lib.afqmc_measure_energy(None, p(d), p(d), None) == ARG
    assert lib.afqmc_get_G(None, 0, 0, p(d)) == ARG
    assert lib.afqmc_set_G(None, 0, 0, p(d)) == ARG
    assert lib.afqmc_get_fields(None, 0, p(i8)) == ARG
    assert lib.afqmc_get_decisions(None, 0, p(u8)) == ARG
    assert lib.afqmc_get_ratios(None, 0, p(d)) == ARG
    assert lib.afqmc_get_info(None, 0, p(ip), p(ip), p(ip), p(ip), p(ip)) == ARG
    assert lib.afqmc_set_graphs(None, 1) == ARG
    assert lib.afqmc_set_wrap(None, 1) == ARG
    assert lib.afqmc_set_profiling(None, 1) == ARG
    assert lib.afqmc_get_profile(None, p(d), p(i64), p(i64)) == ARG
    assert lib.afqmc_cp_init(None, p(d), None, None) == ARG
    assert lib.afqmc_cp_step(None, 1, 4, 4, None, None) == ARG
    assert lib.afqmc_cp_comb(None, 0.5, None, None) == ARG
    assert lib.afqmc_cp_reorth(None, None) == ARG
    assert lib.afqmc_cp_energy(None, p(d), p(d), None) == ARG
    assert lib.afqmc_cp_get_walker(None, 0, p(d), p(d)) == ARG
    assert lib.afqmc_soc_destroy(None) == 0
    assert lib.afqmc_soc_init(None, p(d), None, None) == ARG
    assert lib.afqmc_soc_sweep_slice(None, 1, 1, 1, 8, 4, None, None) == ARG
    assert lib.afqmc_soc_recompute_G(None, None, None) == ARG
    assert lib.afqmc_soc_measure_energy(None, p(d), None) == ARG
    assert lib.afqmc_soc_measure_pairing(None, p(d), None, None, None) == ARG
    assert lib.afqmc_soc_get_G(None, 0, p(d)) == ARG
    assert lib.afqmc_soc_set_G(None, 0, p(d)) == ARG
    assert lib.afqmc_soc_get_fields(None, 0, p(i8)) == ARG
    assert lib.afqmc_soc_get_decisions(None, 0, p(u8)) == ARG
    assert lib.afqmc_soc_get_ratios(None, 0, p(d)) == ARG
    assert lib.afqmc_soc_get_lam_plus(None, 0, p(d)) == ARG
    assert lib.afqmc_soc_get_info(None, p(ip), p(ip), p(ip)) == ARG
    assert lib.afqmc_soc_set_profiling(None, 1) == ARG
    assert lib.afqmc_soc_get_profile(None, p(d), p(i64), p(i64)) == ARG
