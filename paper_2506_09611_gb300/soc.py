"""Thin ctypes binding of the spin-orbit-coupled sweep (include/afqmc_soc.h): argument
marshalling only.  Every function mirrors the C entry point of the same name; all arithmetic
runs in the library's CUDA kernels, and ``afqmc.load()`` raises if the library is missing."""
from __future__ import annotations

import ctypes

import numpy as np

from . import afqmc
from .afqmc import MODES, PRECS, GEMMS, PHASES, _ck, _ptr, _stream

EXPORTS = ["afqmc_soc_create", "afqmc_soc_destroy", "afqmc_soc_init", "afqmc_soc_sweep_slice",
           "afqmc_soc_recompute_G", "afqmc_soc_measure_energy", "afqmc_soc_get_G", "afqmc_soc_set_G",
           "afqmc_soc_get_fields", "afqmc_soc_get_decisions", "afqmc_soc_get_ratios", "afqmc_soc_get_lam_plus",
           "afqmc_soc_get_info", "afqmc_soc_set_profiling", "afqmc_soc_get_profile", "afqmc_soc_measure_pairing"]
KMAX = {"fp32": 64, "fp64": 32}


class afqmc_soc_params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("M", ctypes.c_int), ("n_e", ctypes.c_int), ("n_walkers", ctypes.c_int),
                ("precision", ctypes.c_int), ("gemm", ctypes.c_int), ("stab_every", ctypes.c_int),
                ("t", ctypes.c_double), ("lam", ctypes.c_double), ("U", ctypes.c_double),
                ("dtau", ctypes.c_double), ("seed", ctypes.c_uint64), ("hs", ctypes.c_int)]


HS = {"sy": 0, "sz": 1}  # AFQMC_SOC_HS_SY, AFQMC_SOC_HS_SZ


_done = False


def load():
    global _done
    lib = afqmc.load()
    if _done:
        return lib
    vp, ip, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.afqmc_soc_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(afqmc_soc_params)]
    lib.afqmc_soc_destroy.argtypes = [vp]
    lib.afqmc_soc_init.argtypes = [vp, dp, ctypes.POINTER(ctypes.c_int8), vp]
    lib.afqmc_soc_sweep_slice.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_uint8), vp]
    lib.afqmc_soc_recompute_G.argtypes = [vp, dp, vp]
    lib.afqmc_soc_measure_energy.argtypes = [vp, dp, vp]
    lib.afqmc_soc_measure_pairing.argtypes = [vp, dp, dp, dp, vp]
    lib.afqmc_soc_get_G.argtypes = [vp, ctypes.c_int, dp]
    lib.afqmc_soc_set_G.argtypes = [vp, ctypes.c_int, dp]
    lib.afqmc_soc_get_fields.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int8)]
    lib.afqmc_soc_get_decisions.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_uint8)]
    lib.afqmc_soc_get_ratios.argtypes = [vp, ctypes.c_int, dp]
    lib.afqmc_soc_get_lam_plus.argtypes = [vp, ctypes.c_int, dp]
    lib.afqmc_soc_get_info.argtypes = [vp, ip, ip, ip]
    lib.afqmc_soc_set_profiling.argtypes = [vp, ctypes.c_int]
    lib.afqmc_soc_get_profile.argtypes = [vp, dp, i64p, i64p]
    for name in EXPORTS:
        getattr(lib, name).restype = ctypes.c_int
    _done = True
    return lib


def afqmc_soc_create(L, M, n_e, n_walkers=1, precision="fp64", gemm="tc3", stab_every=10, t=1.0, lam=0.5, U=-4.0,
                     dtau=0.05, seed=1, hs="sy"):
    p = afqmc_soc_params(L=L, M=M, n_e=n_e, n_walkers=n_walkers, precision=PRECS.get(precision, precision),
                         gemm=GEMMS.get(gemm, gemm), stab_every=stab_every, t=t, lam=lam, U=U, dtau=dtau, seed=seed,
                         hs=HS.get(hs, hs))
    h = ctypes.c_void_p()
    _ck("afqmc_soc_create", load().afqmc_soc_create(ctypes.byref(h), ctypes.byref(p)))
    return h


def afqmc_soc_destroy(ctx):
    _ck("afqmc_soc_destroy", load().afqmc_soc_destroy(ctx))


def afqmc_soc_init(ctx, P, fields=None, stream=None):
    """P: 2N x n_e complex trial determinant (host)."""
    Pi = np.ascontiguousarray(np.asarray(P, np.complex128)).view(np.float64)
    f = None if fields is None else np.ascontiguousarray(fields, np.int8)
    _ck("afqmc_soc_init", load().afqmc_soc_init(ctx, _ptr(Pi, ctypes.c_double), _ptr(f, ctypes.c_int8),
                                                _stream(stream)))


def afqmc_soc_sweep_slice(ctx, slice_, direction, mode, k=32, nb=16, replay=None, stream=None):
    rep = None if replay is None else np.ascontiguousarray(replay, np.uint8)
    _ck("afqmc_soc_sweep_slice", load().afqmc_soc_sweep_slice(ctx, slice_, direction, MODES.get(mode, mode), k, nb,
                                                              _ptr(rep, ctypes.c_uint8), _stream(stream)))


def afqmc_soc_recompute_G(ctx, n_walkers=None, stream=None):
    out = None if n_walkers is None else np.zeros(n_walkers)
    _ck("afqmc_soc_recompute_G", load().afqmc_soc_recompute_G(ctx, _ptr(out, ctypes.c_double), _stream(stream)))
    return out


def afqmc_soc_measure_energy(ctx, n_walkers, stream=None):
    e = np.zeros(2 * n_walkers)
    _ck("afqmc_soc_measure_energy", load().afqmc_soc_measure_energy(ctx, _ptr(e, ctypes.c_double), _stream(stream)))
    return e[0::2] + 1j * e[1::2]


def afqmc_soc_get_info(ctx):
    v = [ctypes.c_int() for _ in range(3)]
    _ck("afqmc_soc_get_info", load().afqmc_soc_get_info(ctx, *[ctypes.byref(x) for x in v]))
    return dict(zip(("N", "slice", "dir"), (x.value for x in v)))


def afqmc_soc_get_G(ctx, walker):
    N = afqmc_soc_get_info(ctx)["N"]
    out = np.zeros((2 * N, 2 * N), np.complex128)
    _ck("afqmc_soc_get_G", load().afqmc_soc_get_G(ctx, walker, _ptr(out.view(np.float64), ctypes.c_double)))
    return out


def afqmc_soc_set_G(ctx, walker, G):
    Gi = np.ascontiguousarray(np.asarray(G, np.complex128)).view(np.float64)
    _ck("afqmc_soc_set_G", load().afqmc_soc_set_G(ctx, walker, _ptr(Gi, ctypes.c_double)))


def afqmc_soc_get_fields(ctx, walker, M):
    N = afqmc_soc_get_info(ctx)["N"]
    out = np.zeros((M, N), np.int8)
    _ck("afqmc_soc_get_fields", load().afqmc_soc_get_fields(ctx, walker, _ptr(out, ctypes.c_int8)))
    return out


def afqmc_soc_get_decisions(ctx, walker):
    N = afqmc_soc_get_info(ctx)["N"]
    out = np.zeros(2 * N, np.uint8)
    _ck("afqmc_soc_get_decisions", load().afqmc_soc_get_decisions(ctx, walker, _ptr(out, ctypes.c_uint8)))
    return out


def afqmc_soc_get_ratios(ctx, walker):
    N = afqmc_soc_get_info(ctx)["N"]
    out = np.zeros(4 * N)
    _ck("afqmc_soc_get_ratios", load().afqmc_soc_get_ratios(ctx, walker, _ptr(out, ctypes.c_double)))
    return out[0::2] + 1j * out[1::2]


def afqmc_soc_get_lam_plus(ctx, walker):
    N = afqmc_soc_get_info(ctx)["N"]
    out = np.zeros(N)
    _ck("afqmc_soc_get_lam_plus", load().afqmc_soc_get_lam_plus(ctx, walker, _ptr(out, ctypes.c_double)))
    return out


def afqmc_soc_set_profiling(ctx, on):
    _ck("afqmc_soc_set_profiling", load().afqmc_soc_set_profiling(ctx, int(on)))


def afqmc_soc_get_profile(ctx):
    n = len(PHASES)
    ms = np.zeros(n)
    iv = np.zeros(n, np.int64)
    la = np.zeros(n, np.int64)
    _ck("afqmc_soc_get_profile", load().afqmc_soc_get_profile(ctx, _ptr(ms, ctypes.c_double),
                                                              _ptr(iv, ctypes.c_int64), _ptr(la, ctypes.c_int64)))
    return {p: {"ms": float(ms[i]), "intervals": int(iv[i]), "launches": int(la[i])} for i, p in enumerate(PHASES)}


def afqmc_soc_measure_pairing(ctx, n_walkers, N, want_k=True, stream=None):
    """Per walker D and <Delta^2> (complex arrays), and with want_k the momentum occupations nk
    (n_walkers x 2N complex) and the pairing matrices Mk (n_walkers x N x N complex)."""
    sc = np.zeros(4 * n_walkers)
    nk = np.zeros(4 * N * n_walkers) if want_k else None
    Mk = np.zeros(2 * N * N * n_walkers) if want_k else None
    _ck("afqmc_soc_measure_pairing", load().afqmc_soc_measure_pairing(
        ctx, _ptr(sc, ctypes.c_double), _ptr(nk, ctypes.c_double), _ptr(Mk, ctypes.c_double), _stream(stream)))
    r = {"D": sc[0::4] + 1j * sc[1::4], "Delta2": sc[2::4] + 1j * sc[3::4]}
    if want_k:
        r["nk"] = nk.view(np.complex128).reshape(n_walkers, 2 * N)
        r["Mk"] = Mk.view(np.complex128).reshape(n_walkers, N, N)
    return r


class SocContext:
    """Owns one afqmc_soc_ctx; methods forward to the C entry points above.  hs: "sy" (spin-y
    channel) or "sz" (the imaginary spin-z channel; with lam = 0 the attractive Hubbard model)."""

    def __init__(self, L, M, n_e, n_walkers=1, precision="fp64", gemm="tc3", stab_every=10, t=1.0, lam=0.5, U=-4.0,
                 dtau=0.05, seed=1, hs="sy"):
        self.M, self.n, self.N = M, n_walkers, L * L
        self.h = afqmc_soc_create(L, M, n_e, n_walkers, precision, gemm, stab_every, t, lam, U, dtau, seed, hs)

    def init(self, P, fields=None, stream=None):
        afqmc_soc_init(self.h, P, fields, stream)

    def sweep_slice(self, ell, direction, mode, k=32, nb=16, replay=None, stream=None):
        afqmc_soc_sweep_slice(self.h, ell, direction, mode, k, nb, replay, stream)

    def recompute_G(self, stream=None):
        return afqmc_soc_recompute_G(self.h, self.n, stream)

    def measure_energy(self, stream=None):
        return afqmc_soc_measure_energy(self.h, self.n, stream)

    def measure_pairing(self, want_k=True, stream=None):
        return afqmc_soc_measure_pairing(self.h, self.n, self.N, want_k, stream)

    def G(self, walker=0):
        return afqmc_soc_get_G(self.h, walker)

    def set_G(self, walker, G):
        afqmc_soc_set_G(self.h, walker, G)

    def fields(self, walker=0):
        return afqmc_soc_get_fields(self.h, walker, self.M)

    def decisions(self, walker=0):
        return afqmc_soc_get_decisions(self.h, walker)

    def ratios(self, walker=0):
        return afqmc_soc_get_ratios(self.h, walker)

    def lam_plus(self, walker=0):
        return afqmc_soc_get_lam_plus(self.h, walker)

    def info(self):
        return afqmc_soc_get_info(self.h)

    def set_profiling(self, on=True):
        afqmc_soc_set_profiling(self.h, on)

    def profile(self):
        return afqmc_soc_get_profile(self.h)

    def close(self):
        if self.h is not None:
            afqmc_soc_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
