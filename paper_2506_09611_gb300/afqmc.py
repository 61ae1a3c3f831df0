"""Thin ctypes binding of libafqmc.so (include/afqmc.h): argument marshalling only.

Every function mirrors the C entry point of the same name; all arithmetic runs
in the library's CUDA kernels.  ``load()`` raises if the in-tree library is
missing or cannot be loaded -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libafqmc.so")

AFQMC_OK = 0
ERRORS = {-1: "ARG", -2: "OOM", -3: "CUDA", -4: "NUMERIC", -5: "TIMEOUT", -6: "STATE", -7: "NODEV"}
HS_SZ_REAL, HS_CHARGE_REAL = 0, 1
PREC_FP64, PREC_FP32 = 0, 1
MODE_LOCAL, MODE_DELAYED, MODE_BLOCKFB = 0, 1, 2
MODES = {"local": MODE_LOCAL, "delayed": MODE_DELAYED, "blockfb": MODE_BLOCKFB}
PRECS = {"fp64": PREC_FP64, "fp32": PREC_FP32}
GEMMS = {"tc3": 0, "simt": 1, "tf32": 2}

EXPORTS = ["afqmc_create", "afqmc_destroy", "afqmc_init_walkers", "afqmc_sweep_slice", "afqmc_recompute_G",
           "afqmc_measure_energy", "afqmc_get_G", "afqmc_set_G", "afqmc_get_fields", "afqmc_get_decisions",
           "afqmc_get_ratios", "afqmc_get_info", "afqmc_debug_uniforms", "afqmc_set_profiling", "afqmc_set_graphs",
           "afqmc_get_profile", "afqmc_launch_count", "afqmc_apply_flips", "afqmc_apply_flips_noalloc",
           "afqmc_debug_gemm", "afqmc_debug_dgemm", "afqmc_debug_ozaki_plan", "afqmc_debug_wait_timeout",
           "afqmc_set_wrap", "afqmc_set_wrap_tile", "afqmc_set_form", "afqmc_strerror", "afqmc_cp_init",
           "afqmc_cp_step", "afqmc_cp_comb", "afqmc_cp_reorth", "afqmc_cp_energy", "afqmc_cp_get_walker"]
WRAPS = {"dense": 0, "separable": 1}
FORMS = {"G": 0, "T": 1}
PHASES = ["prep", "wrap", "local", "chain", "flush", "recompute", "elim", "wrap_gemm", "flush_gemm", "lu_o",
          "solve", "dgemm"]


class afqmc_params(ctypes.Structure):
    _fields_ = [("hs", ctypes.c_int), ("precision", ctypes.c_int), ("M", ctypes.c_int),
                ("stab_every", ctypes.c_int), ("t", ctypes.c_double), ("U", ctypes.c_double),
                ("dtau", ctypes.c_double), ("seed", ctypes.c_uint64), ("gemm", ctypes.c_int)]


class afqmc_slice_stats(ctypes.Structure):
    _fields_ = [("proposals", ctypes.c_int32), ("accepts", ctypes.c_int32), ("flipped", ctypes.c_int32),
                ("flushes", ctypes.c_int32), ("max_abs_ratio", ctypes.c_double), ("sign", ctypes.c_double)]


class AfqmcError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__(f"{fn} failed: {code} ({ERRORS.get(code, '?')}): {strerror(code)}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it is missing: there is no CPU path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path} is missing; build it with paper_2506_09611_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, ip, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    lib.afqmc_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(afqmc_params)]
    lib.afqmc_destroy.argtypes = [vp]
    lib.afqmc_init_walkers.argtypes = [vp, ctypes.c_int, ip, ip, ip, dp, ctypes.POINTER(ctypes.c_int8), vp]
    lib.afqmc_sweep_slice.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(afqmc_slice_stats), vp]
    lib.afqmc_recompute_G.argtypes = [vp, dp, vp]
    lib.afqmc_measure_energy.argtypes = [vp, dp, dp, vp]
    lib.afqmc_get_G.argtypes = [vp, ctypes.c_int, ctypes.c_int, dp]
    lib.afqmc_set_G.argtypes = [vp, ctypes.c_int, ctypes.c_int, dp]
    lib.afqmc_get_fields.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int8)]
    lib.afqmc_get_decisions.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_uint8)]
    lib.afqmc_get_ratios.argtypes = [vp, ctypes.c_int, dp]
    lib.afqmc_get_info.argtypes = [vp, ctypes.c_int, ip, ip, ip, ip, ip]
    lib.afqmc_debug_uniforms.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, dp]
    lib.afqmc_debug_wait_timeout.argtypes = [ctypes.c_longlong, vp]
    lib.afqmc_set_profiling.argtypes = [vp, ctypes.c_int]
    lib.afqmc_set_graphs.argtypes = [vp, ctypes.c_int]
    lib.afqmc_set_wrap.argtypes = [vp, ctypes.c_int]
    lib.afqmc_set_wrap_tile.argtypes = [vp, ctypes.c_int]
    lib.afqmc_set_form.argtypes = [vp, ctypes.c_int]
    lib.afqmc_cp_init.argtypes = [vp, dp, dp, vp]
    lib.afqmc_cp_step.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, vp]
    lib.afqmc_cp_comb.argtypes = [vp, ctypes.c_double, ip, vp]
    lib.afqmc_cp_reorth.argtypes = [vp, vp]
    lib.afqmc_cp_energy.argtypes = [vp, dp, dp, vp]
    lib.afqmc_cp_get_walker.argtypes = [vp, ctypes.c_int, dp, dp]
    lib.afqmc_get_profile.argtypes = [vp, dp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    lib.afqmc_launch_count.argtypes = []
    lib.afqmc_apply_flips.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_longlong, vp, vp, vp, vp, ctypes.c_int, vp]
    lib.afqmc_apply_flips_noalloc.argtypes = lib.afqmc_apply_flips.argtypes
    ll = ctypes.c_longlong
    lib.afqmc_debug_gemm.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ll, vp, ll, vp, ll,
                                     ctypes.c_int, vp]
    lib.afqmc_debug_dgemm.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ll, vp, ll, vp, ll,
                                      vp]
    lib.afqmc_debug_ozaki_plan.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ip, ip, ip,
                                           ctypes.c_int, ip, ip, ip]
    lib.afqmc_strerror.argtypes = [ctypes.c_int]
    lib.afqmc_strerror.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("afqmc_strerror", "afqmc_launch_count"):
            getattr(lib, name).restype = ctypes.c_int
    lib.afqmc_launch_count.restype = ctypes.c_int64
    _lib = lib
    return lib


def strerror(code: int) -> str:
    return load().afqmc_strerror(code).decode()


def _ck(fn, code):
    if code != AFQMC_OK:
        raise AfqmcError(fn, code)


def _ptr(a, ct):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ct))


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)  # torch.cuda.Stream


# ---------------------------------------------------------------- C-named entry points

def afqmc_create(hs, precision, M, stab_every, t, U, dtau, seed, gemm=0):
    p = afqmc_params(hs=hs, precision=precision, M=M, stab_every=stab_every, t=t, U=U, dtau=dtau, seed=seed,
                     gemm=gemm)
    h = ctypes.c_void_p()
    _ck("afqmc_create", load().afqmc_create(ctypes.byref(h), ctypes.byref(p)))
    return h


def afqmc_destroy(ctx):
    _ck("afqmc_destroy", load().afqmc_destroy(ctx))


def afqmc_init_walkers(ctx, L, n_up, n_dn, P, fields=None, stream=None):
    L = np.ascontiguousarray(L, np.int32)
    nu = np.ascontiguousarray(n_up, np.int32)
    nd = np.ascontiguousarray(n_dn, np.int32)
    P = np.ascontiguousarray(P, np.float64)
    f = None if fields is None else np.ascontiguousarray(fields, np.int8)
    _ck("afqmc_init_walkers", load().afqmc_init_walkers(ctx, len(L), _ptr(L, ctypes.c_int), _ptr(nu, ctypes.c_int),
                                                        _ptr(nd, ctypes.c_int), _ptr(P, ctypes.c_double),
                                                        _ptr(f, ctypes.c_int8), _stream(stream)))


def afqmc_sweep_slice(ctx, slice_, direction, mode, k=32, nb=4, replay=None, stats=None, stream=None):
    rep = None if replay is None else np.ascontiguousarray(replay, np.uint8)
    st = None if stats is None else stats
    _ck("afqmc_sweep_slice", load().afqmc_sweep_slice(ctx, slice_, direction, mode, k, nb, _ptr(rep, ctypes.c_uint8),
                                                      st, _stream(stream)))


def afqmc_recompute_G(ctx, n_walkers=None, stream=None):
    out = None if n_walkers is None else np.zeros(n_walkers)
    _ck("afqmc_recompute_G", load().afqmc_recompute_G(ctx, _ptr(out, ctypes.c_double), _stream(stream)))
    return out


def afqmc_measure_energy(ctx, n_walkers, stream=None):
    e = np.zeros(n_walkers)
    s = np.zeros(n_walkers)
    _ck("afqmc_measure_energy", load().afqmc_measure_energy(ctx, _ptr(e, ctypes.c_double), _ptr(s, ctypes.c_double),
                                                            _stream(stream)))
    return e, s


def afqmc_get_info(ctx, walker):
    v = [ctypes.c_int() for _ in range(5)]
    _ck("afqmc_get_info", load().afqmc_get_info(ctx, walker, *[ctypes.byref(x) for x in v]))
    return dict(zip(("N", "n_up", "n_dn", "slice", "dir"), (x.value for x in v)))


def afqmc_get_G(ctx, walker, spin):
    N = afqmc_get_info(ctx, walker)["N"]
    out = np.zeros((N, N))
    _ck("afqmc_get_G", load().afqmc_get_G(ctx, walker, spin, _ptr(out, ctypes.c_double)))
    return out


def afqmc_set_G(ctx, walker, spin, G):
    G = np.ascontiguousarray(G, np.float64)
    _ck("afqmc_set_G", load().afqmc_set_G(ctx, walker, spin, _ptr(G, ctypes.c_double)))


def afqmc_get_fields(ctx, walker, M):
    N = afqmc_get_info(ctx, walker)["N"]
    out = np.zeros((M, N), np.int8)
    _ck("afqmc_get_fields", load().afqmc_get_fields(ctx, walker, _ptr(out, ctypes.c_int8)))
    return out


def afqmc_get_decisions(ctx, walker):
    N = afqmc_get_info(ctx, walker)["N"]
    out = np.zeros(2 * N, np.uint8)
    _ck("afqmc_get_decisions", load().afqmc_get_decisions(ctx, walker, _ptr(out, ctypes.c_uint8)))
    return out


def afqmc_get_ratios(ctx, walker):
    N = afqmc_get_info(ctx, walker)["N"]
    out = np.zeros(2 * N)
    _ck("afqmc_get_ratios", load().afqmc_get_ratios(ctx, walker, _ptr(out, ctypes.c_double)))
    return out


def afqmc_debug_uniforms(seed, walker, visit, count):
    out = np.zeros(count)
    _ck("afqmc_debug_uniforms", load().afqmc_debug_uniforms(seed, walker, visit, count, _ptr(out, ctypes.c_double)))
    return out


def afqmc_debug_wait_timeout(limit_ns, stream=None):
    """Run the bounded-wait probe for limit_ns; returns the status code (AFQMC_ERR_TIMEOUT expected)."""
    return int(load().afqmc_debug_wait_timeout(int(limit_ns), _stream(stream)))


def afqmc_set_profiling(ctx, on):
    _ck("afqmc_set_profiling", load().afqmc_set_profiling(ctx, int(on)))


def afqmc_set_graphs(ctx, on):
    _ck("afqmc_set_graphs", load().afqmc_set_graphs(ctx, int(on)))


def afqmc_set_wrap(ctx, mode):
    _ck("afqmc_set_wrap", load().afqmc_set_wrap(ctx, WRAPS.get(mode, mode)))


def afqmc_set_form(ctx, form):
    _ck("afqmc_set_form", load().afqmc_set_form(ctx, FORMS.get(form, form)))


def afqmc_cp_init(ctx, P, phi0=None, stream=None):
    P = np.ascontiguousarray(P, np.float64)
    phi = None if phi0 is None else np.ascontiguousarray(phi0, np.float64)
    _ck("afqmc_cp_init", load().afqmc_cp_init(ctx, _ptr(P, ctypes.c_double), _ptr(phi, ctypes.c_double),
                                              _stream(stream)))


def afqmc_cp_step(ctx, n, mode, k=32, nb=4, stream=None):
    out = np.zeros(n)
    _ck("afqmc_cp_step", load().afqmc_cp_step(ctx, MODES.get(mode, mode), int(k), int(nb),
                                              _ptr(out, ctypes.c_double), _stream(stream)))
    return out


def afqmc_cp_comb(ctx, n, u0, stream=None):
    idx = np.zeros(n, np.int32)
    _ck("afqmc_cp_comb", load().afqmc_cp_comb(ctx, float(u0), _ptr(idx, ctypes.c_int), _stream(stream)))
    return idx


def afqmc_cp_reorth(ctx, stream=None):
    _ck("afqmc_cp_reorth", load().afqmc_cp_reorth(ctx, _stream(stream)))


def afqmc_cp_energy(ctx, n, stream=None):
    el = np.zeros(n)
    em = np.zeros(1)
    _ck("afqmc_cp_energy", load().afqmc_cp_energy(ctx, _ptr(el, ctypes.c_double), _ptr(em, ctypes.c_double),
                                                  _stream(stream)))
    return el, float(em[0])


def afqmc_cp_get_walker(ctx, walker, N, ns):
    phi = np.zeros((2, N, ns))
    lw = np.zeros(1)
    _ck("afqmc_cp_get_walker", load().afqmc_cp_get_walker(ctx, walker, _ptr(phi, ctypes.c_double),
                                                          _ptr(lw, ctypes.c_double)))
    return phi, float(lw[0])


def afqmc_set_wrap_tile(ctx, width):
    _ck("afqmc_set_wrap_tile", load().afqmc_set_wrap_tile(ctx, int(width)))


def afqmc_get_profile(ctx):
    n = len(PHASES)
    ms = np.zeros(n)
    iv = np.zeros(n, np.int64)
    la = np.zeros(n, np.int64)
    _ck("afqmc_get_profile", load().afqmc_get_profile(ctx, _ptr(ms, ctypes.c_double), _ptr(iv, ctypes.c_int64),
                                                      _ptr(la, ctypes.c_int64)))
    return {p: {"ms": float(ms[i]), "intervals": int(iv[i]), "launches": int(la[i])} for i, p in enumerate(PHASES)}


def afqmc_apply_flips(precision, N, ld, G_up, G_dn, sites, delta, m, stream=None):
    """All array arguments are device pointers (ints), e.g. torch tensors' data_ptr()."""
    _ck("afqmc_apply_flips", load().afqmc_apply_flips(PRECS.get(precision, precision), N, ld, ctypes.c_void_p(G_up),
                                                      ctypes.c_void_p(G_dn), ctypes.c_void_p(sites),
                                                      ctypes.c_void_p(delta), m, _stream(stream)))


def afqmc_apply_flips_noalloc(precision, N, ld, G_up, G_dn, sites, delta, m, stream=None):
    """Same as afqmc_apply_flips with no device allocation (static device scratch, N <= 4096)."""
    _ck("afqmc_apply_flips_noalloc",
        load().afqmc_apply_flips_noalloc(PRECS.get(precision, precision), N, ld, ctypes.c_void_p(G_up),
                                         ctypes.c_void_p(G_dn), ctypes.c_void_p(sites), ctypes.c_void_p(delta), m,
                                         _stream(stream)))


def afqmc_debug_gemm(kind, M, N, K, A, lda, Bt, ldb, C, ldc, c_trans=0, stream=None):
    """C = A @ Bt.T with the tensor-core kernel (kind 1: TF32, 2: three-term TF32 split); device pointers."""
    _ck("afqmc_debug_gemm", load().afqmc_debug_gemm(kind, M, N, K, ctypes.c_void_p(A), lda, ctypes.c_void_p(Bt), ldb,
                                                    ctypes.c_void_p(C), ldc, c_trans, _stream(stream)))


def afqmc_debug_dgemm(kind, M, N, K, A, lda, B, ldb, C, ldc, stream=None):
    """C = A @ B in FP64 (kind 0: FP64 SIMT, 1: digit-split tensor-core product); device pointers."""
    _ck("afqmc_debug_dgemm", load().afqmc_debug_dgemm(kind, M, N, K, ctypes.c_void_p(A), lda, ctypes.c_void_p(B), ldb,
                                                      ctypes.c_void_p(C), ldc, _stream(stream)))


def afqmc_debug_ozaki_plan(M, N, K, batch=1, cap=128):
    """The digit-split plan for an M x N x K product: (b, s, [[(p, q), ...] per group])."""
    b, s, ng = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    npa = np.zeros(cap, np.int32)
    pa = np.zeros(cap * 16, np.int32)
    pb = np.zeros(cap * 16, np.int32)
    _ck("afqmc_debug_ozaki_plan", load().afqmc_debug_ozaki_plan(M, N, K, batch, ctypes.byref(b), ctypes.byref(s),
                                                                ctypes.byref(ng), cap, _ptr(npa, ctypes.c_int),
                                                                _ptr(pa, ctypes.c_int), _ptr(pb, ctypes.c_int)))
    groups = [[(int(pa[16 * g + i]), int(pb[16 * g + i])) for i in range(int(npa[g]))] for g in range(min(ng.value, cap))]
    return b.value, s.value, groups


def afqmc_launch_count():
    return int(load().afqmc_launch_count())


# ---------------------------------------------------------------- convenience wrapper

class Context:
    """Owns one afqmc_ctx; methods forward to the C entry points above."""

    def __init__(self, M, dtau=0.05, U=4.0, t=1.0, precision="fp64", hs=HS_SZ_REAL, stab_every=10, seed=1,
                 gemm="tc3", form="G"):
        self.M = M
        self.h = afqmc_create(hs, PRECS.get(precision, precision), M, stab_every, t, U, dtau, seed,
                              GEMMS.get(gemm, gemm))
        if form != "G":
            afqmc_set_form(self.h, form)
        self.n = 0

    def init_walkers(self, L, n_up, n_dn, P, fields=None, stream=None):
        self.n = len(L)
        afqmc_init_walkers(self.h, L, n_up, n_dn, P, fields, stream)

    def sweep_slice(self, ell, direction, mode, k=32, nb=4, replay=None, want_stats=False, stream=None):
        stats = (afqmc_slice_stats * self.n)() if want_stats else None
        afqmc_sweep_slice(self.h, ell, direction, MODES.get(mode, mode), k, nb, replay, stats, stream)
        return stats

    def recompute_G(self, stream=None):
        return afqmc_recompute_G(self.h, self.n, stream)

    def measure_energy(self, stream=None):
        return afqmc_measure_energy(self.h, self.n, stream)

    def G(self, walker, spin):
        return afqmc_get_G(self.h, walker, spin)

    def set_G(self, walker, spin, G):
        afqmc_set_G(self.h, walker, spin, G)

    def fields(self, walker):
        return afqmc_get_fields(self.h, walker, self.M)

    def decisions(self, walker):
        return afqmc_get_decisions(self.h, walker)

    def ratios(self, walker):
        return afqmc_get_ratios(self.h, walker)

    def info(self, walker):
        return afqmc_get_info(self.h, walker)

    def set_profiling(self, on=True):
        afqmc_set_profiling(self.h, on)

    def set_graphs(self, on):
        afqmc_set_graphs(self.h, on)

    def set_wrap(self, mode):
        """"dense" or "separable" (E = Ex (x) Ex, two L-point passes per product); a new context uses
        the separable wrap wherever the lattice's tile fits on chip."""
        afqmc_set_wrap(self.h, mode)

    def set_wrap_tile(self, width):
        """Tile width of the separable wrap (0: the default)."""
        afqmc_set_wrap_tile(self.h, width)

    def profile(self):
        return afqmc_get_profile(self.h)

    def close(self):
        if self.h is not None:
            afqmc_destroy(self.h)
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


class CPContext:
    """A constrained-path AFQMC ensemble (Sec. IV.D) of n_walkers determinants on an L x L lattice
    with n_s particles per spin, guided by the trial determinant P (N x n_s, both spins): a
    T-form FP64 context with one slice (its fields hold the current step's fields) and the
    afqmc_cp_* entry points."""

    def __init__(self, L, ns, n_walkers, P, phi0=None, dtau=0.05, U=4.0, t=1.0, hs=HS_SZ_REAL, seed=1,
                 stream=None):
        N = L * L
        self.L, self.N, self.ns, self.n = L, N, ns, n_walkers
        self.ctx = Context(1, dtau=dtau, U=U, t=t, precision="fp64", hs=hs, stab_every=1, seed=seed, form="T")
        P = np.ascontiguousarray(P, np.float64)
        Pw = np.concatenate([np.concatenate([P.ravel(), P.ravel()]) for _ in range(n_walkers)])
        X = np.ones((n_walkers, 1, N), np.int8)
        self.ctx.init_walkers([L] * n_walkers, [ns] * n_walkers, [ns] * n_walkers, Pw, X, stream)
        afqmc_cp_init(self.ctx.h, P, phi0, stream)

    def step(self, mode="delayed", k=16, nb=4, stream=None):
        return afqmc_cp_step(self.ctx.h, self.n, mode, k, nb, stream)

    def comb(self, u0, stream=None):
        return afqmc_cp_comb(self.ctx.h, self.n, u0, stream)

    def reorth(self, stream=None):
        afqmc_cp_reorth(self.ctx.h, stream)

    def energy(self, stream=None):
        return afqmc_cp_energy(self.ctx.h, self.n, stream)

    def walker(self, j):
        return afqmc_cp_get_walker(self.ctx.h, j, self.N, self.ns)

    def fields(self, j):
        return self.ctx.fields(j)[0]

    def close(self):
        self.ctx.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
