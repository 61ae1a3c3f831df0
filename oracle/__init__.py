"""FP64 CPU oracle for the PQMC auxiliary-field update sweep -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The CUDA
library never calls it and shares no code with it.

The arithmetic lives in ``afqmc_oracle.c`` (plain C, FP64, plain loops, its
own LU and Householder QR) and ``soc_oracle.c`` (the spin-orbit-coupled model
in double complex, its own complex LU and Gram-Schmidt).  This module only compiles it with gcc and
marshals numpy arrays through ctypes.  Every function cites the paper's
passage it follows (see the C source for the formulas).

Parity status of each function (what pins it in ``tests/test_oracle_pins.py``):
  expK            -- scipy.linalg.expm of an independently built K; closed-form spectrum
  setup (HS)      -- the decoupling identity checked for all four occupations
  green_scratch   -- numpy products + solve (unstabilised), projector invariants
  wrap            -- numpy from-scratch G at the next slice
  local_slice     -- brute-force det ratio of the walker overlap; from-scratch G
  delayed_slice   -- identical decisions to local; from-scratch G
  blockfb_slice   -- brute-force stripped force bias, det ratio, exact detailed
                     balance on an enumerable toy, from-scratch G
  energy          -- U=0 closed form; Fock-space brute force on <= 3 sites
  wrap_fft        -- the momentum-space wrap (FFT propagation) equals the dense wrap
  tform_wrap      -- U_L U_R unchanged; 1 - U_R T U_L equals the wrapped G
  tform_delayed_slice
                  -- the paper's T-form delayed update (Sec. III.A): identical decisions and
                     ratios to the G-form oracle and the same G = 1 - U_R T U_L after every
                     slice; T stays (U_L U_R)^{-1} of the updated factors
  tform_blockfb_slice
                  -- the T-form block force bias (Sec. III.B): the same stripped densities,
                     proposals, decisions and ratios as the G-form oracle; the same G

Spin-orbit-coupled model (``soc_oracle.c``, Appendix A), pinned in
``tests/test_soc_oracle_pins.py``:
  H0, expH        -- bond-by-bond real-space H0; split dispersion eps_k +- |L_k|; expm
  HS spin-y       -- the decoupling identity and the one-body rotation on the Fock space
  green_scratch   -- plain products of expm propagators; projector invariants; the weight of a
                     time-reversal-invariant trial state is real positive
  wrap            -- from-scratch G at the next / previous slice
  local_slice     -- every ratio equals the brute-force weight ratio; from-scratch G
  delayed_slice   -- identical decisions, ratios and G to the local update
  block_force_bias-- finite difference of the stripped overlap (fixes the index order)
  blockfb_slice   -- brute-force ratio with the proposal ratio; from-scratch G; exact detailed
                     balance on an enumerable 2 x 2 lattice
  energy          -- U=0 closed form; Fock-space brute force with a random spin-mixing H0
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "afqmc_oracle.c"), os.path.join(_HERE, "soc_oracle.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

HS_SZ_REAL = 0
HS_CHARGE_REAL = 1


class Params(ctypes.Structure):
    _fields_ = [
        ("Lx", ctypes.c_int), ("Ly", ctypes.c_int), ("N", ctypes.c_int), ("M", ctypes.c_int),
        ("hs", ctypes.c_int),
        ("t", ctypes.c_double), ("U", ctypes.c_double), ("dtau", ctypes.c_double),
        ("lam", ctypes.c_double), ("c", ctypes.c_double * 2),
    ]


class SocParams(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_int), ("N", ctypes.c_int),
        ("t", ctypes.c_double), ("lam", ctypes.c_double), ("U", ctypes.c_double), ("dtau", ctypes.c_double),
        ("gamma", ctypes.c_double), ("hs", ctypes.c_int),
    ]


SOC_HS = {"sy": 0, "sz": 1}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build/liboracle.so."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(s) for s in _SRCS):
            os.makedirs(_BUILD, exist_ok=True)
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11", "-o", tmp, *_SRCS, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        i8p = ctypes.POINTER(ctypes.c_int8)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        pp = ctypes.POINTER(Params)
        lib.or_setup.argtypes = [pp]
        lib.or_expK.argtypes = [pp, ctypes.c_double, dp]
        lib.or_hopping.argtypes = [pp, dp]
        lib.or_green_scratch.argtypes = [pp, dp, i8p, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, dp, dp, dp, dp]
        lib.or_green_scratch.restype = ctypes.c_int
        lib.or_wrap.argtypes = [pp, dp, dp, i8p, ctypes.c_int, ctypes.c_int, dp]
        lib.or_local_slice.argtypes = [pp, dp, dp, i8p, dp, u8p, u8p, dp, dp]
        lib.or_delayed_slice.argtypes = [pp, dp, dp, i8p, dp, ctypes.c_int, ctypes.c_int, u8p, u8p, dp,
                                         dp, ctypes.POINTER(ctypes.c_int)]
        lib.or_block_force_bias.argtypes = [pp, dp, i8p, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
        lib.or_blockfb_slice.argtypes = [pp, dp, dp, i8p, dp, dp, ctypes.c_int, u8p, i8p, dp, u8p, dp, dp]
        lib.or_energy.argtypes = [pp, dp, dp, dp]
        lib.or_tform_wrap.argtypes = [pp, dp, dp, i8p, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp]
        lib.or_tform_delayed_slice.argtypes = [pp, dp, dp, dp, dp, dp, dp, ctypes.c_int, ctypes.c_int, i8p, dp,
                                               ctypes.c_int, ctypes.c_int, u8p, u8p, dp, dp, ctypes.POINTER(ctypes.c_int)]
        lib.or_tform_blockfb_slice.argtypes = [pp, dp, dp, dp, dp, dp, dp, ctypes.c_int, ctypes.c_int, i8p, dp, dp,
                                               ctypes.c_int, u8p, i8p, dp, u8p, dp, dp]
        lib.or_energy.restype = ctypes.c_double
        sp = ctypes.POINTER(SocParams)
        vp = ctypes.c_void_p
        lib.soc_setup.argtypes = [sp]
        lib.soc_H0.argtypes = [sp, vp]
        lib.soc_expH.argtypes = [sp, ctypes.c_double, vp]
        lib.soc_green_scratch.argtypes = [sp, vp, i8p, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          vp, dp, vp]
        lib.soc_green_scratch.restype = ctypes.c_int
        lib.soc_wrap.argtypes = [sp, vp, vp, i8p, vp, ctypes.c_int]
        lib.soc_local_slice.argtypes = [sp, vp, i8p, dp, u8p, u8p, dp]
        lib.soc_delayed_slice.argtypes = [sp, vp, i8p, dp, ctypes.c_int, u8p, u8p, dp]
        lib.soc_block_force_bias.argtypes = [sp, vp, i8p, ctypes.c_int, ctypes.c_int, vp]
        lib.soc_blockfb_slice.argtypes = [sp, vp, i8p, dp, dp, ctypes.c_int, u8p, i8p, dp, u8p, dp]
        lib.soc_energy.argtypes = [sp, vp, vp, dp]
        lib.soc_pairing.argtypes = [sp, vp, dp, vp, vp]
        _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i8(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))


def _u8(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Model:
    """Physical parameters + E = exp(-dtau K), Einv = exp(+dtau K) (Eq. 2DHubbard, Eq. BlMat)."""

    def __init__(self, Lx, Ly, t, U, dtau, M, hs=HS_SZ_REAL):
        self.p = Params(Lx=Lx, Ly=Ly, N=Lx * Ly, M=M, hs=hs, t=t, U=U, dtau=dtau)
        if _load().or_setup(ctypes.byref(self.p)) != 0:
            raise ValueError("unsupported HS mode / sign of U")
        self.N = Lx * Ly
        self.M = M
        self.E = self.expK(dtau)
        self.Einv = self.expK(-dtau)
        self.K = np.zeros((self.N, self.N))
        _load().or_hopping(ctypes.byref(self.p), _d(self.K))

    @property
    def lam(self):
        return self.p.lam

    @property
    def c(self):
        return (self.p.c[0], self.p.c[1])

    def expK(self, tau):
        E = np.zeros((self.N, self.N))
        _load().or_expK(ctypes.byref(self.p), float(tau), _d(E))
        return E

    def green_scratch(self, x, P, spin, ell, stab=10, want_factors=False):
        """G(ell) = 1 - R (L R)^{-1} L from scratch (Eqs. GrFMat, GrFMatNew).
        Returns (G, sign(det L R), log|det L R|[, U_R, U_L])."""
        N = self.N
        x = np.ascontiguousarray(x, dtype=np.int8)
        P = _f64(P)
        ns = P.shape[1]
        G = np.zeros((N, N))
        la = np.zeros(1)
        UR = np.zeros((N, ns))
        UL = np.zeros((ns, N))
        sg = _load().or_green_scratch(ctypes.byref(self.p), _d(self.E), _i8(x), _d(P), ns, spin, ell, stab,
                                      _d(G), _d(la), _d(UR), _d(UL))
        if want_factors:
            return G, sg, la[0], UR, UL
        return G, sg, la[0]

    def wrap(self, G, xl, spin, direction):
        """Forward (direction=+1): G <- B_l G B_l^{-1}; backward: G <- B_l^{-1} G B_l (Eq. BlMat)."""
        G = _f64(G).copy()
        xl = np.ascontiguousarray(xl, dtype=np.int8)
        _load().or_wrap(ctypes.byref(self.p), _d(self.E), _d(self.Einv), _i8(xl), spin, direction, _d(G))
        return G

    def wrap_fft(self, G, xl, spin, direction):
        """The wrap of Eq. BlMat with exp(-+dtau K) applied in momentum space (the paper's FFT
        propagation, Sec. II.C): on the periodic lattice K is diagonal in the 2D Fourier basis with
        eigenvalues eps_k = -2t (cos kx + cos ky), so E X = F^{-1} diag(e^{-dtau eps_k}) F X for every
        column of X (numpy's FFT over the site index reshaped to (Ly, Lx)).  G E^{-1} = (E^{-1} G^T)^T
        because E is symmetric.  The same moves as `wrap`."""
        Lx, Ly, N = self.p.Lx, self.p.Ly, self.N
        kx = 2 * np.pi * np.arange(Lx) / Lx
        ky = 2 * np.pi * np.arange(Ly) / Ly
        eps = -2.0 * self.p.t * (np.cos(kx)[None, :] + np.cos(ky)[:, None])  # (Ly, Lx)

        def apply_E(X, tau):  # exp(-tau K) X, X: N x m, site index = x + Lx y
            Xr = X.reshape(Ly, Lx, -1)
            Xk = np.fft.fft2(Xr, axes=(0, 1))
            return np.real(np.fft.ifft2(Xk * np.exp(-tau * eps)[:, :, None], axes=(0, 1))).reshape(N, -1)

        d = np.exp(self.c[spin] * np.asarray(xl, dtype=np.float64))
        G = _f64(G)
        tau = self.p.dtau
        if direction > 0:  # D E G Einv D^{-1}
            T = apply_E(G, tau)
            T = apply_E(T.T, -tau).T
            return d[:, None] * T / d[None, :]
        T = G * d[None, :] / d[:, None]  # D^{-1} G D, then Einv (.) E
        T = apply_E(T, -tau)
        return apply_E(T.T, tau).T

    def local_slice(self, Gu, Gd, xl, u, replay=None):
        """Local update of one slice (Eqs. DetRatiolocal, UpdateLTRlocal); returns (Gu, Gd, xl, dec, ratio, sign)."""
        N = self.N
        Gu, Gd = _f64(Gu).copy(), _f64(Gd).copy()
        xl = np.ascontiguousarray(xl, dtype=np.int8).copy()
        u = _f64(u)
        rep = None if replay is None else np.ascontiguousarray(replay, dtype=np.uint8)
        dec = np.zeros(N, np.uint8)
        ratio = np.zeros(N)
        sg = np.ones(1)
        _load().or_local_slice(ctypes.byref(self.p), _d(Gu), _d(Gd), _i8(xl), _d(u), _u8(rep), _u8(dec),
                               _d(ratio), _d(sg))
        return Gu, Gd, xl, dec, ratio, sg[0]

    def delayed_slice(self, Gu, Gd, xl, u, k, strategy=2, replay=None):
        """Delayed update of one slice (Eqs. DelayRatio, DelayRgenk, FinalDelay)."""
        N = self.N
        Gu, Gd = _f64(Gu).copy(), _f64(Gd).copy()
        xl = np.ascontiguousarray(xl, dtype=np.int8).copy()
        u = _f64(u)
        rep = None if replay is None else np.ascontiguousarray(replay, dtype=np.uint8)
        dec = np.zeros(N, np.uint8)
        ratio = np.zeros(N)
        sg = np.ones(1)
        nfl = ctypes.c_int(0)
        _load().or_delayed_slice(ctypes.byref(self.p), _d(Gu), _d(Gd), _i8(xl), _d(u), int(k), int(strategy),
                                 _u8(rep), _u8(dec), _d(ratio), _d(sg), ctypes.byref(nfl))
        return Gu, Gd, xl, dec, ratio, sg[0], nfl.value

    def block_force_bias(self, G, xl, spin, s0, n):
        """Stripped force bias nbar of block [s0, s0+n) (Eq. BlkFrcBsTnew1, G form)."""
        nbar = np.zeros(n)
        xl = np.ascontiguousarray(xl, dtype=np.int8)
        _load().or_block_force_bias(ctypes.byref(self.p), _d(_f64(G)), _i8(xl), spin, s0, n, _d(nbar))
        return nbar

    def blockfb_slice(self, Gu, Gd, xl, u_prop, u_acc, nb, replay=None):
        """Block force-bias update of one slice (Sec. III.B).
        Returns (Gu, Gd, xl, xprop, lam_plus, dec[nblocks], ratio[nblocks], sign)."""
        N = self.N
        nblocks = (N + nb - 1) // nb
        Gu, Gd = _f64(Gu).copy(), _f64(Gd).copy()
        xl = np.ascontiguousarray(xl, dtype=np.int8).copy()
        rep = None if replay is None else np.ascontiguousarray(replay, dtype=np.uint8)
        xprop = np.zeros(N, np.int8)
        lamp = np.zeros(N)
        dec = np.zeros(nblocks, np.uint8)
        ratio = np.zeros(nblocks)
        sg = np.ones(1)
        _load().or_blockfb_slice(ctypes.byref(self.p), _d(Gu), _d(Gd), _i8(xl), _d(_f64(u_prop)),
                                 _d(_f64(u_acc)), int(nb), _u8(rep), _i8(xprop), _d(lamp), _u8(dec), _d(ratio),
                                 _d(sg))
        return Gu, Gd, xl, xprop, lamp, dec, ratio, sg[0]

    def energy(self, Gu, Gd):
        """Mixed-estimator energy from G by Wick's theorem (Eqs. 2DHubbard, Oxformula)."""
        return _load().or_energy(ctypes.byref(self.p), _d(self.K), _d(_f64(Gu)), _d(_f64(Gd)))

    def tform_wrap(self, UR, UL, xl, spin, direction):
        """T-form wrap (Sec. II.C): forward U_R <- B_l U_R, U_L <- U_L B_l^{-1}; backward the inverse
        moves.  T = (U_L U_R)^{-1} is unchanged.  Returns (U_R, U_L)."""
        UR, UL = _f64(UR).copy(), _f64(UL).copy()
        xl = np.ascontiguousarray(xl, dtype=np.int8)
        _load().or_tform_wrap(ctypes.byref(self.p), _d(self.E), _d(self.Einv), _i8(xl), spin, direction,
                              UR.shape[1], _d(UR), _d(UL))
        return UR, UL

    def tform_delayed_slice(self, UR, UL, T, xl, u, k, strategy=1, replay=None):
        """T-form delayed update of one slice (Eqs. DelayRatio, DelayRgenk, UpdateLTRMat, FinalDelay).
        UR, UL, T: per-spin pairs.  Returns (UR pair, T pair, xl, dec, ratio, sign, flushes)."""
        N = self.N
        URu, URd = _f64(UR[0]).copy(), _f64(UR[1]).copy()
        Tu, Td = _f64(T[0]).copy(), _f64(T[1]).copy()
        ULu, ULd = _f64(UL[0]), _f64(UL[1])
        xl = np.ascontiguousarray(xl, dtype=np.int8).copy()
        u = _f64(u)
        rep = None if replay is None else np.ascontiguousarray(replay, dtype=np.uint8)
        dec = np.zeros(N, np.uint8)
        ratio = np.zeros(N)
        sg = np.ones(1)
        nfl = ctypes.c_int(0)
        _load().or_tform_delayed_slice(ctypes.byref(self.p), _d(URu), _d(URd), _d(ULu), _d(ULd), _d(Tu), _d(Td),
                                       URu.shape[1], URd.shape[1], _i8(xl), _d(u), int(k), int(strategy), _u8(rep),
                                       _u8(dec), _d(ratio), _d(sg), ctypes.byref(nfl))
        return (URu, URd), (Tu, Td), xl, dec, ratio, sg[0], nfl.value

    def tform_blockfb_slice(self, UR, UL, T, xl, u_prop, u_acc, nb, replay=None):
        """T-form block force-bias update of one slice (Eqs. BlkFrcBsTnew1, DetRatio10, BlkFrcBsTnew2).
        Returns (UR pair, T pair, xl, xprop, lam_plus, dec[nblocks], ratio[nblocks], sign)."""
        N = self.N
        nblocks = (N + nb - 1) // nb
        URu, URd = _f64(UR[0]).copy(), _f64(UR[1]).copy()
        Tu, Td = _f64(T[0]).copy(), _f64(T[1]).copy()
        ULu, ULd = _f64(UL[0]), _f64(UL[1])
        xl = np.ascontiguousarray(xl, dtype=np.int8).copy()
        rep = None if replay is None else np.ascontiguousarray(replay, dtype=np.uint8)
        xprop = np.zeros(N, np.int8)
        lamp = np.zeros(N)
        dec = np.zeros(nblocks, np.uint8)
        ratio = np.zeros(nblocks)
        sg = np.ones(1)
        _load().or_tform_blockfb_slice(ctypes.byref(self.p), _d(URu), _d(URd), _d(ULu), _d(ULd), _d(Tu), _d(Td),
                                       URu.shape[1], URd.shape[1], _i8(xl), _d(_f64(u_prop)), _d(_f64(u_acc)),
                                       int(nb), _u8(rep), _i8(xprop), _d(lamp), _u8(dec), _d(ratio), _d(sg))
        return (URu, URd), (Tu, Td), xl, xprop, lamp, dec, ratio, sg[0]


class Walker:
    """One Markov chain driven by the oracle: fields X (M x N), G per spin, sweep position.

    The sweep follows the paper's order (Sec. II.B, Sec. IV): forward l = 1..M (wrap to l, then
    update slice l), backward l = M..1 (update slice l, then wrap down to l-1)."""

    def __init__(self, model: Model, P_up, P_dn, x):
        self.m = model
        self.P = (_f64(P_up), _f64(P_dn))
        self.x = np.ascontiguousarray(x, dtype=np.int8).copy()
        self.pos = 0
        self.G = [None, None]
        self.sign = 1.0
        self.recompute()

    def recompute(self, stab=10):
        sg = 1
        drift = []
        for s in range(2):
            G, s_, _ = self.m.green_scratch(self.x, self.P[s], s, self.pos, stab)
            if self.G[s] is not None:
                drift.append(np.linalg.norm(self.G[s] - G) / np.linalg.norm(G))
            self.G[s] = G
            sg *= s_
        self.sign = float(sg)
        return drift

    def sweep_slice(self, ell, direction, mode, u, k=32, nb=4, strategy=2, replay=None, u_acc=None):
        m, N = self.m, self.m.N
        xl = self.x[ell - 1]
        if direction > 0:
            assert self.pos == ell - 1
            self.G = [m.wrap(self.G[s], xl, s, +1) for s in range(2)]
            self.pos = ell
        else:
            assert self.pos == ell
        if mode == "local":
            Gu, Gd, xn, dec, ratio, sg = m.local_slice(self.G[0], self.G[1], xl, u[:N], replay)
            extra = {}
        elif mode == "delayed":
            Gu, Gd, xn, dec, ratio, sg, nfl = m.delayed_slice(self.G[0], self.G[1], xl, u[:N], k, strategy,
                                                              replay)
            extra = {"flushes": nfl}
        elif mode == "blockfb":
            nblocks = (N + nb - 1) // nb
            ua = u[N:N + nblocks] if u_acc is None else u_acc
            Gu, Gd, xn, xprop, lamp, dec, ratio, sg = m.blockfb_slice(self.G[0], self.G[1], xl, u[:N], ua, nb,
                                                                     replay)
            extra = {"xprop": xprop, "lam_plus": lamp}
        else:
            raise ValueError(mode)
        self.G = [Gu, Gd]
        self.x[ell - 1] = xn
        self.sign *= sg
        if direction < 0:
            self.G = [m.wrap(self.G[s], xn, s, -1) for s in range(2)]
            self.pos = ell - 1
        return dec, ratio, extra


class TWalker:
    """The paper's own walker (Sec. II.C): per spin U_R, U_L and T = (U_L U_R)^{-1}; G = 1 - U_R T U_L
    (Eq. GrFMatNew) is formed only on request.  The same sweep order as Walker; delayed (k = 1 is
    the local update, Eq. UpdateLTRlocal) and block force-bias updates.  T comes from the oracle's
    own stabilised factors at every recompute."""

    def __init__(self, model: Model, P_up, P_dn, x, stab=10):
        self.m = model
        self.P = (_f64(P_up), _f64(P_dn))
        self.x = np.ascontiguousarray(x, dtype=np.int8).copy()
        self.pos = 0
        self.UR = [None, None]
        self.UL = [None, None]
        self.T = [None, None]
        self.sign = 1.0
        self.recompute(stab)

    def recompute(self, stab=10):
        sg = 1
        for s in range(2):
            _, s_, _, UR, UL = self.m.green_scratch(self.x, self.P[s], s, self.pos, stab, want_factors=True)
            self.UR[s], self.UL[s] = UR, UL
            self.T[s] = np.linalg.inv(UL @ UR)
            sg *= s_
        self.sign = float(sg)

    def G(self, s):
        return np.eye(self.m.N) - self.UR[s] @ self.T[s] @ self.UL[s]

    def sweep_slice(self, ell, direction, mode, u, k=32, nb=4, strategy=1, replay=None, u_acc=None):
        """mode "delayed" (k = 1: the local update) or "blockfb"; uniforms as Walker.sweep_slice."""
        m, N = self.m, self.m.N
        xl = self.x[ell - 1]
        if direction > 0:
            assert self.pos == ell - 1
            for s in range(2):
                self.UR[s], self.UL[s] = m.tform_wrap(self.UR[s], self.UL[s], xl, s, +1)
            self.pos = ell
        else:
            assert self.pos == ell
        if mode == "delayed":
            UR, T, xn, dec, ratio, sg, nfl = m.tform_delayed_slice(self.UR, self.UL, self.T, xl, u[:N], k, strategy,
                                                                   replay)
            extra = {"flushes": nfl}
        elif mode == "blockfb":
            nblocks = (N + nb - 1) // nb
            ua = u[N:N + nblocks] if u_acc is None else u_acc
            UR, T, xn, xprop, lamp, dec, ratio, sg = m.tform_blockfb_slice(self.UR, self.UL, self.T, xl, u[:N], ua,
                                                                           nb, replay)
            extra = {"xprop": xprop, "lam_plus": lamp}
        else:
            raise ValueError(mode)
        self.UR, self.T = list(UR), list(T)
        self.x[ell - 1] = xn
        self.sign *= sg
        if direction < 0:
            for s in range(2):
                self.UR[s], self.UL[s] = m.tform_wrap(self.UR[s], self.UL[s], xn, s, -1)
            self.pos = ell - 1
        return dec, ratio, extra


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _vp(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


class SocModel:
    """Spin-orbit-coupled Hubbard model on the 2N x 2N complex orbital basis (Appendix A,
    Eq. 2DSocHubbard): orbitals i (spin up) and N + i (spin down).  E = exp(-dtau H0),
    Einv = exp(+dtau H0) from the closed-form 2 x 2 exponential per momentum.  hs: the
    decoupling channel, "sy" (spin-y, Eq. HSspinSyDep) or "sz" (the imaginary spin-z channel of
    Eqs. HSspinDecomp, BIOpForHubbard; with lam = 0 the attractive Hubbard model of Sec. II.B)."""

    def __init__(self, L, t, lam, U, dtau, M, hs="sy"):
        self.p = SocParams(L=L, N=L * L, t=t, lam=lam, U=U, dtau=dtau, hs=SOC_HS[hs])
        self.hs = hs
        if _load().soc_setup(ctypes.byref(self.p)) != 0:
            raise ValueError("the decoupling needs U <= 0")
        self.N = L * L
        self.M = M
        self.H0 = np.zeros((2 * self.N, 2 * self.N), np.complex128)
        _load().soc_H0(ctypes.byref(self.p), _vp(self.H0))
        self.E = self.expH(dtau)
        self.Einv = self.expH(-dtau)

    @property
    def gamma(self):
        return self.p.gamma

    def expH(self, tau):
        E = np.zeros((2 * self.N, 2 * self.N), np.complex128)
        _load().soc_expH(ctypes.byref(self.p), float(tau), _vp(E))
        return E

    def green_scratch(self, x, P, ell, stab=10):
        """G(ell) = 1 - R (L R)^{-1} L from scratch; returns (G, log|det L R|, phase of det L R)."""
        x = np.ascontiguousarray(x, dtype=np.int8)
        P = _c128(P)
        G = np.zeros((2 * self.N, 2 * self.N), np.complex128)
        la = np.zeros(1)
        ph = np.zeros(1, np.complex128)
        rc = _load().soc_green_scratch(ctypes.byref(self.p), _vp(self.E), _i8(x), self.M, _vp(P), P.shape[1], ell,
                                       stab, _vp(G), _d(la), _vp(ph))
        if rc != 0:
            raise np.linalg.LinAlgError("singular overlap")
        return G, la[0], ph[0]

    def wrap_fft(self, G, xl, direction):
        """The same wrap with exp(-+dtau H0) applied in momentum space (the paper's FFT
        propagation, Sec. II.C, for the spin-orbit-coupled H0 of Appendix A).  H0 is block-diagonal
        in the 2D Fourier basis: per momentum k the 2 x 2 block h_k = [[eps_k, conj(L_k)],
        [L_k, eps_k]] in (up, down), eps_k = -2t (cos kx + cos ky), L_k = 2 lam (sin ky - i sin kx).
        E X = F^{-1} (exp(-dtau h_k) (F X)_k) for every column of X (numpy's FFT over the site index
        of each spin block, exp by numpy's batched eigh); X E^{-1} = (E^{-1} X^+)^+ since E is
        Hermitian.  D(x) mixes each pair (i, N + i) by A(gamma x_i): a rotation (spin-y) or the phases
        diag(e^{i gamma x_i}, e^{-i gamma x_i}) (spin-z)."""
        L, N = self.p.L, self.N
        k = 2 * np.pi * np.arange(L) / L
        kx, ky = k[None, :], k[:, None]  # (ky, kx) grid, site index x + L y
        eps = -2.0 * self.p.t * (np.cos(kx) + np.cos(ky))
        Lk = 2.0 * self.p.lam * (np.sin(ky) - 1j * np.sin(kx))
        h = np.zeros((L, L, 2, 2), np.complex128)
        h[..., 0, 0] = eps
        h[..., 1, 1] = eps
        h[..., 1, 0] = Lk
        h[..., 0, 1] = np.conj(Lk)
        w, v = np.linalg.eigh(h)

        def expk(tau):
            return np.einsum("...ab,...b,...cb->...ac", v, np.exp(-tau * w), np.conj(v))

        def apply_E(X, tau):  # exp(-tau H0) X, X: 2N x m
            Xk = np.fft.fft2(X.reshape(2, L, L, -1), axes=(1, 2))
            Yk = np.einsum("yxab,byxm->ayxm", expk(tau), Xk)
            return np.fft.ifft2(Yk, axes=(1, 2)).reshape(2 * N, -1)

        th = self.p.gamma * np.asarray(xl, dtype=np.float64)
        c, s = np.cos(th), np.sin(th)

        if self.hs == "sz":
            def rot_rows(X, sgn):  # D(sgn x) X
                ph = np.exp(1j * sgn * th)[:, None]
                return np.concatenate([ph * X[:N], np.conj(ph) * X[N:]])

            def rot_cols(X, sgn):  # X D(sgn x), D diagonal
                return rot_rows(X.T, sgn).T
        else:
            def rot_rows(X, sgn):  # D(sgn x) X
                up, dn = X[:N].copy(), X[N:].copy()
                return np.concatenate([c[:, None] * up + sgn * s[:, None] * dn,
                                       -sgn * s[:, None] * up + c[:, None] * dn])

            def rot_cols(X, sgn):  # X D(sgn x)
                return rot_rows(X.T, -sgn).T  # (X D)^T = D^T X^T and A(t)^T = A(-t)

        G = _c128(G)
        tau = self.p.dtau
        if direction > 0:  # D E G Einv D^{-1}
            T = apply_E(G, tau)
            T = apply_E(T.conj().T, -tau).conj().T
            return rot_cols(rot_rows(T, +1.0), -1.0)
        T = rot_cols(rot_rows(G, -1.0), +1.0)  # D^{-1} G D, then Einv (.) E
        T = apply_E(T, -tau)
        return apply_E(T.conj().T, tau).conj().T

    def wrap(self, G, xl, direction):
        """Forward: G <- B_l G B_l^{-1}; backward: G <- B_l^{-1} G B_l, B_l = D(x_l) E."""
        G = _c128(G).copy()
        _load().soc_wrap(ctypes.byref(self.p), _vp(self.E), _vp(self.Einv),
                         _i8(np.ascontiguousarray(xl, dtype=np.int8)), _vp(G), int(direction))
        return G

    def local_slice(self, G, xl, u, replay=None):
        """Rank-2 local update of one slice (Eqs. DetRatioSOC, LocalSOC); returns (G, xl, dec, ratio)."""
        N = self.N
        G = _c128(G).copy()
        xl = np.ascontiguousarray(xl, dtype=np.int8).copy()
        rep = None if replay is None else np.ascontiguousarray(replay, dtype=np.uint8)
        dec = np.zeros(N, np.uint8)
        ratio = np.zeros(2 * N)
        _load().soc_local_slice(ctypes.byref(self.p), _vp(G), _i8(xl), _d(_f64(u)), _u8(rep), _u8(dec), _d(ratio))
        return G, xl, dec, ratio[0::2] + 1j * ratio[1::2]

    def delayed_slice(self, G, xl, u, k, replay=None):
        """Delayed update of one slice, windows of k sites; returns (G, xl, dec, ratio)."""
        N = self.N
        G = _c128(G).copy()
        xl = np.ascontiguousarray(xl, dtype=np.int8).copy()
        rep = None if replay is None else np.ascontiguousarray(replay, dtype=np.uint8)
        dec = np.zeros(N, np.uint8)
        ratio = np.zeros(2 * N)
        _load().soc_delayed_slice(ctypes.byref(self.p), _vp(G), _i8(xl), _d(_f64(u)), int(k), _u8(rep), _u8(dec),
                                  _d(ratio))
        return G, xl, dec, ratio[0::2] + 1j * ratio[1::2]

    def block_force_bias(self, G, xl, s0, n):
        """Stripped spin-flip expectations obar_i of block [s0, s0 + n)."""
        ob = np.zeros(n, np.complex128)
        _load().soc_block_force_bias(ctypes.byref(self.p), _vp(_c128(G)),
                                     _i8(np.ascontiguousarray(xl, dtype=np.int8)), s0, n, _vp(ob))
        return ob

    def blockfb_slice(self, G, xl, u_prop, u_acc, nb, replay=None):
        """Block force-bias update of one slice; returns (G, xl, xprop, lam_plus, dec, ratio)."""
        N = self.N
        nblocks = (N + nb - 1) // nb
        G = _c128(G).copy()
        xl = np.ascontiguousarray(xl, dtype=np.int8).copy()
        rep = None if replay is None else np.ascontiguousarray(replay, dtype=np.uint8)
        xprop = np.zeros(N, np.int8)
        lamp = np.zeros(N)
        dec = np.zeros(nblocks, np.uint8)
        ratio = np.zeros(2 * nblocks)
        _load().soc_blockfb_slice(ctypes.byref(self.p), _vp(G), _i8(xl), _d(_f64(u_prop)), _d(_f64(u_acc)), int(nb),
                                  _u8(rep), _i8(xprop), _d(lamp), _u8(dec), _d(ratio))
        return G, xl, xprop, lamp, dec, ratio[0::2] + 1j * ratio[1::2]

    def energy(self, G, H0=None):
        """Mixed-estimator energy with the spin-coupled Wick contraction (complex); H0 defaults to
        the model's hopping matrix."""
        r = np.zeros(2)
        H0 = self.H0 if H0 is None else _c128(H0)
        _load().soc_energy(ctypes.byref(self.p), _vp(H0), _vp(_c128(G)), _d(r))
        return complex(r[0], r[1])


    def pairing(self, G, want_k=True):
        """The pairing observables of Sec. IV from G (soc_oracle.c soc_pairing): a dict with the
        double occupancy D, the pairing correlator <Delta^2> (both complex mixed estimators), and
        with want_k the momentum occupations nk (2N: spin up, then spin down) and the raw pairing
        matrix Mk[k][k'] = <D+_k D_k'> (N x N), D+_k = c+_{k up} c+_{-k dn}."""
        N = self.N
        out = np.zeros(4)
        nk = np.zeros(2 * N, np.complex128) if want_k else None
        Mk = np.zeros((N, N), np.complex128) if want_k else None
        _load().soc_pairing(ctypes.byref(self.p), _vp(_c128(G)), _d(out), _vp(nk), _vp(Mk))
        r = {"D": complex(out[0], out[1]), "Delta2": complex(out[2], out[3])}
        if want_k:
            r["nk"], r["Mk"] = nk, Mk
        return r


class SocWalker:
    """One spin-coupled Markov chain driven by the oracle, in the same sweep order as ``Walker``."""

    def __init__(self, model: SocModel, P, x):
        self.m = model
        self.P = _c128(P)
        self.x = np.ascontiguousarray(x, dtype=np.int8).copy()
        self.pos = 0
        self.G = None
        self.recompute()

    def recompute(self, stab=10):
        G, _, _ = self.m.green_scratch(self.x, self.P, self.pos, stab)
        drift = None if self.G is None else np.linalg.norm(self.G - G) / np.linalg.norm(G)
        self.G = G
        return drift

    def sweep_slice(self, ell, direction, mode, u, k=32, nb=4, replay=None):
        m, N = self.m, self.m.N
        xl = self.x[ell - 1]
        if direction > 0:
            assert self.pos == ell - 1
            self.G = m.wrap(self.G, xl, +1)
            self.pos = ell
        else:
            assert self.pos == ell
        if mode == "local":
            G, xn, dec, ratio = m.local_slice(self.G, xl, u[:N], replay)
            extra = {}
        elif mode == "delayed":
            G, xn, dec, ratio = m.delayed_slice(self.G, xl, u[:N], k, replay)
            extra = {}
        elif mode == "blockfb":
            nblocks = (N + nb - 1) // nb
            G, xn, xprop, lamp, dec, ratio = m.blockfb_slice(self.G, xl, u[:N], u[N:N + nblocks], nb, replay)
            extra = {"xprop": xprop, "lam_plus": lamp}
        else:
            raise ValueError(mode)
        self.G = G
        self.x[ell - 1] = xn
        if direction < 0:
            self.G = m.wrap(self.G, xn, -1)
            self.pos = ell - 1
        return dec, ratio, extra
