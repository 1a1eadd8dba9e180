"""Plain CPU oracle for the over-relaxed diffusive integer lattice gas.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this package.  It
shares no code with the CUDA library (``paper_2203_01380_gb300``) and neither
imports the other.

The integer work (Philox4x32-10, binomial pmf and alias tables, Poisson tables, the time step,
the initial state and the integer sums) lives in ``ilg_oracle.c``, compiled with
plain ``gcc`` into ``liboracle.so`` beside it.  The floating-point projections
(measured amplitude A^LG of Sec. V and the structure factor) are evaluated here
exactly in rational arithmetic from the double-precision sines and cosines, and
rounded once at the end.

Pins: every function here is checked in ``tests/test_oracle_*.py`` against
something other than itself (cuRAND's host Philox generator, exact rational
CDFs, exact enumeration of the collision law, the paper's moment-space
collision and diffusion constant, exact invariants).  Parity unpinned: the bit
pattern of Seekins' own sampler, which the paper does not give; the oracle is
pinned to the distribution the paper states instead.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ilg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

NMAX = 63          # largest trial count of one alias-table row (chunks of 63 trials)
ALIAS_COLS = 64    # columns per alias row: a draw u takes column u >> 26
POISSON_KMAX = 4096
D1Q3, D2Q5, D2Q9 = 1, 2, 3
TWO32 = 1 << 32


def build(force: bool = False) -> str:
    """Compile ilg_oracle.c with gcc into liboracle.so (no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
             "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _StepParams(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int32), ("Lx", ctypes.c_uint32), ("Ly", ctypes.c_uint32),
        ("flip", ctypes.c_int32), ("P_omega", ctypes.c_uint64), ("P_rest", ctypes.c_uint64),
        ("seed", ctypes.c_uint64), ("replica", ctypes.c_uint32),
        ("thr_omega", ctypes.c_void_p), ("alias_omega", ctypes.c_void_p),
        ("thr_rest", ctypes.c_void_p), ("alias_rest", ctypes.c_void_p),
        ("sampler", ctypes.c_int32),
        ("P_axis", ctypes.c_uint64), ("thr_axis", ctypes.c_void_p), ("alias_axis", ctypes.c_void_p),
    ]


class _InitParams(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int32), ("Lx", ctypes.c_uint32), ("Ly", ctypes.c_uint32),
        ("n0", ctypes.c_double), ("amp", ctypes.c_double),
        ("mode_mx", ctypes.c_int32), ("mode_my", ctypes.c_int32),
        ("init_weighted", ctypes.c_int32), ("theta", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("replica", ctypes.c_uint32),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
        u16p = np.ctypeslib.ndpointer(np.uint16, flags="C_CONTIGUOUS")
        i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
        L.oracle_philox.argtypes = [u32p, u32p, u32p]
        L.oracle_philox.restype = None
        L.oracle_binomial_table.argtypes = [ctypes.c_uint64, ctypes.c_uint32, u32p]
        L.oracle_binomial_table.restype = None
        u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
        L.oracle_alias_table.argtypes = [ctypes.c_uint64, ctypes.c_uint32, u32p, u8p]
        L.oracle_alias_table.restype = None
        L.oracle_poisson_table.argtypes = [ctypes.c_double, u32p, ctypes.c_uint32]
        L.oracle_poisson_table.restype = ctypes.c_uint32
        L.oracle_step_region.argtypes = [ctypes.POINTER(_StepParams), u16p, u16p, ctypes.c_uint32,
                                         ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                         ctypes.c_int, ctypes.c_uint32]
        L.oracle_step_region.restype = ctypes.c_int
        L.oracle_init_region.argtypes = [ctypes.POINTER(_InitParams), u16p, ctypes.c_uint32,
                                         ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]
        L.oracle_init_region.restype = ctypes.c_int
        L.oracle_init_lambda.argtypes = [ctypes.POINTER(_InitParams), ctypes.c_uint32,
                                         ctypes.c_uint32, ctypes.c_int]
        L.oracle_init_lambda.restype = ctypes.c_double
        L.oracle_sums.argtypes = [ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint32, u16p, i64p,
                                  i64p, ctypes.POINTER(ctypes.c_uint64)]
        L.oracle_sums.restype = None
        L.oracle_collide_many.argtypes = [ctypes.POINTER(_StepParams), u32p, ctypes.c_uint32,
                                          ctypes.c_uint32, ctypes.c_uint32, u32p]
        L.oracle_collide_many.restype = None
        L.oracle_particle_bounds.argtypes = [ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                             np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")]
        L.oracle_particle_bounds.restype = None
        _lib = L
    return _lib


# --------------------------------------------------------------------------
# parameters (Sec. III: omega^j = 2 - omega*; Sec. II: weights and theta)
# --------------------------------------------------------------------------

def num_vel(lattice: int) -> int:
    return {D1Q3: 3, D2Q5: 5, D2Q9: 9}[lattice]


def quantise(p: float) -> int:
    """Probability -> integer P with p ~ P / 2^32: floor(p * 2^32 + 1/2), clamped."""
    v = math.floor(p * 4294967296.0 + 0.5)
    return int(min(max(v, 0), TWO32))


def weights(lattice: int, theta: float):
    """w_i in storage order (rest first); theta = sum_i w_i v_{i,x}^2 per axis."""
    if lattice == D1Q3:
        return [1.0 - theta, theta / 2.0, theta / 2.0]
    if lattice == D2Q9:
        # products of the D1Q3 weights in x and y: rest, four axis, four diagonal
        wa, wd = (theta * (1.0 - theta)) / 2.0, (theta * theta) / 4.0
        return [(1.0 - theta) * (1.0 - theta)] + [wa] * 4 + [wd] * 4
    return [1.0 - 2.0 * theta, theta / 2.0, theta / 2.0, theta / 2.0, theta / 2.0]


def axis_share(theta: float) -> float:
    """D2Q9: probability that a moving particle takes an axis velocity,
    4 w_axis / (1 - w_0), with the weights above."""
    w = weights(D2Q9, theta)
    return (4.0 * w[1]) / (1.0 - w[0])


def split_omega(omega_eff: float):
    """omega_eff -> (flip, omega*): above 1 the flip is on and omega* = 2 - omega_eff."""
    if omega_eff > 1.0:
        return 1, 2.0 - omega_eff
    return 0, omega_eff


def binomial_table(P: int, nmax: int = NMAX) -> np.ndarray:
    T = np.zeros(nmax * (nmax + 1) // 2, dtype=np.uint32)
    lib().oracle_binomial_table(ctypes.c_uint64(P), nmax, T)
    return T


ALIAS_ENTRIES = (NMAX + 1) * ALIAS_COLS   # rows n = 0..NMAX, 64 columns each


def alias_table(P: int, nmax: int = NMAX):
    """(thr, alias) of the alias tables of Binomial(n, P/2^32), n = 0..nmax <= 63; row n
    at offset 64 n, column j of row n covering the draws j 2^26 <= u < (j+1) 2^26."""
    if not 0 <= nmax < ALIAS_COLS:
        raise ValueError("alias rows hold at most 64 outcomes")
    n_ent = (nmax + 1) * ALIAS_COLS
    thr = np.zeros(n_ent, dtype=np.uint32)
    al = np.zeros(n_ent, dtype=np.uint8)
    lib().oracle_alias_table(ctypes.c_uint64(P), nmax, thr, al)
    return thr, al


def poisson_table(lam: float) -> np.ndarray:
    T = np.zeros(POISSON_KMAX, dtype=np.uint32)
    K = lib().oracle_poisson_table(lam, T, POISSON_KMAX)
    if K == 0:
        raise ValueError("Poisson table exceeds the cap")
    return T[:K].copy()


def particle_bounds(lattice: int, P_omega: int, P_rest: int, P_axis: int = 0) -> list:
    """Boundaries B_0..B_Q of the particle sampler (one word per particle)."""
    B = np.zeros(10, dtype=np.uint64)
    lib().oracle_particle_bounds(lattice, P_omega, P_rest, P_axis, B)
    return [int(b) for b in B[:num_vel(lattice) + 1]]


def philox(ctr, key) -> np.ndarray:
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox(np.asarray(ctr, dtype=np.uint32), np.asarray(key, dtype=np.uint32), out)
    return out


class Lattice:
    """Parameters of one lattice, as the library's ilg_params carries them."""

    def __init__(self, lattice, Lx, Ly=1, n0=10.0, amp=0.0, mode_mx=0, mode_my=0,
                 init_weighted=0, omega_eff=1.0, theta=1.0 / 3.0, seed=0, replica=0, sampler=0):
        self.lattice, self.Lx, self.Ly = lattice, int(Lx), int(Ly if lattice != D1Q3 else 1)
        self.sampler = int(sampler)   # 0: binomial draws through alias tables; 1: one word per particle
        self.n0, self.amp, self.mode_mx, self.mode_my = float(n0), float(amp), mode_mx, mode_my
        self.init_weighted, self.omega_eff, self.theta = init_weighted, float(omega_eff), float(theta)
        self.seed, self.replica = int(seed), int(replica)
        self.Q = num_vel(lattice)
        self.flip, self.omega_star = split_omega(self.omega_eff)
        self.w = weights(lattice, self.theta)
        self.P_omega = quantise(self.omega_star)
        self.P_rest = quantise(self.w[0])
        none = (np.zeros(1, np.uint32), np.zeros(1, np.uint8))
        self._A_omega = alias_table(self.P_omega) if 0 < self.P_omega < TWO32 else none
        self._A_rest = alias_table(self.P_rest) if 0 < self.P_rest < TWO32 else none
        self.P_axis = quantise(axis_share(self.theta)) if lattice == D2Q9 else 0
        self._A_axis = alias_table(self.P_axis) if 0 < self.P_axis < TWO32 else none

    def _sp(self):
        return _StepParams(self.lattice, self.Lx, self.Ly, self.flip, self.P_omega, self.P_rest,
                           self.seed, self.replica, self._A_omega[0].ctypes.data, self._A_omega[1].ctypes.data,
                           self._A_rest[0].ctypes.data, self._A_rest[1].ctypes.data, self.sampler,
                           self.P_axis, self._A_axis[0].ctypes.data, self._A_axis[1].ctypes.data)

    def _ip(self):
        return _InitParams(self.lattice, self.Lx, self.Ly, self.n0, self.amp, self.mode_mx,
                           self.mode_my, self.init_weighted, self.theta, self.seed, self.replica)

    @property
    def shape(self):
        return (self.Q, self.Ly, self.Lx)

    # ---- initial state ---------------------------------------------------
    def init(self) -> np.ndarray:
        return self.init_region(0, 0, self.Lx, self.Ly)

    def init_region(self, x0, y0, w, h) -> np.ndarray:
        out = np.zeros((self.Q, h, w), dtype=np.uint16)
        if lib().oracle_init_region(ctypes.byref(self._ip()), out.reshape(-1), x0, y0, w, h) != 0:
            raise ValueError("invalid initial mean")
        return out

    def init_lambda(self, gx, gy, v) -> float:
        return lib().oracle_init_lambda(ctypes.byref(self._ip()), gx, gy, v)

    # ---- time step --------------------------------------------------------
    def step(self, state: np.ndarray, t: int) -> np.ndarray:
        state = np.ascontiguousarray(state, dtype=np.uint16)
        out = np.zeros_like(state)
        sp = self._sp()
        rc = lib().oracle_step_region(ctypes.byref(sp), state.reshape(-1), out.reshape(-1), 0, 0,
                                      self.Lx, self.Ly, 1, t)
        if rc != 0:
            raise OverflowError(f"occupation above 65535 in step {t}")
        return out

    def run(self, state: np.ndarray, t0: int, steps: int) -> np.ndarray:
        for s in range(steps):
            state = self.step(state, t0 + s)
        return state

    def step_region(self, patch: np.ndarray, x0: int, y0: int, t: int) -> np.ndarray:
        """One step of a patch at global (x0, y0); cells fed from outside are invalid."""
        patch = np.ascontiguousarray(patch, dtype=np.uint16)
        _, h, w = patch.shape
        out = np.zeros_like(patch)
        sp = self._sp()
        rc = lib().oracle_step_region(ctypes.byref(sp), patch.reshape(-1), out.reshape(-1),
                                      x0 % self.Lx, y0 % self.Ly, w, h, 0, t)
        if rc != 0:
            raise OverflowError(f"occupation above 65535 in step {t}")
        return out

    def window(self, x0, y0, w, h, t_end, t0=0, initial=None):
        """State of the w x h window at (x0, y0) after t_end - t0 steps from the
        oracle's own initial state (light cone: a (w+2s) x (h+2s) patch)."""
        s = t_end - t0
        pad_y = s if self.lattice != D1Q3 else 0
        px, py = x0 - s, y0 - pad_y
        pw, ph = w + 2 * s, h + 2 * pad_y
        if initial is None:
            patch = self.init_region(px % self.Lx, py % self.Ly, pw, ph)
        else:
            patch = initial
        for k in range(s):
            patch = self.step_region(patch, px + k, py + (k if self.lattice != D1Q3 else 0), t0 + k)
            patch = patch[:, (1 if self.lattice != D1Q3 else 0):patch.shape[1] - (1 if self.lattice != D1Q3 else 0), 1:-1]
            patch = np.ascontiguousarray(patch)
        return patch

    # ---- collision alone ---------------------------------------------------
    def collide_many(self, m, t, node0, count) -> np.ndarray:
        m = np.asarray(m, dtype=np.uint32)
        out = np.zeros((count, self.Q), dtype=np.uint32)
        sp = self._sp()
        lib().oracle_collide_many(ctypes.byref(sp), m, t, node0, count, out.reshape(-1))
        return out

    # ---- observables --------------------------------------------------------
    def sums(self, state):
        state = np.ascontiguousarray(state, dtype=np.uint16)
        col = np.zeros(self.Lx, dtype=np.int64)
        row = np.zeros(self.Ly, dtype=np.int64)
        M = ctypes.c_uint64()
        lib().oracle_sums(self.lattice, self.Lx, self.Ly, state.reshape(-1), col, row, ctypes.byref(M))
        return int(M.value), col, row

    def observables(self, state, modes):
        """mass, column sums, and per axis mode (mx, my): exact (Re, Im), A^LG, S(k)."""
        M, col, row = self.sums(state)
        res = []
        for (mx, my) in modes:
            if my == 0:
                re, im, scale = project_exact(col, self.Lx, mx, M)
            else:
                re, im, scale = project_exact(row, self.Ly, my, M)
            K = self.Lx * self.Ly
            res.append(dict(re=re, im=im, amp=im / (K / 2.0), Sk=(re * re + im * im) / K, scale=scale))
        return M, col, row, res


def trig(r: int, L: int):
    """cos and sin of 2 pi r / L in double precision (host libm)."""
    ph = (6.283185307179586 * float(r)) / float(L)
    return math.cos(ph), math.sin(ph)


def project_exact(sums: np.ndarray, L: int, m: int, M: int):
    """Projections of Sec. V's measured profile on mode m, with D(x) = L*sums[x] - M:
    re = sum_x cos(2 pi r / L) D(x) / L and im = sum_x sin(2 pi r / L) D(x) / L,
    r = (m x) mod L, evaluated exactly from the double cosines and sines and rounded
    once.  Returns (re, im, scale) where scale = sum_x |D(x)| / L bounds the
    condition of both sums."""
    mm = m % L
    re = Fraction(0)
    im = Fraction(0)
    scale = 0
    for x in range(L):
        r = (mm * x) % L
        c, s = trig(r, L)
        d = L * int(sums[x]) - M
        re += Fraction(c) * d
        im += Fraction(s) * d
        scale += abs(d)
    return float(re / L), float(im / L), scale / L
