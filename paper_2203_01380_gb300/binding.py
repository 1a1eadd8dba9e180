"""ctypes binding of libilg.so (argument marshalling only; every step runs in the
library's CUDA kernels).  Importing this module fails loudly when the library
has not been built: there is no CPU fallback.

Names follow ``include/ilg.h``; see that header for the meaning of every
argument, the layouts and the error behaviour.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libilg.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()'). "
        "The lattice-gas path has no CPU fallback.")

_lib = ctypes.CDLL(LIB_PATH)

ILG_OK, ILG_E_INVALID, ILG_E_OOM, ILG_E_OVERFLOW, ILG_E_CUDA, ILG_E_TIMEOUT, ILG_E_STATE = range(7)
D1Q3, D2Q5, D2Q9 = 1, 2, 3
NUM_VEL = {D1Q3: 3, D2Q5: 5, D2Q9: 9}
STATUS_NAMES = {0: "ILG_OK", 1: "ILG_E_INVALID", 2: "ILG_E_OOM", 3: "ILG_E_OVERFLOW", 4: "ILG_E_CUDA",
                5: "ILG_E_TIMEOUT", 6: "ILG_E_STATE"}


class IlgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int32), ("Lx", ctypes.c_uint32), ("Ly", ctypes.c_uint32),
        ("mode_mx", ctypes.c_int32), ("mode_my", ctypes.c_int32), ("init_weighted", ctypes.c_int32),
        ("n0", ctypes.c_double), ("amp", ctypes.c_double), ("omega_eff", ctypes.c_double),
        ("theta", ctypes.c_double), ("seed", ctypes.c_uint64), ("replica", ctypes.c_uint32),
        ("sampler", ctypes.c_uint32),
    ]


_vp = ctypes.c_void_p
_u16p = np.ctypeslib.ndpointer(np.uint16, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")

_lib.ilg_last_error.argtypes = [_vp]
_lib.ilg_last_error.restype = ctypes.c_char_p
_lib.ilg_create.argtypes = [ctypes.POINTER(Params), _vp, ctypes.POINTER(_vp)]
_lib.ilg_destroy.argtypes = [_vp]
_lib.ilg_init.argtypes = [_vp]
_lib.ilg_set_state.argtypes = [_vp, _vp, ctypes.c_size_t, ctypes.c_uint64]
_lib.ilg_set_state_device.argtypes = [_vp, _vp, ctypes.c_size_t, ctypes.c_uint64]
_lib.ilg_get_state.argtypes = [_vp, _vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_uint64)]
_lib.ilg_get_state_device.argtypes = [_vp, _vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_uint64)]
_lib.ilg_step.argtypes = [_vp, ctypes.c_uint32]
_lib.ilg_set_temporal_blocking.argtypes = [_vp, ctypes.c_uint32]
_lib.ilg_observables.argtypes = [_vp, _vp, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64),
                                 ctypes.POINTER(ctypes.c_uint64), _vp, _vp, _vp, _vp, _vp, _vp]
_lib.ilg_observables_noalloc.argtypes = [ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint32, _vp, _vp,
                                         ctypes.c_uint32, _vp, ctypes.POINTER(ctypes.c_uint64), _vp, _vp, _vp,
                                         _vp]
_lib.ilg_batch_create.argtypes = [_vp, ctypes.c_uint32, _vp, ctypes.POINTER(_vp)]
_lib.ilg_batch_destroy.argtypes = [_vp]
_lib.ilg_batch_last_error.argtypes = [_vp]
_lib.ilg_batch_last_error.restype = ctypes.c_char_p
_lib.ilg_batch_init.argtypes = [_vp]
_lib.ilg_batch_set_state.argtypes = [_vp, ctypes.c_uint32, _vp, ctypes.c_size_t, ctypes.c_uint64]
_lib.ilg_batch_get_state.argtypes = [_vp, ctypes.c_uint32, _vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_uint64)]
_lib.ilg_batch_run.argtypes = [_vp, ctypes.c_uint32, ctypes.c_int32, _vp]
_lib.ilg_batch_run_record.argtypes = [_vp, ctypes.c_uint32, ctypes.c_int32, _vp, _vp]
_lib.ilg_batch_observables.argtypes = [_vp, ctypes.c_int32, _vp, _vp]
_lib.ilg_batch_ensemble.argtypes = [_vp, ctypes.c_uint32, ctypes.c_int32, _vp, _vp]
class Tuning(ctypes.Structure):
    _fields_ = [("choice", ctypes.c_uint32), ("tb_depth", ctypes.c_uint32), ("threads", ctypes.c_uint32),
                ("n", ctypes.c_uint32), ("ms_per_step", ctypes.c_double * 8)]


CONTEXT_CANDIDATES = ("vec8", "vec4", "node", "tb2", "tb4", "seg8", "warpv8", "warpv4")
BATCH_CANDIDATES = ("threads256", "threads512", "threads1024")


def _tuning_dict(t: Tuning, names) -> dict:
    return dict(choice=names[t.choice], tb_depth=int(t.tb_depth), threads=int(t.threads),
                ms_per_step={names[k]: (float(t.ms_per_step[k]) if t.ms_per_step[k] >= 0 else None)
                             for k in range(t.n)})


_lib.ilg_autotune.argtypes = [_vp, ctypes.c_uint32, ctypes.POINTER(Tuning)]
_lib.ilg_autotune.restype = ctypes.c_int
_lib.ilg_set_step_kernel.argtypes = [_vp, ctypes.c_int32]
_lib.ilg_set_step_kernel.restype = ctypes.c_int
_lib.ilg_batch_autotune.argtypes = [_vp, ctypes.c_uint32, ctypes.POINTER(Tuning)]
_lib.ilg_batch_autotune.restype = ctypes.c_int


class Result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int32), ("reserved", ctypes.c_uint32),
                ("t", ctypes.c_uint64), ("mass", ctypes.c_uint64), ("amp", ctypes.c_double), ("Sk", ctypes.c_double),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


_lib.ilg_server_create.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, _vp,
                                   ctypes.POINTER(_vp)]
_lib.ilg_server_submit.argtypes = [_vp, ctypes.c_uint64, ctypes.POINTER(Params), ctypes.c_uint32, _vp]
_lib.ilg_server_poll.argtypes = [_vp, ctypes.POINTER(Result), ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32)]
_lib.ilg_server_wait_idle.argtypes = [_vp, ctypes.c_double]
_lib.ilg_server_stats.argtypes = [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_uint32)]
_lib.ilg_server_destroy.argtypes = [_vp]
_lib.ilg_server_set_policy.argtypes = [_vp, ctypes.c_int32]
_lib.ilg_server_last_error.argtypes = [_vp]
_lib.ilg_server_last_error.restype = ctypes.c_char_p
_lib.ilg_philox.argtypes = [_u32p, ctypes.c_uint64, _u32p, ctypes.c_size_t, _vp]
_lib.ilg_binomial_table.argtypes = [ctypes.c_uint64, _u32p]
_lib.ilg_alias_table.argtypes = [ctypes.c_uint64, _u32p, _u32p]
_lib.ilg_poisson_table.argtypes = [ctypes.c_double, _u32p, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32)]
_lib.ilg_int_peak.argtypes = [ctypes.c_int32, ctypes.c_double, _vp, ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_double)]
for _f in ("ilg_set_temporal_blocking", "ilg_create", "ilg_destroy", "ilg_init", "ilg_set_state", "ilg_set_state_device", "ilg_get_state",
           "ilg_get_state_device", "ilg_step", "ilg_observables", "ilg_philox", "ilg_binomial_table",
           "ilg_alias_table", "ilg_poisson_table", "ilg_int_peak", "ilg_observables_noalloc", "ilg_batch_create", "ilg_batch_destroy",
           "ilg_batch_init", "ilg_batch_set_state", "ilg_batch_get_state", "ilg_batch_run", "ilg_batch_run_record",
           "ilg_batch_observables",
           "ilg_batch_ensemble",
           "ilg_server_create", "ilg_server_submit", "ilg_server_poll", "ilg_server_wait_idle", "ilg_server_stats",
           "ilg_server_destroy", "ilg_server_set_policy"):
    getattr(_lib, _f).restype = ctypes.c_int


def lib():
    return _lib


def stream_handle(stream) -> int:
    """cudaStream_t as an integer: None/0 -> legacy default stream; objects with
    a ``cuda_stream`` attribute (e.g. torch.cuda.Stream) give theirs."""
    if stream is None:
        return 0
    if hasattr(stream, "cuda_stream"):
        return int(stream.cuda_stream)
    return int(stream)


def _check(status: int, ctx=None):
    if status != ILG_OK:
        msg = _lib.ilg_last_error(ctx).decode(errors="replace")
        raise IlgError(status, msg)


SAMPLER_BINOMIAL, SAMPLER_PARTICLE = 0, 1


def make_params(lattice, Lx, Ly=1, n0=10.0, amp=0.0, mode_mx=0, mode_my=0, init_weighted=0,
                omega_eff=1.0, theta=1.0 / 3.0, seed=0, replica=0, sampler=0, **_ignored) -> Params:
    return Params(int(lattice), int(Lx), int(Ly if lattice != D1Q3 else 1), int(mode_mx), int(mode_my),
                  int(init_weighted), float(n0), float(amp), float(omega_eff), float(theta), int(seed),
                  int(replica), int(sampler))


class Lattice:
    """One lattice context (ilg_create ... ilg_destroy)."""

    def __init__(self, lattice, Lx, Ly=1, stream=None, **kw):
        self.params = make_params(lattice, Lx, Ly, **kw)
        self.Q = NUM_VEL[lattice]
        self.Lx, self.Ly = self.params.Lx, self.params.Ly
        self.stream = stream_handle(stream)
        h = _vp()
        _check(_lib.ilg_create(ctypes.byref(self.params), _vp(self.stream), ctypes.byref(h)), None)
        self._h = h

    @property
    def shape(self):
        return (self.Q, self.Ly, self.Lx)

    @property
    def size(self):
        return self.Q * self.Ly * self.Lx

    def close(self):
        if getattr(self, "_h", None):
            _lib.ilg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def init(self):
        _check(_lib.ilg_init(self._h), self._h)

    def set_state(self, state: np.ndarray, t: int = 0):
        s = np.ascontiguousarray(state, dtype=np.uint16)
        if s.size != self.size:
            raise ValueError("state has the wrong size")
        _check(_lib.ilg_set_state(self._h, s.ctypes.data, s.size, int(t)), self._h)

    def set_state_device(self, ptr: int, n: int, t: int = 0):
        _check(_lib.ilg_set_state_device(self._h, _vp(ptr), n, int(t)), self._h)

    def get_state(self, out: np.ndarray | None = None):
        if out is None:
            out = np.empty(self.shape, dtype=np.uint16)
        t = ctypes.c_uint64()
        _check(_lib.ilg_get_state(self._h, out.ctypes.data, out.size, ctypes.byref(t)), self._h)
        return out, int(t.value)

    def get_state_device(self, ptr: int, n: int) -> int:
        t = ctypes.c_uint64()
        _check(_lib.ilg_get_state_device(self._h, _vp(ptr), n, ctypes.byref(t)), self._h)
        return int(t.value)

    def step(self, T: int):
        _check(_lib.ilg_step(self._h, int(T)), self._h)

    def autotune(self, trial_steps: int = 20) -> dict:
        """ilg_autotune: time the launch shapes on a copy of the state, keep the fastest."""
        t = Tuning()
        _check(_lib.ilg_autotune(self._h, int(trial_steps), ctypes.byref(t)), self._h)
        return _tuning_dict(t, CONTEXT_CANDIDATES)

    def set_step_kernel(self, candidate: int):
        """ilg_set_step_kernel: 0 8-node vectors, 1 4-node vectors, 2 node-parallel, 5 warp
        segments of 8-node vectors, 6 / 7 the shared-memory-staged warp kernel with 8 / 4
        nodes per lane, -1 default."""
        _check(_lib.ilg_set_step_kernel(self._h, int(candidate)), self._h)

    def set_temporal_blocking(self, depth: int):
        _check(_lib.ilg_set_temporal_blocking(self._h, int(depth)), self._h)

    def observables(self, modes=(), col_sums=False, row_sums=False):
        modes = np.ascontiguousarray(np.asarray(modes, dtype=np.int32).reshape(-1, 2))
        n = len(modes)
        re, im, amp, Sk = (np.zeros(n) for _ in range(4))
        col = np.zeros(self.Lx, dtype=np.int64) if col_sums else None
        row = np.zeros(self.Ly, dtype=np.int64) if row_sums else None
        t = ctypes.c_uint64()
        M = ctypes.c_uint64()
        _check(_lib.ilg_observables(self._h, modes.ctypes.data if n else None, n, ctypes.byref(t), ctypes.byref(M),
                                    re.ctypes.data, im.ctypes.data, amp.ctypes.data, Sk.ctypes.data,
                                    col.ctypes.data if col is not None else None,
                                    row.ctypes.data if row is not None else None), self._h)
        return dict(t=int(t.value), mass=int(M.value), re=re, im=im, amp=amp, Sk=Sk, col=col, row=row)


class Batch:
    """Batched D1Q3 rings (ilg_batch_*); replicas: list of parameter dicts."""

    def __init__(self, replicas, stream=None):
        self.params = (Params * len(replicas))(*[make_params(**r) for r in replicas])
        self.n = len(replicas)
        self.L = [int(p.Lx) for p in self.params]
        h = _vp()
        st = _lib.ilg_batch_create(self.params, self.n, _vp(stream_handle(stream)), ctypes.byref(h))
        if st != ILG_OK:
            raise IlgError(st, _lib.ilg_batch_last_error(None).decode(errors="replace"))
        self._h = h

    def _check(self, st):
        if st != ILG_OK:
            raise IlgError(st, _lib.ilg_batch_last_error(self._h).decode(errors="replace"))

    def close(self):
        if getattr(self, "_h", None):
            _lib.ilg_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def init(self):
        self._check(_lib.ilg_batch_init(self._h))

    def set_state(self, i, state, t=0):
        s = np.ascontiguousarray(state, dtype=np.uint16)
        self._check(_lib.ilg_batch_set_state(self._h, i, s.ctypes.data, s.size, int(t)))

    def get_state(self, i):
        out = np.empty((3, 1, self.L[i]), dtype=np.uint16)
        t = ctypes.c_uint64()
        self._check(_lib.ilg_batch_get_state(self._h, i, out.ctypes.data, out.size, ctypes.byref(t)))
        return out, int(t.value)

    def run(self, T, record_mode=None):
        rec = np.zeros((self.n, T)) if record_mode is not None else None
        self._check(_lib.ilg_batch_run(self._h, int(T), int(record_mode or 0),
                                       rec.ctypes.data if rec is not None else None))
        return rec

    def run_record(self, T, record_mode=1):
        """ilg_batch_run_record: T steps with the amplitude of record_mode and the state of
        every ring after every step; returns (amp (n, T), [per ring (T, 3, 1, L) states])."""
        amp = np.zeros((self.n, T))
        states = np.zeros(T * 3 * sum(self.L), dtype=np.uint16)
        self._check(_lib.ilg_batch_run_record(self._h, int(T), int(record_mode), amp.ctypes.data, states.ctypes.data))
        out, off = [], 0
        for L in self.L:
            out.append(states[off:off + T * 3 * L].reshape(T, 3, 1, L))
            off += T * 3 * L
        return amp, out

    def observables(self, mode=1):
        mass = np.zeros(self.n, dtype=np.uint64)
        amp = np.zeros(self.n)
        self._check(_lib.ilg_batch_observables(self._h, int(mode), mass.ctypes.data, amp.ctypes.data))
        return mass, amp

    ENSEMBLE_ROWS = ("mean_re", "mean_im", "var_re", "var_im", "cov_re", "cov_im")

    def autotune(self, trial_steps: int = 50) -> dict:
        """ilg_batch_autotune: time the block shapes on copies of the rings, keep the fastest."""
        t = Tuning()
        self._check(_lib.ilg_batch_autotune(self._h, int(trial_steps), ctypes.byref(t)))
        return _tuning_dict(t, BATCH_CANDIDATES)

    def ensemble(self, T, mode=1, record=False):
        """T steps with the ensemble statistics of mode `mode` at t = 0..T (dict of
        arrays named as ENSEMBLE_ROWS) and, optionally, the per-ring record
        (n, T + 1, 2) of (re, im)."""
        stats = np.zeros((6, T + 1))
        rec = np.zeros((self.n, T + 1, 2)) if record else None
        self._check(_lib.ilg_batch_ensemble(self._h, int(T), int(mode), stats.ctypes.data,
                                            rec.ctypes.data if rec is not None else None))
        out = dict(zip(self.ENSEMBLE_ROWS, stats))
        if record:
            out["record"] = rec
        return out


class Server:
    """Serving loop for D2Q5 requests (ilg_server_*)."""

    def __init__(self, seed, hbm_bytes, max_slots=256, quantum=32, stream=None):
        h = _vp()
        st = _lib.ilg_server_create(int(seed), int(hbm_bytes), int(max_slots), int(quantum),
                                    _vp(stream_handle(stream)), ctypes.byref(h))
        if st != ILG_OK:
            raise IlgError(st, _lib.ilg_server_last_error(None).decode(errors="replace"))
        self._h = h
        self._states = {}   # id -> host buffer receiving the final state

    def _check(self, st):
        if st != ILG_OK:
            raise IlgError(st, _lib.ilg_server_last_error(self._h).decode(errors="replace"))

    def set_policy(self, smallest_first: bool):
        self._check(_lib.ilg_server_set_policy(self._h, 1 if smallest_first else 0))

    def submit(self, rid, steps, want_state=False, **params):
        p = make_params(**params)
        buf = None
        if want_state:
            buf = np.zeros((5, p.Ly, p.Lx), dtype=np.uint16)
            self._states[rid] = buf
        self._check(_lib.ilg_server_submit(self._h, int(rid), ctypes.byref(p), int(steps),
                                           buf.ctypes.data if buf is not None else None))

    def poll(self, cap=1024):
        out = (Result * cap)()
        n = ctypes.c_uint32()
        self._check(_lib.ilg_server_poll(self._h, out, cap, ctypes.byref(n)))
        res = []
        for r in out[:n.value]:
            d = {k: getattr(r, k) for k, _ in Result._fields_ if k != "reserved"}
            d["state"] = self._states.pop(r.id, None)
            res.append(d)
        return res

    def wait_idle(self, timeout_s=600.0):
        self._check(_lib.ilg_server_wait_idle(self._h, float(timeout_s)))

    def stats(self):
        b, nu, pk = ctypes.c_double(), ctypes.c_double(), ctypes.c_uint32()
        self._check(_lib.ilg_server_stats(self._h, ctypes.byref(b), ctypes.byref(nu), ctypes.byref(pk)))
        return dict(busy_s=b.value, node_updates=nu.value, peak_resident=pk.value)

    def close(self):
        if getattr(self, "_h", None):
            _lib.ilg_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class LBParams(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int32), ("Lx", ctypes.c_uint32), ("Ly", ctypes.c_uint32),
        ("mode_mx", ctypes.c_int32), ("mode_my", ctypes.c_int32), ("init_weighted", ctypes.c_int32),
        ("n0", ctypes.c_double), ("amp", ctypes.c_double), ("omega_j", ctypes.c_double),
        ("omega", ctypes.c_double), ("theta", ctypes.c_double),
    ]


_lib.ilg_lb_create.argtypes = [ctypes.POINTER(LBParams), _vp, ctypes.POINTER(_vp)]
_lib.ilg_lb_destroy.argtypes = [_vp]
_lib.ilg_lb_last_error.argtypes = [_vp]
_lib.ilg_lb_last_error.restype = ctypes.c_char_p
_lib.ilg_lb_init.argtypes = [_vp]
_lib.ilg_lb_set_state.argtypes = [_vp, _vp, ctypes.c_size_t, ctypes.c_uint64]
_lib.ilg_lb_get_state.argtypes = [_vp, _vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_uint64)]
_lib.ilg_lb_step.argtypes = [_vp, ctypes.c_uint32]
_lib.ilg_lb_observables.argtypes = [_vp, _vp, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64),
                                    ctypes.POINTER(ctypes.c_double), _vp, _vp, _vp]
for _f in ("ilg_lb_create", "ilg_lb_destroy", "ilg_lb_init", "ilg_lb_set_state", "ilg_lb_get_state", "ilg_lb_step",
           "ilg_lb_observables"):
    getattr(_lib, _f).restype = ctypes.c_int


_lib.ilg_lb_rates.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
_lib.ilg_lb_rates.restype = ctypes.c_int


def lb_rates(omega_eff: float):
    """ilg_lb_rates: (omega_j, omega) of the comparator for the lattice gas's omega_eff."""
    oj, om = ctypes.c_double(), ctypes.c_double()
    _check(_lib.ilg_lb_rates(float(omega_eff), ctypes.byref(oj), ctypes.byref(om)))
    return oj.value, om.value


class LB:
    """Lattice Boltzmann comparator (ilg_lb_*), double precision on the device."""

    def __init__(self, lattice, Lx, Ly=1, n0=10.0, amp=0.0, mode_mx=0, mode_my=0, init_weighted=0,
                 omega_j=1.0, omega=1.0, theta=1.0 / 3.0, stream=None, **_ignored):
        self.params = LBParams(int(lattice), int(Lx), int(Ly if lattice != D1Q3 else 1), int(mode_mx), int(mode_my),
                               int(init_weighted), float(n0), float(amp), float(omega_j), float(omega), float(theta))
        self.Q = NUM_VEL[lattice]
        self.Lx, self.Ly = self.params.Lx, self.params.Ly
        h = _vp()
        st = _lib.ilg_lb_create(ctypes.byref(self.params), _vp(stream_handle(stream)), ctypes.byref(h))
        if st != ILG_OK:
            raise IlgError(st, _lib.ilg_lb_last_error(None).decode(errors="replace"))
        self._h = h

    @property
    def shape(self):
        return (self.Q, self.Ly, self.Lx)

    def _check(self, st):
        if st != ILG_OK:
            raise IlgError(st, _lib.ilg_lb_last_error(self._h).decode(errors="replace"))

    def close(self):
        if getattr(self, "_h", None):
            _lib.ilg_lb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def init(self):
        self._check(_lib.ilg_lb_init(self._h))

    def set_state(self, f: np.ndarray, t: int = 0):
        f = np.ascontiguousarray(f, dtype=np.float64)
        self._check(_lib.ilg_lb_set_state(self._h, f.ctypes.data, f.size, int(t)))

    def get_state(self):
        out = np.empty(self.shape, dtype=np.float64)
        t = ctypes.c_uint64()
        self._check(_lib.ilg_lb_get_state(self._h, out.ctypes.data, out.size, ctypes.byref(t)))
        return out, int(t.value)

    def step(self, T: int):
        self._check(_lib.ilg_lb_step(self._h, int(T)))

    def observables(self, modes=()):
        modes = np.ascontiguousarray(np.asarray(modes, dtype=np.int32).reshape(-1, 2))
        n = len(modes)
        re, im, amp = (np.zeros(n) for _ in range(3))
        t = ctypes.c_uint64()
        M = ctypes.c_double()
        self._check(_lib.ilg_lb_observables(self._h, modes.ctypes.data if n else None, n, ctypes.byref(t),
                                            ctypes.byref(M), re.ctypes.data, im.ctypes.data, amp.ctypes.data))
        return dict(t=int(t.value), mass=float(M.value), re=re, im=im, amp=amp)


def observables_noalloc(lattice: int, Lx: int, Ly: int, state_dev_ptr: int, modes=(), stream=None):
    """ilg_observables_noalloc on a device state (see include/ilg.h)."""
    modes = np.ascontiguousarray(np.asarray(modes, dtype=np.int32).reshape(-1, 2))
    n = len(modes)
    re, im, amp, Sk = (np.zeros(n) for _ in range(4))
    M = ctypes.c_uint64()
    _check(_lib.ilg_observables_noalloc(int(lattice), int(Lx), int(Ly), _vp(state_dev_ptr),
                                        modes.ctypes.data if n else None, n, _vp(stream_handle(stream)),
                                        ctypes.byref(M), re.ctypes.data, im.ctypes.data, amp.ctypes.data,
                                        Sk.ctypes.data))
    return dict(mass=int(M.value), re=re, im=im, amp=amp, Sk=Sk)


def philox(ctr: np.ndarray, seed: int, stream=None) -> np.ndarray:
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.zeros_like(ctr)
    _check(_lib.ilg_philox(ctr.reshape(-1), int(seed), out.reshape(-1), len(ctr), _vp(stream_handle(stream))))
    return out


def binomial_table(P: int) -> np.ndarray:
    out = np.zeros(2016, dtype=np.uint32)
    _check(_lib.ilg_binomial_table(int(P), out))
    return out


def alias_table(P: int):
    thr = np.zeros(4096, dtype=np.uint32)
    al = np.zeros(4096, dtype=np.uint32)
    _check(_lib.ilg_alias_table(int(P), thr, al))
    return thr, al


def poisson_table(lam: float, cap: int = 4096) -> np.ndarray:
    out = np.zeros(cap, dtype=np.uint32)
    K = ctypes.c_uint32()
    _check(_lib.ilg_poisson_table(float(lam), out, cap, ctypes.byref(K)))
    return out[:K.value].copy()


INT_PEAK_KINDS = ("philox_blocks", "lop3", "imad", "imad_wide", "lop3_imad_mix")


def int_peak(kind: int, seconds: float = 1.0, stream=None) -> dict:
    """ilg_int_peak: measured integer throughput of the GPU (see include/ilg.h)."""
    rate, ms = ctypes.c_double(), ctypes.c_double()
    _check(_lib.ilg_int_peak(int(kind), float(seconds), _vp(stream_handle(stream)), ctypes.byref(rate),
                             ctypes.byref(ms)))
    return dict(kind=INT_PEAK_KINDS[kind], rate=rate.value, ms=ms.value)


_lib.ilg_inject_alloc_failure.argtypes = [ctypes.c_int64]
_lib.ilg_inject_alloc_failure.restype = ctypes.c_int


def inject_alloc_failure(after: int):
    """ilg_inject_alloc_failure: the library's (after+1)-th next device allocation fails;
    after < 0 switches injection off."""
    _check(_lib.ilg_inject_alloc_failure(int(after)))
