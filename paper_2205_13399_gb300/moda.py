"""ctypes binding of the C ABI in include/moda.h (argument marshalling only).

Every step of the annealing path runs in the CUDA library; this module only
converts numpy arrays and torch streams to the plain pointers the ABI takes.
It raises at import time when the library has not been built: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import platform
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", f"libmoda_{platform.machine()}.so")

OK, EINVAL, ENOMEM, EOVERFLOW, EUNSUPPORTED, ECUDA, ETIMEOUT, EBUSY = range(8)
STATUS_NAMES = ["MODA_OK", "MODA_EINVAL", "MODA_ENOMEM", "MODA_EOVERFLOW",
                "MODA_EUNSUPPORTED", "MODA_ECUDA", "MODA_ETIMEOUT", "MODA_EBUSY"]
ACCEPT = {"strict": 0, "lenient": 1}
ARCHIVE = {"explore": 0, "exploit": 1}
ESCAPE = {"archive": 0, "offset": 1}
FIELD_CACHE = {"auto": 0, "on": 1, "off": 2}
ENGINE = {"auto": 0, "block": 1, "warp": 2}

# Functions declared in include/moda.h.
ABI_FUNCTIONS = [
    "moda_create_instance", "moda_destroy_instance", "moda_instance_info",
    "moda_anneal", "moda_wait", "moda_read_replica", "moda_read_trace",
    "moda_read_archive", "moda_run_elapsed_ms", "moda_destroy_run",
    "moda_last_error", "moda_anneal_noalloc", "moda_anneal_batch",
    "moda_server_create", "moda_server_submit", "moda_server_poll", "moda_server_info",
    "moda_server_destroy", "moda_probe_int_peak", "moda_probe_smem_peak", "moda_scalarize",
    "moda_sbda_front", "moda_read_snapshot", "moda_qubo_create", "moda_qubo_destroy",
    "moda_qubo_anneal", "moda_qrun_wait", "moda_qrun_read", "moda_qrun_elapsed_ms",
    "moda_qrun_destroy", "moda_autotune", "moda_check_accept",
]


class MODAError(RuntimeError):
    def __init__(self, status: int, message: str):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {message}")
        self.status = status


class Penalty(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("w1", ctypes.c_int64), ("w2", ctypes.c_int64)]


class Params(ctypes.Structure):
    _fields_ = [
        ("replicas", ctypes.c_int32),
        ("replica_base", ctypes.c_int32),
        ("I_max", ctypes.c_int64),
        ("delta0", ctypes.c_double),
        ("deltaf", ctypes.c_double),
        ("xi", ctypes.c_double),
        ("beta", ctypes.c_int64),
        ("archive_size", ctypes.c_int32),
        ("accept", ctypes.c_int32),
        ("archive", ctypes.c_int32),
        ("escape", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("block_threads", ctypes.c_int32),
        ("trace", ctypes.c_int32),
        ("field_cache", ctypes.c_int32),
        ("prefetch", ctypes.c_int32),
        ("normalize", ctypes.c_int32),
        ("snapshot_every", ctypes.c_int32),
        ("fast_forward", ctypes.c_int32),
        ("engine", ctypes.c_int32),
        ("cache_slots", ctypes.c_int32),
    ]


class Point(ctypes.Structure):
    _fields_ = [
        ("E1", ctypes.c_int64), ("E2", ctypes.c_int64),
        ("c1", ctypes.c_int64), ("c2", ctypes.c_int64),
        ("g", ctypes.c_int64),
        ("feasible", ctypes.c_int32), ("replica", ctypes.c_int32),
        ("slot", ctypes.c_int32), ("pad", ctypes.c_int32),
    ]


class DeviceOutputs(ctypes.Structure):
    """Device output buffers of moda_anneal_noalloc (caller-owned)."""
    _fields_ = [
        ("arch_E", ctypes.c_void_p),
        ("arch_bits", ctypes.c_void_p),
        ("arch_count", ctypes.c_void_p),
        ("x_final", ctypes.c_void_p),
        ("E_final", ctypes.c_void_p),
        ("stats", ctypes.c_void_p),
        ("error", ctypes.c_void_p),
    ]


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libmoda is not built ({path}); run "
                          "`python -m paper_2205_13399_gb300.build`")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    st = ctypes.c_int
    lib.moda_create_instance.restype = st
    lib.moda_create_instance.argtypes = [i32, P, P, P, ctypes.POINTER(Penalty), ctypes.POINTER(P)]
    lib.moda_destroy_instance.restype = None
    lib.moda_destroy_instance.argtypes = [P]
    lib.moda_instance_info.restype = st
    lib.moda_instance_info.argtypes = [P, ctypes.POINTER(i32), ctypes.POINTER(i64),
                                       ctypes.POINTER(i64)]
    lib.moda_anneal.restype = st
    lib.moda_anneal.argtypes = [P, ctypes.POINTER(Params), P, ctypes.POINTER(P)]
    lib.moda_wait.restype = st
    lib.moda_wait.argtypes = [P, i64]
    lib.moda_read_replica.restype = st
    lib.moda_read_replica.argtypes = [P, i32, P, P, P, P, P, P]
    lib.moda_read_trace.restype = st
    lib.moda_read_trace.argtypes = [P, i32, P]
    lib.moda_read_archive.restype = st
    lib.moda_read_archive.argtypes = [P, i32, ctypes.POINTER(Point), i32,
                                      ctypes.POINTER(i32), P]
    lib.moda_read_snapshot.restype = st
    lib.moda_read_snapshot.argtypes = [P, i32, i32, ctypes.POINTER(Point), i32,
                                       ctypes.POINTER(i32), P]
    lib.moda_run_elapsed_ms.restype = st
    lib.moda_run_elapsed_ms.argtypes = [P, ctypes.POINTER(ctypes.c_float)]
    lib.moda_destroy_run.restype = None
    lib.moda_destroy_run.argtypes = [P]
    lib.moda_last_error.restype = ctypes.c_char_p
    lib.moda_last_error.argtypes = []
    lib.moda_anneal_batch.restype = st
    lib.moda_anneal_batch.argtypes = [ctypes.POINTER(P), ctypes.POINTER(Params), i32, P,
                                      ctypes.POINTER(P)]
    sz = ctypes.c_size_t
    lib.moda_server_create.restype = st
    lib.moda_server_create.argtypes = [sz, P, ctypes.POINTER(P)]
    lib.moda_server_submit.restype = st
    lib.moda_server_submit.argtypes = [P, P, ctypes.POINTER(Params), ctypes.POINTER(i64)]
    lib.moda_server_poll.restype = st
    lib.moda_server_poll.argtypes = [P, i64, ctypes.POINTER(P)]
    lib.moda_server_info.restype = st
    lib.moda_server_info.argtypes = [P, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                     ctypes.POINTER(sz), ctypes.POINTER(sz)]
    lib.moda_server_destroy.restype = None
    lib.moda_server_destroy.argtypes = [P]
    for name in ("moda_probe_int_peak", "moda_probe_smem_peak"):
        f = getattr(lib, name)
        f.restype = st
        f.argtypes = [i32, P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float)]
    lib.moda_check_accept.restype = st
    lib.moda_check_accept.argtypes = [P, P, P, i32, P, P, P]
    lib.moda_scalarize.restype = st
    lib.moda_scalarize.argtypes = [P, i32, i32, ctypes.POINTER(P)]
    lib.moda_sbda_front.restype = st
    lib.moda_sbda_front.argtypes = [P, ctypes.POINTER(P), i32, ctypes.POINTER(Point), i32,
                                    ctypes.POINTER(i32), P]
    lib.moda_qubo_create.restype = st
    lib.moda_qubo_create.argtypes = [i32, i32, P, ctypes.POINTER(P)]
    lib.moda_qubo_destroy.restype = None
    lib.moda_qubo_destroy.argtypes = [P]
    lib.moda_qubo_anneal.restype = st
    lib.moda_qubo_anneal.argtypes = [P, ctypes.POINTER(Params), P, ctypes.POINTER(P)]
    lib.moda_qrun_wait.restype = st
    lib.moda_qrun_wait.argtypes = [P]
    lib.moda_qrun_read.restype = st
    lib.moda_qrun_read.argtypes = [P, P, P, P, P, P, P, P]
    lib.moda_qrun_elapsed_ms.restype = st
    lib.moda_qrun_elapsed_ms.argtypes = [P, ctypes.POINTER(ctypes.c_float)]
    lib.moda_qrun_destroy.restype = None
    lib.moda_qrun_destroy.argtypes = [P]
    lib.moda_autotune.restype = st
    lib.moda_autotune.argtypes = [P, ctypes.POINTER(Params), i32, P, ctypes.POINTER(Params),
                                  ctypes.POINTER(ctypes.c_float)]
    lib.moda_anneal_noalloc.restype = st
    lib.moda_anneal_noalloc.argtypes = [i32, P, P, P, ctypes.POINTER(Penalty),
                                        ctypes.POINTER(Params), ctypes.POINTER(DeviceOutputs), P]
    return lib


_lib = load_library()


def _check(status: int):
    if status != OK:
        raise MODAError(status, _lib.moda_last_error().decode(errors="replace"))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream_handle(stream) -> int | None:
    """A cudaStream_t from a torch.cuda.Stream, an int handle, or None."""
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


class Instance:
    """A bi-objective QAP instance resident on the current CUDA device
    (``moda_create_instance``).  F1, F2, D: n x n non-negative int16; D
    symmetric with a zero diagonal.  ``w=(w1, w2)`` gives explicit penalty
    weights; default: the paper's choice (Eq. vermap)."""

    def __init__(self, F1, F2, D, w=None):
        D = np.ascontiguousarray(np.asarray(D, dtype=np.int16))
        n = int(D.shape[0])
        self._F1 = np.ascontiguousarray(np.asarray(F1, dtype=np.int16))
        self._F2 = np.ascontiguousarray(np.asarray(F2, dtype=np.int16))
        self._D = D
        pen = None if w is None else ctypes.byref(Penalty(1, int(w[0]), int(w[1])))
        h = ctypes.c_void_p()
        _check(_lib.moda_create_instance(n, _ptr(self._F1), _ptr(self._F2), _ptr(self._D),
                                         pen, ctypes.byref(h)))
        self._h = h
        self._info()

    @classmethod
    def _from_handle(cls, h):
        self = cls.__new__(cls)
        self._h = h
        self._info()
        return self

    def scalarize(self, gamma_num: int, gamma_den: int) -> "Instance":
        """``moda_scalarize``: the single-objective instance of Alg. 2 for
        gamma = gamma_num / gamma_den, scaled by gamma_den."""
        h = ctypes.c_void_p()
        _check(_lib.moda_scalarize(self._h, int(gamma_num), int(gamma_den), ctypes.byref(h)))
        return Instance._from_handle(h)

    def _info(self):
        nn = ctypes.c_int32()
        w1, w2 = ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.moda_instance_info(self._h, ctypes.byref(nn), ctypes.byref(w1),
                                       ctypes.byref(w2)))
        self.n = nn.value
        self.m = self.n * self.n
        self.W = (self.m + 31) // 32
        self.w = (w1.value, w2.value)

    def close(self):
        if getattr(self, "_h", None):
            _lib.moda_destroy_instance(self._h)
            self._h = None

    def __del__(self):
        self.close()


@dataclass
class ReplicaResult:
    count: np.ndarray   # [R]
    E: np.ndarray       # [R, s, 2]
    bits: np.ndarray    # [R, s, W] uint32
    x: np.ndarray       # [R, W] uint32
    E_final: np.ndarray  # [R, 2]
    stats: np.ndarray   # [R, 8] (see moda_read_replica)


def unpack_bits(words: np.ndarray, m: int) -> np.ndarray:
    """[..., W] uint32 words -> [..., m] uint8 bits (bit p in word p // 32)."""
    w = np.asarray(words, dtype=np.uint32)
    b = ((w[..., :, None] >> np.arange(32, dtype=np.uint32)) & 1).astype(np.uint8)
    return b.reshape(*w.shape[:-1], w.shape[-1] * 32)[..., :m]


class Run:
    """Handle of one enqueued anneal (``moda_anneal``)."""

    def __init__(self, inst: Instance, handle, params: Params):
        self.inst = inst  # keeps the instance alive while the run exists
        self._h = handle
        self.params = params
        self.R = params.replicas
        self.s = params.archive_size if params.archive_size > 0 else inst.m

    def wait(self, timeout_ms: int = -1):
        _check(_lib.moda_wait(self._h, int(timeout_ms)))
        return self

    def elapsed_ms(self) -> float:
        ms = ctypes.c_float()
        _check(_lib.moda_run_elapsed_ms(self._h, ctypes.byref(ms)))
        return float(ms.value)

    def read(self, replica: int = -1) -> ReplicaResult:
        R = self.R if replica < 0 else 1
        s, W = self.s, self.inst.W
        out = ReplicaResult(
            count=np.zeros(R, dtype=np.int32),
            E=np.zeros((R, s, 2), dtype=np.int64),
            bits=np.zeros((R, s, W), dtype=np.uint32),
            x=np.zeros((R, W), dtype=np.uint32),
            E_final=np.zeros((R, 2), dtype=np.int64),
            stats=np.zeros((R, 8), dtype=np.int64),
        )
        _check(_lib.moda_read_replica(self._h, int(replica), _ptr(out.count), _ptr(out.E),
                                      _ptr(out.bits), _ptr(out.x), _ptr(out.E_final),
                                      _ptr(out.stats)))
        return out

    def read_trace(self, replica: int) -> np.ndarray:
        tr = np.zeros((self.params.I_max, 3), dtype=np.int64)
        _check(_lib.moda_read_trace(self._h, int(replica), _ptr(tr)))
        return tr

    def read_archive(self, replica: int = -1, cap: int | None = None, perms: bool = True,
                     snapshot: int | None = None):
        """Non-dominated archive members (``moda_read_archive``, or
        ``moda_read_snapshot`` of snapshot ``snapshot``) as a list of dicts
        with E1, E2, c1, c2, g, feasible, replica, slot and perm."""
        cnt = ctypes.c_int32()
        if snapshot is None:
            def call(*a):
                return _lib.moda_read_archive(self._h, int(replica), *a)
        else:
            def call(*a):
                return _lib.moda_read_snapshot(self._h, int(snapshot), int(replica), *a)
        _check(call(None, 0, ctypes.byref(cnt), None))
        total = cnt.value if cap is None else min(cap, cnt.value)
        pts = (Point * max(total, 1))()
        pbuf = np.zeros((max(total, 1), self.inst.n), dtype=np.uint8)
        _check(call(pts, total, ctypes.byref(cnt), _ptr(pbuf) if perms else None))
        out = []
        for k in range(total):
            p = pts[k]
            d = dict(E1=p.E1, E2=p.E2, c1=p.c1, c2=p.c2, g=p.g, feasible=bool(p.feasible),
                     replica=p.replica, slot=p.slot)
            if perms:
                d["perm"] = [int(v) for v in pbuf[k]] if p.feasible else None
            out.append(d)
        return out

    def close(self):
        if getattr(self, "_h", None):
            _lib.moda_destroy_run(self._h)
            self._h = None

    def __del__(self):
        self.close()


def make_params(*, replicas: int, I_max: int, seed: int = 0, accept: str = "strict",
                archive: str = "explore", escape: str = "archive", delta0: float = 1e9,
                deltaf: float = 1e4, xi: float = 1e-3, beta: int | None = None,
                archive_size: int = 0, replica_base: int = 0, block_threads: int = 0,
                trace: bool = False, field_cache: str = "auto", prefetch: int = 0,
                normalize: bool = False, snapshot_every: int = 0,
                fast_forward: bool = False, engine: str = "auto",
                cache_slots: int = 0) -> Params:
    if beta is None:
        beta = int(round(delta0 / I_max)) if I_max > 0 else 0
    return Params(int(replicas), int(replica_base), int(I_max), float(delta0), float(deltaf),
                  float(xi), int(beta), int(archive_size), ACCEPT[accept], ARCHIVE[archive],
                  ESCAPE[escape], int(seed) & 0xFFFFFFFFFFFFFFFF, int(block_threads),
                  int(bool(trace)), FIELD_CACHE[field_cache], int(prefetch), int(bool(normalize)),
                  int(snapshot_every), int(bool(fast_forward)), ENGINE[engine],
                  int(cache_slots))


def anneal_noalloc(F1, F2, D, outputs: dict, params: Params | None = None, stream=None,
                   w=None, **kw) -> None:
    """``moda_anneal_noalloc``: anneal without any device allocation by the
    library.  ``outputs`` maps arch_E, arch_bits, arch_count, x_final,
    E_final, stats and error to caller-owned device buffers (anything with a
    ``data_ptr()``, e.g. torch tensors, or int addresses) sized as in
    include/moda.h.  Returns once the work is enqueued on ``stream``."""
    if params is None:
        params = make_params(**kw)
    D = np.ascontiguousarray(np.asarray(D, dtype=np.int16))
    n = int(D.shape[0])
    F1 = np.ascontiguousarray(np.asarray(F1, dtype=np.int16))
    F2 = np.ascontiguousarray(np.asarray(F2, dtype=np.int16))
    if D.shape != (n, n) or F1.shape != (n, n) or F2.shape != (n, n):
        raise ValueError("F1, F2 and D must all be n x n")
    # The C ABI cannot see buffer sizes: check those of tensor outputs here
    # (bytes as documented in include/moda.h; int addresses are trusted).
    m = n * n
    W = (m + 31) // 32
    R = int(params.replicas)
    s = int(params.archive_size) if params.archive_size > 0 else m
    need = {"arch_E": R * s * 16, "arch_bits": R * s * W * 4 + 32, "arch_count": R * 4,
            "x_final": R * W * 4, "E_final": R * 16, "stats": R * 8 * 8, "error": 4}
    for k, v in outputs.items():
        if not isinstance(v, int) and k in need:
            have = int(v.numel()) * int(v.element_size())
            if have < need[k]:
                raise ValueError(f"output {k} holds {have} bytes, needs {need[k]}")
    addr = {k: (v if isinstance(v, int) else int(v.data_ptr())) for k, v in outputs.items()}
    out = DeviceOutputs(addr["arch_E"], addr["arch_bits"], addr["arch_count"], addr["x_final"],
                        addr["E_final"], addr["stats"], addr["error"])
    pen = None if w is None else ctypes.byref(Penalty(1, int(w[0]), int(w[1])))
    _check(_lib.moda_anneal_noalloc(n, _ptr(F1), _ptr(F2), _ptr(D), pen, ctypes.byref(params),
                                    ctypes.byref(out), _stream_handle(stream)))


def anneal(inst: Instance, params: Params | None = None, stream=None, **kw) -> Run:
    """Enqueue ``params.replicas`` independent MDA runs (``moda_anneal``) on
    ``stream`` (a torch.cuda.Stream, a raw handle, or None for the default
    stream) and return without waiting."""
    if params is None:
        params = make_params(**kw)
    h = ctypes.c_void_p()
    _check(_lib.moda_anneal(inst._h, ctypes.byref(params), _stream_handle(stream),
                            ctypes.byref(h)))
    return Run(inst, h, params)


def anneal_batch(instances, params_list, stream=None) -> list[Run]:
    """``moda_anneal_batch``: run i is ``anneal(instances[i], params_list[i])``;
    all of them are enqueued as one CUDA graph launch on ``stream``."""
    k = len(instances)
    if k != len(params_list) or k == 0:
        raise ValueError("need as many params as instances (at least one)")
    hs = (ctypes.c_void_p * k)(*[inst._h for inst in instances])
    ps = (Params * k)(*params_list)
    outs = (ctypes.c_void_p * k)()
    _check(_lib.moda_anneal_batch(hs, ps, k, _stream_handle(stream), outs))
    return [Run(instances[i], ctypes.c_void_p(outs[i]), params_list[i]) for i in range(k)]


class Server:
    """``moda_server_*``: requests are admitted in arrival order while their
    device buffers fit ``hbm_budget`` bytes (0: free memory less a reserve)
    and run beside those already running."""

    def __init__(self, hbm_budget: int = 0, stream=None):
        h = ctypes.c_void_p()
        _check(_lib.moda_server_create(int(hbm_budget), _stream_handle(stream), ctypes.byref(h)))
        self._h = h
        self._req = {}

    def submit(self, inst: Instance, params: Params | None = None, **kw) -> int:
        if params is None:
            params = make_params(**kw)
        t = ctypes.c_int64()
        _check(_lib.moda_server_submit(self._h, inst._h, ctypes.byref(params), ctypes.byref(t)))
        self._req[t.value] = (inst, params)
        return t.value

    def poll(self, ticket: int):
        """The finished Run of ``ticket``, or None while it waits or runs."""
        h = ctypes.c_void_p()
        st = _lib.moda_server_poll(self._h, int(ticket), ctypes.byref(h))
        if st != OK:
            self._req.pop(int(ticket), None)
            _check(st)
        if not h.value:
            return None
        inst, params = self._req.pop(int(ticket))
        return Run(inst, h, params)

    def info(self) -> dict:
        pe, ru = ctypes.c_int64(), ctypes.c_int64()
        used, budget = ctypes.c_size_t(), ctypes.c_size_t()
        _check(_lib.moda_server_info(self._h, ctypes.byref(pe), ctypes.byref(ru),
                                     ctypes.byref(used), ctypes.byref(budget)))
        return dict(pending=pe.value, running=ru.value, bytes_in_use=used.value,
                    budget=budget.value)

    def close(self):
        if getattr(self, "_h", None):
            _lib.moda_server_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


def probe_int_peak(iters: int = 20000, stream=None) -> tuple[float, float]:
    """``moda_probe_int_peak``: (INT32 lane operations per second, kernel ms)."""
    v, ms = ctypes.c_double(), ctypes.c_float()
    _check(_lib.moda_probe_int_peak(int(iters), _stream_handle(stream), ctypes.byref(v),
                                    ctypes.byref(ms)))
    return float(v.value), float(ms.value)


def check_accept(a, delta, idx, stream=None) -> tuple[np.ndarray, np.ndarray]:
    """``moda_check_accept``: the device's acceptance decisions
    a <= fl(delta T[idx]) and the path each took (1 / 0: FP32, -1: double)."""
    a = np.ascontiguousarray(np.asarray(a, dtype=np.int64).reshape(-1))
    delta = np.ascontiguousarray(np.asarray(delta, dtype=np.float64).reshape(-1))
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.uint32).reshape(-1))
    if not (a.size == delta.size == idx.size):
        raise ValueError("a, delta and idx need the same length")
    acc = np.zeros(a.size, dtype=np.uint8)
    path = np.zeros(a.size, dtype=np.int8)
    _check(_lib.moda_check_accept(_ptr(a), _ptr(delta), _ptr(idx), int(a.size),
                                  _stream_handle(stream), _ptr(acc), _ptr(path)))
    return acc.astype(bool), path


def probe_smem_peak(iters: int = 20000, stream=None) -> tuple[float, float]:
    """``moda_probe_smem_peak``: (shared-memory load bytes per second, kernel ms)."""
    v, ms = ctypes.c_double(), ctypes.c_float()
    _check(_lib.moda_probe_smem_peak(int(iters), _stream_handle(stream), ctypes.byref(v),
                                     ctypes.byref(ms)))
    return float(v.value), float(ms.value)


def sbda(inst: Instance, *, replicas: int, I_max: int, seed: int = 0, gamma_den: int = 10,
         gammas=None, delta0: float = 1e9, deltaf: float = 1e4, xi: float = 1e-3,
         beta: int | None = None, block_threads: int = 0, normalize: bool = False,
         stream=None):
    """SB-DA (Alg. 2): one DA run (Alg. 1) per weight gamma = g / gamma_den,
    g in ``gammas`` (default 0..gamma_den), all enqueued as one
    ``moda_anneal_batch`` launch, then the merged non-dominated feasible
    front (``moda_sbda_front``).  The scalarised instances are integers
    scaled by gamma_den, so the temperatures and the offset rate are scaled
    by it too; with ``normalize`` each scalarised QUBO is normalised as in
    Sec. 4.2 (params.normalize: the acceptance test sees s Delta E in IEEE
    double, s = 2^23 / its largest cost coefficient, in which gamma_den
    cancels) and they are taken as given.  Returns (runs, front); front
    points are dicts with c1, c2, weight (index into gammas), replica and
    perm."""
    gammas = list(range(gamma_den + 1)) if gammas is None else list(gammas)
    if beta is None:
        beta = int(round(delta0 / I_max)) if I_max > 0 else 0
    f = 1 if normalize else gamma_den
    insts = [inst.scalarize(g, gamma_den) for g in gammas]
    params = [make_params(replicas=replicas, I_max=I_max, seed=seed, escape="offset",
                          archive_size=1, delta0=delta0 * f, deltaf=deltaf * f, xi=xi,
                          beta=beta * f, block_threads=block_threads,
                          normalize=normalize) for _ in gammas]
    runs = anneal_batch(insts, params, stream=stream)
    for r in runs:
        r.wait()
    return runs, sbda_front(inst, runs)


def sbda_front(inst: Instance, runs) -> list[dict]:
    """``moda_sbda_front`` over finished runs, one per weight."""
    k = len(runs)
    hs = (ctypes.c_void_p * k)(*[r._h for r in runs])
    tot = ctypes.c_int32()
    _check(_lib.moda_sbda_front(inst._h, hs, k, None, 0, ctypes.byref(tot), None))
    cnt = max(tot.value, 1)
    pts = (Point * cnt)()
    perm = np.zeros((cnt, inst.n), dtype=np.uint8)
    _check(_lib.moda_sbda_front(inst._h, hs, k, pts, tot.value, ctypes.byref(tot), _ptr(perm)))
    return [dict(c1=pts[i].c1, c2=pts[i].c2, weight=pts[i].slot, replica=pts[i].replica,
                 perm=[int(v) for v in perm[i]]) for i in range(tot.value)]


class Qubo:
    """K (1..3) objectives as explicit m x m QUBO matrices (upper triangle
    used), resident on the current device (``moda_qubo_create``)."""

    def __init__(self, Q):
        Q = np.ascontiguousarray(np.asarray(Q, dtype=np.int32))
        if Q.ndim != 3 or Q.shape[1] != Q.shape[2]:
            raise ValueError("Q must be K x m x m")
        self.K, self.m = int(Q.shape[0]), int(Q.shape[1])
        self.W = (self.m + 31) // 32
        h = ctypes.c_void_p()
        _check(_lib.moda_qubo_create(self.K, self.m, _ptr(Q), ctypes.byref(h)))
        self._h = h

    def anneal(self, params: Params | None = None, stream=None, **kw) -> "QRun":
        """``moda_qubo_anneal``: enqueue ``params.replicas`` runs."""
        if params is None:
            params = make_params(**kw)
        h = ctypes.c_void_p()
        _check(_lib.moda_qubo_anneal(self._h, ctypes.byref(params), _stream_handle(stream),
                                     ctypes.byref(h)))
        return QRun(self, h, params)

    def close(self):
        if getattr(self, "_h", None):
            _lib.moda_qubo_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


class QRun:
    """Handle of an explicit-QUBO anneal (``moda_qrun_*``)."""

    def __init__(self, q: Qubo, handle, params: Params):
        self.q, self._h, self.params = q, handle, params
        self.R = params.replicas
        self.s = params.archive_size if params.archive_size > 0 else q.m

    def wait(self):
        _check(_lib.moda_qrun_wait(self._h))
        return self

    def elapsed_ms(self) -> float:
        ms = ctypes.c_float()
        _check(_lib.moda_qrun_elapsed_ms(self._h, ctypes.byref(ms)))
        return float(ms.value)

    def read(self, trace: bool = False) -> dict:
        R, s, K, W = self.R, self.s, self.q.K, self.q.W
        out = {"count": np.zeros(R, dtype=np.int32), "E": np.zeros((R, s, K), dtype=np.int64),
               "bits": np.zeros((R, s, W), dtype=np.uint32), "x": np.zeros((R, W), dtype=np.uint32),
               "E_final": np.zeros((R, K), dtype=np.int64), "stats": np.zeros((R, 4), dtype=np.int64)}
        tr = np.zeros((R, self.params.I_max, K + 1), dtype=np.int64) if trace else None
        _check(_lib.moda_qrun_read(self._h, _ptr(out["count"]), _ptr(out["E"]), _ptr(out["bits"]),
                                   _ptr(out["x"]), _ptr(out["E_final"]), _ptr(out["stats"]),
                                   _ptr(tr) if trace else None))
        if trace:
            out["trace"] = tr
        return out

    def close(self):
        if getattr(self, "_h", None):
            _lib.moda_qrun_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


def autotune(inst: Instance, params: Params | None = None, trial_iters: int = 2000,
             stream=None, **kw) -> tuple[Params, float]:
    """``moda_autotune``: the fastest block shape and prefetch distance for
    ``params`` on ``inst`` (short trials); returns (tuned params, trial ms)."""
    if params is None:
        params = make_params(**kw)
    best = Params()
    ms = ctypes.c_float()
    _check(_lib.moda_autotune(inst._h, ctypes.byref(params), int(trial_iters),
                              _stream_handle(stream), ctypes.byref(best), ctypes.byref(ms)))
    return best, float(ms.value)
