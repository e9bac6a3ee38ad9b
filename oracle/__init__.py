"""Plain CPU oracle for the multi-objective Digital Annealer (MDA) on the
bi-objective QAP (Ayodele et al., arXiv 2205.13399).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` legs are the only callers.
The CUDA library never imports, links or executes anything in this folder,
and nothing here imports the CUDA library.

``moda_oracle.c`` holds the annealing loop (Sec. 3.3, Alg. 3-5) on explicit
QUBO matrices; ``front.py`` holds the numpy pieces (QAP cost of Sec. 2.1,
brute-force Pareto fronts, the dominance filter and the 2-D hypervolume of
Sec. 4.3).  This module compiles the C file with the host compiler
(``-O2 -ffp-contract=off``) and wraps it with ctypes.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

from .front import (  # noqa: F401
    decode_permutation,
    encode_permutation,
    hypervolume_2d,
    nondominated,
    pareto_front_bruteforce,
    qap_cost,
)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "moda_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", f"liboracle_{platform.machine()}.so")
_lib = None
_lock = threading.Lock()

ACCEPT = {"strict": 0, "lenient": 1}
ARCHIVE = {"explore": 0, "exploit": 1}
ESCAPE = {"archive": 0, "offset": 1}


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library next to this file."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
           "-fPIC", "-shared", "-pthread", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [
        ("I_max", ctypes.c_int64),
        ("delta0", ctypes.c_double),
        ("deltaf", ctypes.c_double),
        ("xi", ctypes.c_double),
        ("beta", ctypes.c_int64),
        ("archive_size", ctypes.c_int64),
        ("accept", ctypes.c_int),
        ("archive", ctypes.c_int),
        ("escape", ctypes.c_int),
        ("check", ctypes.c_int),
        ("seed", ctypes.c_uint64),
        ("normalize", ctypes.c_int),
        ("snap_every", ctypes.c_int64),
    ]


class _DAParams(ctypes.Structure):
    _fields_ = [
        ("I_max", ctypes.c_int64),
        ("delta0", ctypes.c_double),
        ("deltaf", ctypes.c_double),
        ("xi", ctypes.c_double),
        ("beta", ctypes.c_int64),
        ("seed", ctypes.c_uint64),
        ("normalize", ctypes.c_int),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        lib.oracle_instance_new.restype = P
        lib.oracle_instance_new.argtypes = [ctypes.c_int, P, P, P, ctypes.c_int, i64, i64]
        lib.oracle_instance_free.argtypes = [P]
        lib.oracle_instance_w.restype = i64
        lib.oracle_instance_w.argtypes = [P, ctypes.c_int]
        lib.oracle_instance_m.restype = i64
        lib.oracle_instance_m.argtypes = [P]
        lib.oracle_instance_pg.restype = i64
        lib.oracle_instance_pg.argtypes = [P]
        lib.oracle_instance_copy.argtypes = [P, ctypes.c_int, P]
        for f in ("oracle_energy", "oracle_cost"):
            getattr(lib, f).restype = i64
            getattr(lib, f).argtypes = [P, ctypes.c_int, P]
        lib.oracle_constraint.restype = i64
        lib.oracle_constraint.argtypes = [P, P]
        lib.oracle_philox4x32_10.argtypes = [P, P, P]
        lib.oracle_schedule.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, i64, P]
        lib.oracle_neglog_table.argtypes = [P]
        lib.oracle_penalty_w.restype = i64
        lib.oracle_penalty_w.argtypes = [i64, P]
        lib.oracle_cost_qubo.argtypes = [ctypes.c_int, P, P, P]
        lib.oracle_constraint_qubo.argtypes = [ctypes.c_int, P, P]
        lib.oracle_archive_update.restype = ctypes.c_int
        lib.oracle_archive_update.argtypes = [ctypes.c_int, i64, P, P, P, ctypes.c_uint32]
        lib.oracle_accept_count.restype = i64
        lib.oracle_accept_count.argtypes = [i64, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32,
                                            ctypes.c_uint32, i64]
        lib.oracle_mda_run_many.restype = ctypes.c_int
        lib.oracle_mda_run_many.argtypes = [P, ctypes.POINTER(_Params), i64, P, ctypes.c_int,
                                            P, P, P, P, P, P, P, P, P, P]
        lib.oracle_norm_scale.restype = ctypes.c_double
        lib.oracle_norm_scale.argtypes = [P, ctypes.c_int]
        lib.oracle_sbda_qubo.restype = P
        lib.oracle_sbda_qubo.argtypes = [P, i64, i64]
        lib.oracle_squbo_free.argtypes = [P]
        lib.oracle_squbo_w.restype = i64
        lib.oracle_squbo_w.argtypes = [P]
        lib.oracle_squbo_scale.restype = ctypes.c_double
        lib.oracle_squbo_scale.argtypes = [P]
        lib.oracle_squbo_energy.restype = i64
        lib.oracle_squbo_energy.argtypes = [P, P]
        lib.oracle_da_run_many.restype = ctypes.c_int
        lib.oracle_da_run_many.argtypes = [P, ctypes.POINTER(_DAParams), i64, P, ctypes.c_int,
                                           P, P, P, P, P]
        lib.oracle_kqubo_new.restype = P
        lib.oracle_kqubo_new.argtypes = [ctypes.c_int, i64, P]
        lib.oracle_kqubo_free.argtypes = [P]
        lib.oracle_kqubo_energy.restype = i64
        lib.oracle_kqubo_energy.argtypes = [P, ctypes.c_int, P]
        lib.oracle_kqubo_run.restype = ctypes.c_int
        lib.oracle_kqubo_run.argtypes = [P, ctypes.POINTER(_Params), ctypes.c_uint32,
                                         P, P, P, P, P, P, P]
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _mat(a, n):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.int64))
    if a.shape != (n, n):
        raise ValueError(f"expected an {n}x{n} matrix, got {a.shape}")
    return a


class Instance:
    """Explicit QUBOs of one bi-objective QAP instance (Sec. 2.2-2.3, 3.3).

    ``w=None`` sets each penalty weight from Eq. vermap on the objective's
    own cost QUBO; ``w=(w1, w2)`` uses explicit weights (alpha_k = w_k/2).
    """

    def __init__(self, F1, F2, D, w=None):
        lib = _load()
        D = np.asarray(D)
        n = int(D.shape[0])
        self.n, self.m = n, n * n
        self._F1, self._F2, self._D = _mat(F1, n), _mat(F2, n), _mat(D, n)
        kind, w1, w2 = (0, 0, 0) if w is None else (1, int(w[0]), int(w[1]))
        h = lib.oracle_instance_new(n, _ptr(self._F1), _ptr(self._F2), _ptr(self._D), kind, w1, w2)
        if not h:
            raise MemoryError("oracle_instance_new failed")
        self._h = ctypes.c_void_p(h)
        self.w = (int(lib.oracle_instance_w(self._h, 0)), int(lib.oracle_instance_w(self._h, 1)))
        self.pg = int(lib.oracle_instance_pg(self._h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.oracle_instance_free(h)
            self._h = None

    def matrix(self, which: str) -> np.ndarray:
        """Upper-triangular 'R', 'S' (cost), 'G' (constraint), 'Y' or 'Z'."""
        idx = {"R": 0, "S": 1, "G": 2, "Y": 3, "Z": 4}[which]
        out = np.empty((self.m, self.m), dtype=np.int64)
        _lib.oracle_instance_copy(self._h, idx, _ptr(out))
        return out

    def _bits(self, x):
        x = np.ascontiguousarray(np.asarray(x, dtype=np.uint8).reshape(-1))
        if x.size != self.m:
            raise ValueError("state has the wrong length")
        return x

    def norm_scale(self, k: int) -> float:
        """s_k = 2^23 / (largest coefficient of cost QUBO k), Sec. 4.2."""
        return float(_load().oracle_norm_scale(self._h, int(k)))

    def energy(self, k: int, x) -> int:
        return int(_lib.oracle_energy(self._h, k, _ptr(self._bits(x))))

    def cost(self, k: int, x) -> int:
        return int(_lib.oracle_cost(self._h, k, _ptr(self._bits(x))))

    def constraint(self, x) -> int:
        return int(_lib.oracle_constraint(self._h, _ptr(self._bits(x))))


def cost_qubo(H, D) -> np.ndarray:
    """Upper-triangular cost QUBO of Eq. cqap for one flow matrix."""
    lib = _load()
    D = np.asarray(D)
    n = int(D.shape[0])
    H, D = _mat(H, n), _mat(D, n)
    C = np.empty((n * n, n * n), dtype=np.int64)
    lib.oracle_cost_qubo(n, _ptr(H), _ptr(D), _ptr(C))
    return C


def constraint_qubo(n: int):
    """Upper-triangular G and p_g of Eq. gqap."""
    lib = _load()
    G = np.empty((n * n, n * n), dtype=np.int64)
    pg = np.zeros(1, dtype=np.int64)
    lib.oracle_constraint_qubo(n, _ptr(G), _ptr(pg))
    return G, int(pg[0])


def penalty_w(C) -> int:
    """Eq. vermap on the symmetric form of an upper-triangular QUBO."""
    lib = _load()
    C = np.ascontiguousarray(np.asarray(C, dtype=np.int64))
    return int(lib.oracle_penalty_w(C.shape[0], _ptr(C)))


def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one 4-word counter under a 2-word key."""
    lib = _load()
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.empty(4, dtype=np.uint32)
    lib.oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def schedule(delta0: float, deltaf: float, xi: float, count: int) -> np.ndarray:
    lib = _load()
    out = np.empty(count, dtype=np.float64)
    lib.oracle_schedule(delta0, deltaf, xi, count, _ptr(out))
    return out


def neglog_table() -> np.ndarray:
    lib = _load()
    out = np.empty(65536, dtype=np.float64)
    lib.oracle_neglog_table(_ptr(out))
    return out


def archive_update(kind: str, s: int, archive: list, E_new, u: int = 0) -> list:
    """One explorative (Alg. 4) or exploitative (Alg. 5) update of an archive
    given as a list of (E1, E2); ``u`` is the exploit draw."""
    lib = _load()
    E = np.zeros((max(s, 1), 2), dtype=np.int64)
    for i, (a, b) in enumerate(archive):
        E[i] = (a, b)
    cnt = np.array([len(archive)], dtype=np.int64)
    en = np.asarray(E_new, dtype=np.int64)
    rc = lib.oracle_archive_update(ARCHIVE[kind], int(s), _ptr(cnt), _ptr(E), _ptr(en),
                                   int(u) & 0xFFFFFFFF)
    if rc != 0:
        raise MemoryError
    return [tuple(int(v) for v in E[i]) for i in range(int(cnt[0]))]


def accept_count(a: int, delta: float, seed: int, step: int, replica: int, groups: int) -> int:
    """How many of the 4*groups acceptance tests of penalty ``a`` pass."""
    lib = _load()
    return int(lib.oracle_accept_count(int(a), float(delta), int(seed), int(step), int(replica),
                                       int(groups)))


def run(inst: Instance, *, I_max: int, replicas, seed: int = 0, accept: str = "strict",
        archive: str = "explore", escape: str = "archive", delta0: float = 1e9,
        deltaf: float = 1e4, xi: float = 1e-3, beta: int | None = None,
        archive_size: int = 0, check: bool = False, trace: bool = False,
        threads: int | None = None, normalize: bool = False, snapshot_every: int = 0) -> dict:
    """Alg. 3 for each replica index in ``replicas`` (an int r means the
    replica indices 0..r-1).

    Returns numpy arrays: ``count`` [R], ``E`` [R, s, 2], ``bits`` [R, s, m],
    ``x`` [R, m], ``E_final`` [R, 2], ``stats`` [R, 4] (flips, jumps to the
    archive, escapes with an empty archive, offset raises) and ``trace``
    [R, I_max, 3] (E1, E2, event) when asked for.
    """
    lib = _load()
    if isinstance(replicas, (int, np.integer)):
        replicas = range(int(replicas))  # a count means replicas 0..count-1
    reps = np.ascontiguousarray(np.asarray(replicas, dtype=np.uint32).reshape(-1))
    R, m = reps.size, inst.m
    s = archive_size if archive_size > 0 else m
    if beta is None:
        beta = int(round(delta0 / I_max)) if I_max > 0 else 0
    prm = _Params(int(I_max), float(delta0), float(deltaf), float(xi), int(beta), int(s),
                  ACCEPT[accept], ARCHIVE[archive], ESCAPE[escape], int(bool(check)),
                  int(seed) & 0xFFFFFFFFFFFFFFFF, int(bool(normalize)), int(snapshot_every))
    out = {
        "count": np.zeros(R, dtype=np.int64),
        "E": np.zeros((R, s, 2), dtype=np.int64),
        "bits": np.zeros((R, s, m), dtype=np.uint8),
        "x": np.zeros((R, m), dtype=np.uint8),
        "E_final": np.zeros((R, 2), dtype=np.int64),
        "stats": np.zeros((R, 4), dtype=np.int64),
    }
    tr = np.zeros((R, I_max, 3), dtype=np.int64) if trace else None
    ns = I_max // snapshot_every if snapshot_every > 0 else 0
    snap = None
    if ns > 0:
        snap = {"count": np.zeros((R, ns), dtype=np.int64),
                "E": np.zeros((R, ns, s, 2), dtype=np.int64),
                "bits": np.zeros((R, ns, s, m), dtype=np.uint8)}
    nth = threads if threads else (os.cpu_count() or 1)
    rc = lib.oracle_mda_run_many(inst._h, ctypes.byref(prm), R, _ptr(reps), int(nth),
                                 _ptr(out["count"]), _ptr(out["E"]), _ptr(out["bits"]),
                                 _ptr(out["x"]), _ptr(out["E_final"]), _ptr(out["stats"]),
                                 _ptr(tr) if tr is not None else None,
                                 _ptr(snap["count"]) if snap else None,
                                 _ptr(snap["E"]) if snap else None,
                                 _ptr(snap["bits"]) if snap else None)
    if rc != 0:
        raise RuntimeError(f"oracle run failed with code {rc}")
    if tr is not None:
        out["trace"] = tr
    if snap is not None:
        out["snapshots"] = snap
    return out


def da_run(inst: Instance, gnum: int, gden: int, *, I_max: int, replicas, seed: int = 0,
           delta0: float = 1e9, deltaf: float = 1e4, xi: float = 1e-3,
           beta: int | None = None, threads: int | None = None,
           normalize: bool = False) -> dict:
    """Alg. 1 (DA) on the scalarised QUBO of Alg. 2 for gamma = gnum / gden,
    in integers scaled by gden: Q = gnum R + (gden - gnum) S + alpha G with
    alpha from Eq. vermap on that cost, temperatures delta0 * gden and
    deltaf * gden, offset rate beta * gden (beta defaults to delta0 / I_max).
    ``normalize``: the QUBO normalised as in Sec. 4.2 (its cost part's
    largest coefficient set to 2^23, ``scale`` = 2^23 / that coefficient):
    the acceptance test sees scale * Delta E - E_off in IEEE double, and the
    temperatures and offset rate are taken as given, in the normalised
    QUBO's units (the gden factor cancels in the scale).
    Returns ``w``, ``scale`` and per replica ``best_x`` [R, m], ``best_E``
    [R], ``x`` [R, m], ``E_final`` [R] and ``stats`` [R, 2] (flips, offset
    raises); energies are the unnormalised integers."""
    lib = _load()
    if isinstance(replicas, (int, np.integer)):
        replicas = range(int(replicas))
    reps = np.ascontiguousarray(np.asarray(replicas, dtype=np.uint32).reshape(-1))
    R, m = reps.size, inst.m
    if beta is None:
        beta = int(round(delta0 / I_max)) if I_max > 0 else 0
    q = lib.oracle_sbda_qubo(inst._h, int(gnum), int(gden))
    if not q:
        raise ValueError("bad scalarisation weight")
    try:
        f = 1 if normalize else gden
        prm = _DAParams(int(I_max), float(delta0) * f, float(deltaf) * f, float(xi),
                        int(beta) * f, int(seed) & 0xFFFFFFFFFFFFFFFF, int(bool(normalize)))
        out = {"w": int(lib.oracle_squbo_w(q)), "scale": float(lib.oracle_squbo_scale(q)),
               "best_x": np.zeros((R, m), dtype=np.uint8),
               "best_E": np.zeros(R, dtype=np.int64),
               "x": np.zeros((R, m), dtype=np.uint8),
               "E_final": np.zeros(R, dtype=np.int64),
               "stats": np.zeros((R, 2), dtype=np.int64)}
        nth = threads if threads else (os.cpu_count() or 1)
        rc = lib.oracle_da_run_many(q, ctypes.byref(prm), R, _ptr(reps), int(nth),
                                    _ptr(out["best_x"]), _ptr(out["best_E"]), _ptr(out["x"]),
                                    _ptr(out["E_final"]), _ptr(out["stats"]))
        if rc != 0:
            raise RuntimeError(f"oracle DA failed with code {rc}")
        out["energy_check"] = [int(lib.oracle_squbo_energy(q, _ptr(np.ascontiguousarray(x))))
                               for x in out["best_x"][:2]]
    finally:
        lib.oracle_squbo_free(q)
    return out


def sbda(inst: Instance, *, gden: int = 10, gammas=None, **kw) -> dict:
    """Alg. 2: one DA run (``da_run``) per weight gamma = g / gden, g in
    ``gammas`` (default 0..gden), then the non-dominated feasible solutions
    of all runs by their QAP costs (c1, c2).  Returns ``runs`` (per weight)
    and ``front``: a list of (c1, c2, weight index, replica) sorted by c1,
    among equal cost vectors the lowest (weight index, replica)."""
    gammas = list(range(gden + 1)) if gammas is None else list(gammas)
    runs = [da_run(inst, g, gden, **kw) for g in gammas]
    cand = []
    for gi, r in enumerate(runs):
        for rep, x in enumerate(r["best_x"]):
            if inst.constraint(x) == 0:
                cand.append((inst.cost(0, x), inst.cost(1, x), gi, rep))
    keep = nondominated([(c[0], c[1]) for c in cand])
    front = sorted((cand[i] for i in keep), key=lambda c: (c[0], c[1]))
    return {"runs": runs, "front": front}


class KQubo:
    """K objectives given as explicit m x m QUBOs (upper triangle used),
    E_k(x) = x^T Q_k x."""

    def __init__(self, Q):
        Q = np.ascontiguousarray(np.asarray(Q, dtype=np.int64))
        if Q.ndim != 3 or Q.shape[1] != Q.shape[2]:
            raise ValueError("Q must be K x m x m")
        self.K, self.m = int(Q.shape[0]), int(Q.shape[1])
        self._Q = Q
        self._h = _load().oracle_kqubo_new(self.K, self.m, _ptr(Q))
        if not self._h:
            raise MemoryError("oracle_kqubo_new failed")

    def energy(self, k: int, x) -> int:
        x = np.ascontiguousarray(np.asarray(x, dtype=np.uint8).reshape(-1))
        return int(_load().oracle_kqubo_energy(self._h, int(k), _ptr(x)))

    def __del__(self):
        if getattr(self, "_h", None):
            _load().oracle_kqubo_free(self._h)
            self._h = None


def kqubo_run(q: KQubo, *, I_max: int, replicas, seed: int = 0, accept: str = "strict",
              archive: str = "explore", escape: str = "archive", delta0: float = 1e9,
              deltaf: float = 1e4, xi: float = 1e-3, beta: int | None = None,
              archive_size: int = 0, check: bool = False, trace: bool = False) -> dict:
    """Alg. 3 on K explicit QUBOs for each replica index in ``replicas`` (an
    int r means 0..r-1).  Returns ``count`` [R], ``E`` [R, s, K], ``bits``
    [R, s, m], ``x`` [R, m], ``E_final`` [R, K], ``stats`` [R, 4] and, when
    asked, ``trace`` [R, I_max, K + 1] (energies, event)."""
    lib = _load()
    if isinstance(replicas, (int, np.integer)):
        replicas = range(int(replicas))
    reps = [int(r) for r in replicas]
    R, m, K = len(reps), q.m, q.K
    s = archive_size if archive_size > 0 else m
    if beta is None:
        beta = int(round(delta0 / I_max)) if I_max > 0 else 0
    prm = _Params(int(I_max), float(delta0), float(deltaf), float(xi), int(beta), int(s),
                  ACCEPT[accept], ARCHIVE[archive], ESCAPE[escape], int(bool(check)),
                  int(seed) & 0xFFFFFFFFFFFFFFFF, 0, 0)
    out = {"count": np.zeros(R, dtype=np.int64), "E": np.zeros((R, s, K), dtype=np.int64),
           "bits": np.zeros((R, s, m), dtype=np.uint8), "x": np.zeros((R, m), dtype=np.uint8),
           "E_final": np.zeros((R, K), dtype=np.int64), "stats": np.zeros((R, 4), dtype=np.int64)}
    if trace:
        out["trace"] = np.zeros((R, I_max, K + 1), dtype=np.int64)
    for i, r in enumerate(reps):
        cnt = np.zeros(1, dtype=np.int64)
        E = np.ascontiguousarray(out["E"][i])
        bits = np.ascontiguousarray(out["bits"][i])
        x = np.zeros(m, dtype=np.uint8)
        Ef = np.zeros(K, dtype=np.int64)
        st = np.zeros(4, dtype=np.int64)
        tr = np.zeros((I_max, K + 1), dtype=np.int64) if trace else None
        rc = lib.oracle_kqubo_run(q._h, ctypes.byref(prm), r, _ptr(cnt), _ptr(E), _ptr(bits),
                                  _ptr(x), _ptr(Ef), _ptr(st), _ptr(tr) if trace else None)
        if rc != 0:
            raise RuntimeError(f"oracle K-objective run failed with code {rc}")
        out["count"][i] = cnt[0]
        out["E"][i], out["bits"][i], out["x"][i] = E, bits, x
        out["E_final"][i], out["stats"][i] = Ef, st
        if trace:
            out["trace"][i] = tr
    return out
