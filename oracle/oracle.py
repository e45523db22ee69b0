"""ctypes wrapper of the sequential C++ oracle (ldl_oracle.cpp).

Test infrastructure only: used by tests/, the smoke check and the benchmark's
CPU-baseline leg, never by the library itself.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ldl_oracle.cpp")
_LIB = os.path.join(_HERE, "libldl_oracle.so")

# N=2, L=4, M=5, alpha=0.001, beta=0.01 are the paper's defaults (Sec. IV-D);
# gamma = 1 as in all of the paper's experiments.
PARAM_DEFAULTS = dict(directed=0, gamma_num=1, gamma_den=1, N=2, L=4, M=5, M_static=20,
                      alpha_inv=1000, beta_inv=100)


def build_oracle(force: bool = False) -> str:
    """Compile the oracle shared library with g++ (plain -O2, no -march)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build_oracle())
        P = C.c_void_p
        lib.orc_create.restype = P
        lib.orc_create.argtypes = [P, C.c_int64, C.c_int64, P, P, P, P]
        lib.orc_apply.restype = C.c_int32
        lib.orc_apply.argtypes = [P, P, C.c_int64]
        lib.orc_destroy.argtypes = [P]
        lib.orc_top.restype = C.c_int32
        lib.orc_top.argtypes = [P]
        lib.orc_level.argtypes = [P, C.c_int32, P, P, P, P, P, P]
        lib.orc_level_nnz.restype = C.c_int64
        lib.orc_level_nnz.argtypes = [P, C.c_int32]
        lib.orc_level_adj.argtypes = [P, C.c_int32, P, P, P]
        lib.orc_comm.argtypes = [P, P, P, P]
        lib.orc_scalars.argtypes = [P, P, P, P]
        lib.orc_q_repair.argtypes = [P, P, P]
        lib.orc_modularity.restype = C.c_double
        lib.orc_modularity.argtypes = [P]
        lib.orc_counters.argtypes = [P, P]
        lib.orc_check.restype = C.c_char_p
        lib.orc_check.argtypes = [P]
        lib.orc_gain.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, P, P]
        lib.orc_decouple.argtypes = [C.c_int64, P, P, P, P, P, C.c_int64, P]
        lib.orc_best_move.restype = C.c_int32
        lib.orc_best_move.argtypes = [P, C.c_int32, C.c_int32, P, P, P]
        lib.orc_best_ref.restype = C.c_int32
        lib.orc_best_ref.argtypes = [P, C.c_int32, C.c_int32, P, P, P]
        lib.orc_set_partition.restype = C.c_int32
        lib.orc_set_partition.argtypes = [P, P]
        lib.orc_grow.restype = C.c_int32
        lib.orc_grow.argtypes = [P, C.c_int64]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


@dataclass
class LevelState:
    lab: np.ndarray
    par: np.ndarray
    kout: np.ndarray
    kin: np.ndarray
    cnt: np.ndarray
    alive: np.ndarray


class OracleError(RuntimeError):
    def __init__(self, status: int):
        super().__init__(f"oracle status {status}")
        self.status = status


class Oracle:
    """One LD-Leiden state: created from a CSR snapshot by static Leiden,
    updated batch by batch."""

    def __init__(self, g, **params):
        p = dict(PARAM_DEFAULTS)
        p["directed"] = int(g.directed)
        p.update(params)
        self.params = p
        self.n = int(g.n)
        lib = _load()
        pv = np.array([p["directed"], p["gamma_num"], p["gamma_den"], p["N"], p["L"], p["M"],
                       p["M_static"], p["alpha_inv"], p["beta_inv"]], dtype=np.int64)
        rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
        col = np.ascontiguousarray(g.col, dtype=np.int32)
        w = np.ascontiguousarray(g.w, dtype=np.int32)
        st = np.zeros(1, dtype=np.int32)
        self._h = lib.orc_create(_ptr(pv), self.n, len(col), _ptr(rp), _ptr(col), _ptr(w), _ptr(st))
        if not self._h:
            raise OracleError(int(st[0]))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _load().orc_destroy(h)
            self._h = None

    def apply(self, batch: np.ndarray) -> int:
        b = np.ascontiguousarray(batch, dtype=np.int32).reshape(-1, 4)
        return int(_load().orc_apply(self._h, _ptr(b), b.shape[0]))

    @property
    def top(self) -> int:
        return int(_load().orc_top(self._h))

    def level(self, r: int) -> LevelState:
        n = self.n
        a = [np.zeros(n, np.int32), np.zeros(n, np.int32), np.zeros(n, np.int64),
             np.zeros(n, np.int64), np.zeros(n, np.int32), np.zeros(n, np.uint8)]
        _load().orc_level(self._h, r, *[_ptr(x) for x in a])
        return LevelState(*a)

    def level_adj(self, r: int):
        lib = _load()
        nnz = int(lib.orc_level_nnz(self._h, r))
        rp = np.zeros(self.n + 1, np.int64)
        col = np.zeros(nnz, np.int32)
        w = np.zeros(nnz, np.int64)
        lib.orc_level_adj(self._h, r, _ptr(rp), _ptr(col), _ptr(w))
        return rp, col, w

    def comm(self):
        n = self.n
        a = [np.zeros(n, np.int64) for _ in range(3)]
        _load().orc_comm(self._h, *[_ptr(x) for x in a])
        return tuple(a)

    def scalars(self):
        m = np.zeros(1, np.int64)
        hi = np.zeros(1, np.int64)
        lo = np.zeros(1, np.uint64)
        _load().orc_scalars(self._h, _ptr(m), _ptr(hi), _ptr(lo))
        return int(m[0]), (int(hi[0]) << 64) + int(lo[0])

    def q_after_repair(self) -> int:
        hi = np.zeros(1, np.int64)
        lo = np.zeros(1, np.uint64)
        _load().orc_q_repair(self._h, _ptr(hi), _ptr(lo))
        return (int(hi[0]) << 64) + int(lo[0])

    def modularity(self) -> float:
        return float(_load().orc_modularity(self._h))

    def counters(self) -> dict:
        c = np.zeros(8, np.int64)
        _load().orc_counters(self._h, _ptr(c))
        keys = ["moves", "refine_moves", "rollbacks", "rounds", "scanned", "candidates",
                "agg_records", "passes"]
        return dict(zip(keys, (int(x) for x in c)))

    def check(self) -> str:
        return _load().orc_check(self._h).decode()

    def gain(self, r: int, v: int, b: int) -> int:
        hi = np.zeros(1, np.int64)
        lo = np.zeros(1, np.uint64)
        _load().orc_gain(self._h, r, v, b, _ptr(hi), _ptr(lo))
        return (int(hi[0]) << 64) + int(lo[0])

    def labels(self) -> np.ndarray:
        return self.level(0).lab

    def _best(self, fn, r: int, v: int):
        t = np.zeros(1, np.int32)
        hi = np.zeros(1, np.int64)
        lo = np.zeros(1, np.uint64)
        have = int(fn(self._h, r, v, _ptr(t), _ptr(hi), _ptr(lo)))
        if have < 0:
            raise ValueError(f"bad arguments r={r} v={v}")
        return (int(t[0]), (int(hi[0]) << 64) + int(lo[0])) if have else None

    def best_move(self, r: int, v: int):
        """(target, gain) the move loop's BestMove picks for node v at level r,
        or None when v has no adjacent community with a positive gain."""
        return self._best(_load().orc_best_move, r, v)

    def best_ref(self, r: int, v: int):
        """(target, gain) the refinement loop's BestRef picks for the singleton
        node v at level r < top, or None."""
        return self._best(_load().orc_best_ref, r, v)

    def grow(self, n_new: int) -> None:
        """Adds isolated vertices up to n_new (the vertex set may change
        between batches)."""
        if int(_load().orc_grow(self._h, int(n_new))) != 0:
            raise ValueError("grow needs n_new >= n")
        self.n = int(n_new)

    def set_partition(self, lab) -> None:
        """Test set-up of a one-level state: replace the level-0 partition and
        recompute the community statistics from it."""
        a = np.ascontiguousarray(lab, dtype=np.int32)
        if int(_load().orc_set_partition(self._h, _ptr(a))) != 0:
            raise ValueError("set_partition needs a one-level state and labels in [0, n)")


def decouple(v, src, dst, gains, id_space: Optional[int] = None) -> np.ndarray:
    """Run the oracle's decoupling filter on explicit candidates; gains are
    Python ints (up to 127 bits).  Returns a 0/1 accepted mask."""
    v = np.ascontiguousarray(v, dtype=np.int32)
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    g = [int(x) for x in gains]
    hi = np.array([x >> 64 for x in g], dtype=np.int64)
    lo = np.array([x & ((1 << 64) - 1) for x in g], dtype=np.uint64)
    if id_space is None:
        id_space = int(max(src.max(initial=0), dst.max(initial=0))) + 1
    out = np.zeros(len(v), np.uint8)
    _load().orc_decouple(len(v), _ptr(v), _ptr(src), _ptr(dst), _ptr(hi), _ptr(lo), id_space,
                         _ptr(out))
    return out
