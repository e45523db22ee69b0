"""Python binding of the C ABI in include/ldl.h (argument marshalling only).

Every step of the update runs in the CUDA library libldl.so; this module only
converts numpy arrays / torch tensors to pointers and status codes to
exceptions.  There is no CPU fallback: if the library cannot be loaded the
import of LDL raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

from .build import build

LDL_OK, LDL_E_INVALID, LDL_E_RANGE, LDL_E_NO_EDGE, LDL_E_NEG_WEIGHT, LDL_E_NOMEM, LDL_E_CUDA, \
    LDL_E_TIMEOUT, LDL_E_OVERFLOW = range(9)
INSERT, DELETE, REWEIGHT = 0, 1, 2
STATUS_NAMES = {0: "OK", 1: "INVALID", 2: "RANGE", 3: "NO_EDGE", 4: "NEG_WEIGHT", 5: "NOMEM",
                6: "CUDA", 7: "TIMEOUT", 8: "OVERFLOW"}
STAGES = ["ingest", "repair", "expand", "bestmove", "decouple", "commit", "refine", "aggregate",
          "pushdown", "agg.emit", "agg.sort", "agg.apply", "agg.up", "agg.exist", "ref.dissolve", "ref.loop"]


class ldl_params(C.Structure):
    _fields_ = [("directed", C.c_int32), ("gamma_num", C.c_int32), ("gamma_den", C.c_int32),
                ("N", C.c_int32), ("L", C.c_int32), ("M", C.c_int32), ("M_static", C.c_int32),
                ("alpha_inv", C.c_int32), ("beta_inv", C.c_int32), ("cluster_max_deg", C.c_int32),
                ("kernel_stats", C.c_int32), ("bin_deg", C.c_int32 * 4), ("no_rollback", C.c_int32),
                ("cuda_stream", C.c_void_p)]


class ldl_result(C.Structure):
    _fields_ = [("labels", C.c_void_p), ("n", C.c_int64), ("changed", C.c_void_p),
                ("n_changed", C.c_int64), ("levels", C.c_int32),
                ("parent", C.c_void_p), ("comm", C.c_void_p), ("refined", C.c_void_p),
                ("alive", C.c_void_p),
                ("frontier_nodes", C.c_int64 * 8), ("edges_scanned", C.c_int64),
                ("moves", C.c_int64), ("refine_moves", C.c_int64), ("rejected", C.c_int64),
                ("rollbacks", C.c_int64), ("rounds", C.c_int64), ("agg_records", C.c_int64),
                ("decouple_rounds", C.c_int64), ("host_syncs", C.c_int64),
                ("pending_records", C.c_int64), ("pending_applied", C.c_int64),
                ("split_members", C.c_int64)]


class LdlError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load(path: Optional[str] = None):
    """Load libldl.so (building it first when the sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = build()
    if not os.path.exists(path):
        raise OSError(f"CUDA library not found: {path}")
    lib = C.CDLL(path)
    P, I32, I64 = C.c_void_p, C.c_int32, C.c_int64
    sig = {
        "ldl_default_params": (None, [P]),
        "ldl_create": (I32, [P, I64, I64, P, P, P, P]),
        "ldl_apply_batch": (I32, [P, P, I64, I32, P]),
        "ldl_modularity": (I32, [P, P]),
        "ldl_modularity_num": (I32, [P, P, P, P]),
        "ldl_destroy": (None, [P]),
        "ldl_last_error": (C.c_char_p, [P]),
        "ldl_levels": (I32, [P]),
        "ldl_get_level": (I32, [P, I32, P, P, P, P, P, P]),
        "ldl_level_nnz": (I32, [P, I32, P]),
        "ldl_get_adjacency": (I32, [P, I32, P, P, P]),
        "ldl_get_communities": (I32, [P, P, P, P]),
        "ldl_stage_times": (I32, [P, P]),
        "ldl_set_timing": (I32, [P, I32]),
        "ldl_debug_fail_alloc_after": (None, [I64]),
        "ldl_debug_scan_wait_timeout": (I32, []),
        "ldl_copy_changed": (I32, [P, P, P]),
        "ldl_copy_changed_noalloc": (I32, [P, P, P]),
        "ldl_launch_count": (I64, []),
        "ldl_set_kernel_stats": (I32, [P, I32]),
        "ldl_get_kernel_stats": (I32, [P, P]),
        "ldl_apply_batches": (I32, [P, P, P, I32, I32, I32, P, P]),
        "ldl_estimate_bytes": (I32, [P, I64, I64, P]),
        "ldl_server_create": (I32, [I32, P]),
        "ldl_server_admit": (I32, [P, P, I64, I64, P, P, P, P]),
        "ldl_server_submit": (I32, [P, P, P, I64, P]),
        "ldl_server_wait": (I32, [P, I64, I32, P, P, P, P]),
        "ldl_server_destroy": (None, [P]),
        "ldl_debug_decouple": (I32, [P, I64, P, P, P, P, P, P]),
        "ldl_debug_sort_pairs": (I32, [P, I64, P, P, I32]),
        "ldl_debug_hub_table_slots": (None, [I64]),
        "ldl_debug_alloc_counts": (None, [P, P]),
        "ldl_batch_estimate_bytes": (I32, [P, I64, P]),
        "ldl_server_stats": (I32, [P, P, P]),
        "ldl_server_debug_free_bytes": (I32, [P, I64]),
        "ldl_save": (I32, [P, C.c_char_p]),
        "ldl_load": (I32, [C.c_char_p, P, P]),
        "ldl_grow": (I32, [P, I64]),
        "ldl_num_vertices": (I64, [P]),
        "ldl_is_directed": (I32, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    """Names the header declares (for the export check)."""
    return ["ldl_default_params", "ldl_create", "ldl_apply_batch", "ldl_modularity",
            "ldl_modularity_num", "ldl_destroy", "ldl_last_error", "ldl_levels", "ldl_get_level",
            "ldl_level_nnz", "ldl_get_adjacency", "ldl_get_communities", "ldl_stage_times",
            "ldl_set_timing", "ldl_debug_fail_alloc_after", "ldl_debug_scan_wait_timeout", "ldl_copy_changed", "ldl_copy_changed_noalloc", "ldl_launch_count",
            "ldl_set_kernel_stats", "ldl_get_kernel_stats", "ldl_apply_batches", "ldl_estimate_bytes",
            "ldl_server_create", "ldl_server_admit", "ldl_server_submit", "ldl_server_wait",
            "ldl_server_destroy", "ldl_debug_decouple", "ldl_debug_alloc_counts", "ldl_batch_estimate_bytes",
            "ldl_server_stats", "ldl_server_debug_free_bytes", "ldl_save", "ldl_load", "ldl_grow",
            "ldl_num_vertices", "ldl_is_directed", "ldl_debug_sort_pairs", "ldl_debug_hub_table_slots"]


def launch_count() -> int:
    return int(load().ldl_launch_count())


def alloc_counts():
    """(all, in_batch): device allocations attempted by the library, and those
    made while a batch was changing a context's state."""
    a, b = C.c_int64(), C.c_int64()
    load().ldl_debug_alloc_counts(C.byref(a), C.byref(b))
    return int(a.value), int(b.value)


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


@dataclass
class Level:
    lab: np.ndarray
    par: np.ndarray
    kout: np.ndarray
    kin: np.ndarray
    cnt: np.ndarray
    alive: np.ndarray


def make_params(directed=False, gamma_num=1, gamma_den=1, N=2, L=4, M=5, M_static=20, alpha_inv=1000,
                beta_inv=100, stream=None, cluster_max_deg=0, kernel_stats=0, bin_deg=None,
                no_rollback=0) -> ldl_params:
    p = ldl_params()
    load().ldl_default_params(C.byref(p))
    p.directed, p.gamma_num, p.gamma_den = int(directed), gamma_num, gamma_den
    p.N, p.L, p.M, p.M_static = N, L, M, M_static
    p.alpha_inv, p.beta_inv = alpha_inv, beta_inv
    p.cluster_max_deg = cluster_max_deg
    p.kernel_stats = kernel_stats
    p.no_rollback = int(no_rollback)
    if bin_deg is not None:
        for i, t in enumerate(bin_deg):
            p.bin_deg[i] = int(t)
    p.cuda_stream = stream
    return p


# sweep kernel groups of ldl_get_kernel_stats, in its order
SWEEP_GROUPS = ("sweep_group8", "sweep_warp", "sweep_block128", "sweep_block256", "sweep_cluster", "sweep_hub_acc",
                "sweep_hub_rest")


class LDL:
    """One device-resident LD-Leiden instance (ldl_create ... ldl_destroy).

    `stream` is a cudaStream_t handle (e.g. torch.cuda.Stream().cuda_stream);
    None uses the legacy default stream."""

    def __init__(self, n, row_ptr, col, w, directed=False, gamma_num=1, gamma_den=1, N=2, L=4, M=5,
                 M_static=20, alpha_inv=1000, beta_inv=100, stream=None, server=None, cluster_max_deg=0,
                 kernel_stats=0, bin_deg=None, no_rollback=0):
        lib = load()
        p = make_params(directed, gamma_num, gamma_den, N, L, M, M_static, alpha_inv, beta_inv, stream,
                        cluster_max_deg, kernel_stats, bin_deg, no_rollback)
        self.n = int(n)
        self.directed = bool(directed)
        rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
        cl = np.ascontiguousarray(col, dtype=np.int32)
        wt = np.ascontiguousarray(w, dtype=np.int32)
        h = C.c_void_p()
        if server is None:
            st = lib.ldl_create(C.byref(p), self.n, len(cl), _ptr(rp), _ptr(cl), _ptr(wt), C.byref(h))
        else:
            st = lib.ldl_server_admit(server._h, C.byref(p), self.n, len(cl), _ptr(rp), _ptr(cl), _ptr(wt),
                                      C.byref(h))
        if st != LDL_OK:
            raise LdlError(st, lib.ldl_last_error(None).decode())
        self._h = h
        self.last = ldl_result()

    @classmethod
    def from_graph(cls, g, **kw):
        return cls(g.n, g.row_ptr, g.col, g.w, directed=g.directed, **kw)

    @classmethod
    def load(cls, path: str, stream=None, **kw):
        """A context resumed from a file written by save() (ldl_load); n and
        the direction come from the file."""
        lib = load()
        obj = cls.__new__(cls)
        p = make_params(stream=stream, **kw)
        h = C.c_void_p()
        st = lib.ldl_load(os.fsencode(path), C.byref(p), C.byref(h))
        if st != LDL_OK:
            raise LdlError(st, lib.ldl_last_error(None).decode())
        obj._h = h
        obj.last = ldl_result()
        obj.n = int(lib.ldl_num_vertices(h))
        obj.directed = bool(lib.ldl_is_directed(h))
        return obj

    def save(self, path: str):
        """Writes the whole state to a file (ldl_save)."""
        self._check(load().ldl_save(self._h, os.fsencode(path)))

    def grow(self, n_new: int):
        """Appends isolated vertices up to n_new (ldl_grow)."""
        self._check(load().ldl_grow(self._h, int(n_new)))
        self.n = int(n_new)

    def close(self):
        if getattr(self, "_h", None):
            load().ldl_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != LDL_OK:
            raise LdlError(st, load().ldl_last_error(self._h).decode())

    def apply(self, batch, on_device: bool = False) -> ldl_result:
        """Apply one batch: an int32 array of shape (count, 4) = (src, dst, op, w),
        host (numpy) or device (torch CUDA tensor with on_device=True)."""
        if hasattr(batch, "data_ptr"):  # a torch tensor, host (pinned) or device
            cnt = int(batch.shape[0])
            ptr = _ptr(batch)
            on_device = bool(batch.is_cuda)
        elif on_device:
            raise ValueError("on_device needs a CUDA tensor")
        else:
            batch = np.ascontiguousarray(batch, dtype=np.int32).reshape(-1, 4)
            cnt = batch.shape[0]
            ptr = _ptr(batch)
        self._check(load().ldl_apply_batch(self._h, ptr, cnt, int(on_device), C.byref(self.last)))
        return self.last

    def try_apply(self, batch) -> int:
        batch = np.ascontiguousarray(batch, dtype=np.int32).reshape(-1, 4)
        return int(load().ldl_apply_batch(self._h, _ptr(batch), batch.shape[0], 0, C.byref(self.last)))

    def modularity(self) -> float:
        q = C.c_double()
        self._check(load().ldl_modularity(self._h, C.byref(q)))
        return q.value

    def numerator(self):
        hi, lo, m = C.c_int64(), C.c_uint64(), C.c_int64()
        self._check(load().ldl_modularity_num(self._h, C.byref(hi), C.byref(lo), C.byref(m)))
        return int(m.value), (int(hi.value) << 64) + int(lo.value)

    @property
    def levels(self) -> int:
        return int(load().ldl_levels(self._h))

    @property
    def top(self) -> int:
        return self.levels - 1

    def level(self, r: int) -> Level:
        n = self.n
        a = [np.zeros(n, np.int32), np.zeros(n, np.int32), np.zeros(n, np.int64),
             np.zeros(n, np.int64), np.zeros(n, np.int32), np.zeros(n, np.uint8)]
        self._check(load().ldl_get_level(self._h, r, *[_ptr(x) for x in a]))
        return Level(*a)

    def labels(self) -> np.ndarray:
        return self.level(0).lab

    def level_adj(self, r: int):
        nnz = C.c_int64()
        self._check(load().ldl_level_nnz(self._h, r, C.byref(nnz)))
        rp = np.zeros(self.n + 1, np.int64)
        col = np.zeros(nnz.value, np.int32)
        w = np.zeros(nnz.value, np.int64)
        self._check(load().ldl_get_adjacency(self._h, r, _ptr(rp), _ptr(col), _ptr(w)))
        return rp, col, w

    def comm(self):
        a = [np.zeros(self.n, np.int64) for _ in range(3)]
        self._check(load().ldl_get_communities(self._h, *[_ptr(x) for x in a]))
        return tuple(a)

    def set_timing(self, on: bool = True):
        self._check(load().ldl_set_timing(self._h, int(on)))

    def stage_times(self) -> dict:
        t = np.zeros(16, np.float64)
        self._check(load().ldl_stage_times(self._h, _ptr(t)))
        return dict(zip(STAGES, t.tolist()))

    def changed(self):
        """(ids, labels) of the vertices whose label changed in the last batch."""
        k = int(self.last.n_changed)
        ids = np.zeros(k, np.int32)
        lab = np.zeros(k, np.int32)
        self._check(load().ldl_copy_changed(self._h, _ptr(ids), _ptr(lab)))
        return ids, lab

    def changed_noalloc(self):
        """As changed(), through the allocation-free entry point."""
        k = int(self.last.n_changed)
        ids = np.zeros(k, np.int32)
        lab = np.zeros(k, np.int32)
        self._check(load().ldl_copy_changed_noalloc(self._h, _ptr(ids), _ptr(lab)))
        return ids, lab

    def debug_decouple(self, v, src, dst, gains) -> np.ndarray:
        """Runs the device decoupling filter on explicit candidates (gains are
        Python ints up to 127 bits); returns the 0/1 accepted mask."""
        v = np.ascontiguousarray(v, dtype=np.int32)
        src = np.ascontiguousarray(src, dtype=np.int32)
        dst = np.ascontiguousarray(dst, dtype=np.int32)
        g = [int(x) for x in gains]
        hi = np.array([x >> 64 for x in g], dtype=np.int64)
        lo = np.array([x & ((1 << 64) - 1) for x in g], dtype=np.uint64)
        out = np.zeros(len(v), np.uint8)
        self._check(load().ldl_debug_decouple(self._h, len(v), _ptr(v), _ptr(src), _ptr(dst), _ptr(hi), _ptr(lo),
                                              _ptr(out)))
        return out

    def debug_sort_pairs(self, keys, vals, bits: int):
        """Sorts (key, value) pairs on the device, stably by the low `bits`
        key bits; returns the sorted copies."""
        k = np.array(keys, dtype=np.uint64, copy=True)
        v = np.array(vals, dtype=np.uint64, copy=True)
        self._check(load().ldl_debug_sort_pairs(self._h, len(k), _ptr(k), _ptr(v), bits))
        return k, v

    def hierarchy(self):
        """Per level r of the last result: (parent, comm, refined, alive) copied
        from the device pointers that ldl_apply_batch returned."""
        import torch

        r = self.last
        n = self.n
        out = []

        class _Dev:
            def __init__(self, ptr, typestr):
                self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False),
                                                 "version": 2}

        def rd(arr, k, typestr):
            ptr = C.cast(arr, C.POINTER(C.c_void_p))[k]
            return torch.as_tensor(_Dev(ptr, typestr), device="cuda").cpu().numpy().copy()

        for k in range(r.levels):
            out.append(dict(parent=rd(r.parent, k, "<i4"), comm=rd(r.comm, k, "<i4"),
                            refined=rd(r.refined, k, "<i4"), alive=rd(r.alive, k, "|u1")))
        return out

    def set_kernel_stats(self, on: bool = True):
        self._check(load().ldl_set_kernel_stats(self._h, int(on)))

    def kernel_stats(self) -> dict:
        t = np.zeros(4 * len(SWEEP_GROUPS), np.float64)
        self._check(load().ldl_get_kernel_stats(self._h, _ptr(t)))
        out = {}
        for k, name in enumerate(SWEEP_GROUPS):
            out[name] = dict(launches=t[4 * k], ms=t[4 * k + 1], bytes=t[4 * k + 2], entries=t[4 * k + 3])
        return out

    def result_dict(self) -> dict:
        r = self.last
        return dict(n_changed=r.n_changed, levels=r.levels, frontier_nodes=list(r.frontier_nodes),
                    edges_scanned=r.edges_scanned, moves=r.moves, refine_moves=r.refine_moves,
                    rejected=r.rejected, rollbacks=r.rollbacks, rounds=r.rounds,
                    agg_records=r.agg_records, decouple_rounds=r.decouple_rounds,
                    host_syncs=r.host_syncs, pending_records=r.pending_records,
                    pending_applied=r.pending_applied, split_members=r.split_members)


def apply_batches(instances, batches, threads: int = 0):
    """Batched form: one batch per instance, applied concurrently.  Returns
    the per-instance statuses (raises on the first failure)."""
    g = len(instances)
    arrs = [np.ascontiguousarray(b, dtype=np.int32).reshape(-1, 4) for b in batches]
    ctxs = (C.c_void_p * g)(*[d._h.value for d in instances])
    ptrs = (C.c_void_p * g)(*[a.ctypes.data for a in arrs])
    counts = (C.c_int64 * g)(*[a.shape[0] for a in arrs])
    st = (C.c_int32 * g)()
    res = (ldl_result * g)()
    rc = load().ldl_apply_batches(ctxs, ptrs, counts, g, 0, threads, st, res)
    for d, r in zip(instances, res):
        d.last = r
    if rc != LDL_OK:
        i = next(k for k in range(g) if st[k] != LDL_OK)
        raise LdlError(rc, load().ldl_last_error(instances[i]._h).decode())
    return list(st)


class Server:
    """Served form: a native request server (ldl_server_*)."""

    def __init__(self, workers: int = 4):
        h = C.c_void_p()
        st = load().ldl_server_create(workers, C.byref(h))
        if st != LDL_OK:
            raise LdlError(st, "server create")
        self._h = h

    def admit(self, g, **kw) -> LDL:
        return LDL(g.n, g.row_ptr, g.col, g.w, directed=g.directed, server=self, **kw)

    def submit(self, inst: LDL, batch) -> int:
        b = np.ascontiguousarray(batch, dtype=np.int32).reshape(-1, 4)
        t = C.c_int64()
        st = load().ldl_server_submit(self._h, inst._h, _ptr(b), b.shape[0], C.byref(t))
        if st != LDL_OK:
            raise LdlError(st, "submit")
        return int(t.value)

    def wait(self, ticket: int, timeout_ms: int = -1):
        st, res = C.c_int32(), ldl_result()
        q, sv = C.c_double(), C.c_double()
        rc = load().ldl_server_wait(self._h, ticket, timeout_ms, C.byref(st), C.byref(res), C.byref(q), C.byref(sv))
        if rc != LDL_OK:
            raise LdlError(rc, "wait")
        return int(st.value), res, q.value, sv.value

    def stats(self):
        """(deferred, retried): requests deferred for memory, and requests
        rolled back after running out of memory and queued again."""
        a, b = C.c_int64(), C.c_int64()
        st = load().ldl_server_stats(self._h, C.byref(a), C.byref(b))
        if st != LDL_OK:
            raise LdlError(st, "stats")
        return int(a.value), int(b.value)

    def debug_free_bytes(self, nbytes: int):
        """Test hook: admission treats `nbytes` as the device's free memory
        (-1: ask the device)."""
        load().ldl_server_debug_free_bytes(self._h, int(nbytes))

    def close(self):
        if getattr(self, "_h", None):
            load().ldl_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
