"""Python binding of libflgpu (GB300 graph facility location).

Argument marshalling over the C ABI of ``include/fl.h`` only: every step of the
path runs in the library's CUDA kernels.  Arrays may be NumPy arrays (host
memory) or CUDA ``torch.Tensor`` objects (device memory); PyTorch provides
device memory and streams.  If the library cannot be loaded this module raises:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
_lock = threading.Lock()
_lib = None

FL_OK, FL_EINVAL, FL_ESTATE, FL_ENOMEM, FL_ECUDA, FL_ETIMEOUT = range(6)
FL_MEM_HOST, FL_MEM_DEVICE = 0, 1

EXPORTS = ("fl_graph_create", "fl_graph_create_weighted", "fl_graph_destroy", "fl_build_sketches", "fl_sketch_stats",
           "fl_export_sketches", "fl_export_ads", "fl_solve_create", "fl_solve_destroy",
           "fl_compute_radii", "fl_open_facilities", "fl_assign_clients", "fl_objective",
           "fl_solve_stats", "fl_mis_log", "fl_status_str", "fl_last_error", "fl_profile_enable", "fl_profile_reset",
           "fl_profile_query", "fl_hop_stats", "fl_hop_model", "fl_batch_create_union", "fl_batch_create_replicas",
           "fl_batch_solve", "fl_batch_info", "fl_batch_destroy", "fl_assign_nearest_noalloc",
           "fl_ball_sizes", "fl_ball_estimates", "fl_compute_radii_exact", "fl_open_facilities_eps",
           "fl_eps_stats", "fl_get_schedule", "fl_set_schedule", "fl_autotune", "fl_autotune_forget",
           "fl_batch_set_schedule")

PROF_CLASSES = {"sketch_merge": 0, "sketch_expand": 1, "sketch_other": 2, "radius": 3, "keys": 4,
                "mis": 5, "bfs": 6, "other": 7, "exact": 8}


class Schedule(ctypes.Structure):
    """fl_schedule: launch and round-switch parameters (never results)."""
    _fields_ = [("hop_group", ctypes.c_int32), ("sparse_div", ctypes.c_int32), ("dense_div", ctypes.c_int32),
                ("edge_div", ctypes.c_int32), ("graph_bfs", ctypes.c_int32), ("level_cap", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class FLError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"[{status}] {msg}")
        self.status = status


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libflgpu.so (building it when missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise OSError(f"libflgpu.so not found at {_build.LIB}; run build()")
        lib = ctypes.CDLL(_build.LIB)
        i64, u64, vp, ci = ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int
        P64 = ctypes.POINTER(i64)
        sig = {
            "fl_graph_create": ([i64, vp, vp, i64, ci, vp, ctypes.POINTER(vp)], ci),
            "fl_graph_create_weighted": ([i64, vp, vp, vp, i64, ci, vp, ctypes.POINTER(vp)], ci),
            "fl_graph_destroy": ([vp], ci),
            "fl_build_sketches": ([vp, ci, u64], ci),
            "fl_sketch_stats": ([vp, P64, P64, P64, P64], ci),
            "fl_export_sketches": ([vp, vp, vp, ci], ci),
            "fl_export_ads": ([vp, vp, vp, vp, vp, vp, vp, vp, ci], ci),
            "fl_solve_create": ([vp, ctypes.POINTER(vp)], ci),
            "fl_solve_destroy": ([vp], ci),
            "fl_compute_radii": ([vp, vp, vp, ci, vp], ci),
            "fl_open_facilities": ([vp, vp, P64, ci], ci),
            "fl_assign_clients": ([vp, vp, vp, ci], ci),
            "fl_objective": ([vp, ctypes.POINTER(ctypes.c_double), P64, P64], ci),
            "fl_solve_stats": ([vp, P64, P64], ci),
            "fl_mis_log": ([vp, i64, P64, vp], ci),
            "fl_status_str": ([ci], ctypes.c_char_p),
            "fl_last_error": ([ctypes.c_char_p, ctypes.c_size_t], ci),
            "fl_profile_enable": ([vp, ci], ci),
            "fl_profile_reset": ([vp], ci),
            "fl_profile_query": ([vp, ci, P64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], ci),
            "fl_hop_stats": ([vp, i64, P64, vp, vp, vp, vp], ci),
            "fl_hop_model": ([vp, i64, P64, vp, vp, vp, vp, vp], ci),
            "fl_batch_create_union": ([ci, vp, vp, vp, vp, ci, vp, ctypes.POINTER(vp)], ci),
            "fl_batch_create_replicas": ([vp, ci, vp, ctypes.POINTER(vp)], ci),
            "fl_batch_solve": ([vp, ci, ci, u64, vp, vp, vp, vp, vp, vp, vp, vp, vp, ci], ci),
            "fl_batch_info": ([vp, P64, P64], ci),
            "fl_batch_destroy": ([vp], ci),
            "fl_assign_nearest_noalloc": ([i64, vp, vp, i64, vp, vp, vp, vp], ci),
            "fl_ball_sizes": ([vp, i64, vp, ctypes.c_int32, vp, ci, vp], ci),
            "fl_ball_estimates": ([vp, i64, vp, ctypes.c_int32, vp, ci, vp], ci),
            "fl_compute_radii_exact": ([vp, vp, vp, ci, vp], ci),
            "fl_open_facilities_eps": ([vp, ctypes.c_double, vp, vp, ci, vp, P64, vp, vp], ci),
            "fl_eps_stats": ([vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), P64, P64,
                              P64], ci),
            "fl_get_schedule": ([vp, ctypes.POINTER(Schedule)], ci),
            "fl_set_schedule": ([vp, ctypes.POINTER(Schedule)], ci),
            "fl_autotune": ([vp, ci, u64, vp, vp, ci, ci, ctypes.POINTER(Schedule), ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_double)], ci),
            "fl_autotune_forget": ([], ci),
            "fl_batch_set_schedule": ([vp, ctypes.POINTER(Schedule)], ci),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(rc: int):
    if rc != FL_OK:
        lib = load(False)
        buf = ctypes.create_string_buffer(1024)
        lib.fl_last_error(buf, 1024)
        raise FLError(rc, f"{lib.fl_status_str(rc).decode()}: {buf.value.decode(errors='replace')}")


def _arg(a, dtype=None):
    """(pointer, mem_kind, keepalive) for a NumPy array or a CUDA tensor; None -> NULL."""
    if a is None:
        return None, None, None
    if isinstance(a, np.ndarray):
        if dtype is not None and a.dtype != dtype:
            raise TypeError(f"expected {np.dtype(dtype)}, got {a.dtype}")
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data_as(ctypes.c_void_p), FL_MEM_HOST, a
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(a, torch.Tensor):
        if dtype is not None and _TORCH_DTYPES.get(a.dtype) != np.dtype(dtype):
            raise TypeError(f"expected {np.dtype(dtype)}, got {a.dtype}")
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        kind = FL_MEM_DEVICE if a.is_cuda else FL_MEM_HOST
        return ctypes.c_void_p(a.data_ptr()), kind, a
    raise TypeError(f"unsupported array type {type(a)}")


def _torch_dtypes():
    try:
        import torch
    except ImportError:  # pragma: no cover
        return {}
    return {torch.int64: np.dtype(np.int64), torch.int32: np.dtype(np.int32), torch.uint8: np.dtype(np.uint8),
            torch.bool: np.dtype(np.bool_), torch.float64: np.dtype(np.float64), torch.uint64: np.dtype(np.uint64)}


_TORCH_DTYPES = _torch_dtypes()


def _kind(*kinds):
    ks = {k for k in kinds if k is not None}
    if len(ks) > 1:
        raise ValueError("all arrays of one call must live in the same memory (host or device)")
    return ks.pop() if ks else FL_MEM_HOST


class Graph:
    """fl_graph: a CSR graph on the device with its sketches and ADS."""

    def __init__(self, rowp, cols, stream=None, lengths=None):
        """lengths: int32 edge length per CSR entry (a weighted graph, see
        fl_graph_create_weighted), or None."""
        self._lib = load()
        p_r, k_r, _ = _arg(rowp, np.int64)
        p_c, k_c, _ = _arg(cols, np.int32)
        self.n = int(len(rowp) - 1)
        self.nnz = int(len(cols))
        st = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0))
        h = ctypes.c_void_p()
        self.weighted = lengths is not None
        if lengths is None:
            kind = _kind(k_r, k_c)
            _check(self._lib.fl_graph_create(self.n, p_r, p_c, self.nnz, kind, st, ctypes.byref(h)))
        else:
            if len(lengths) != len(cols):
                raise ValueError("lengths must have one entry per CSR column")
            p_w, k_w, _ = _arg(lengths, np.int32)
            kind = _kind(k_r, k_c, k_w)
            _check(self._lib.fl_graph_create_weighted(self.n, p_r, p_c, p_w, self.nnz, kind, st, ctypes.byref(h)))
        self._h = h
        self.k = None
        self.seed = None

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fl_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build_sketches(self, k: int, seed: int):
        _check(self._lib.fl_build_sketches(self._h, k, seed))
        self.k, self.seed = k, seed

    def stats(self) -> dict:
        v = [ctypes.c_int64() for _ in range(4)]
        _check(self._lib.fl_sketch_stats(self._h, *[ctypes.byref(x) for x in v]))
        return dict(hops=v[0].value, edge_merges=v[1].value, ads_entries=v[2].value, ads_groups=v[3].value)

    def hop_stats(self) -> list:
        """Per processed hop of the last build (the last one changed no sketch):
        vertices changed; CSR entries scanned, of them by the mask merge, and
        kernel ms (these three 0 unless profiling was on)."""
        H = ctypes.c_int64()
        _check(self._lib.fl_hop_stats(self._h, 0, ctypes.byref(H), None, None, None, None))
        h = H.value
        sc, mk, ch = (np.zeros(h, np.int64) for _ in range(3))
        ms = np.zeros(h, np.float64)
        _check(self._lib.fl_hop_stats(self._h, h, ctypes.byref(H), sc.ctypes.data_as(ctypes.c_void_p),
                                      mk.ctypes.data_as(ctypes.c_void_p), ch.ctypes.data_as(ctypes.c_void_p),
                                      ms.ctypes.data_as(ctypes.c_void_p)))
        return [dict(hop=i + 1, scanned=int(sc[i]), mask=int(mk[i]), changed=int(ch[i]), ms=float(ms[i]))
                for i in range(h)]

    @property
    def schedule(self) -> dict:
        sc = Schedule()
        _check(self._lib.fl_get_schedule(self._h, ctypes.byref(sc)))
        return sc.as_dict()

    def set_schedule(self, **kw):
        sc = Schedule(**{**self.schedule, **kw})
        _check(self._lib.fl_set_schedule(self._h, ctypes.byref(sc)))

    def autotune(self, k: int, seed: int, cost, client, max_trials: int = 16) -> dict:
        """Pick this graph's schedule for k by timing the path (see fl_autotune)."""
        p_c, k_c, _ = _arg(cost, np.float64)
        p_m, k_m, _ = _arg(client, np.uint8)
        sc, d, t = Schedule(), ctypes.c_double(), ctypes.c_double()
        _check(self._lib.fl_autotune(self._h, int(k), int(seed), p_c, p_m, _kind(k_c, k_m), int(max_trials),
                                     ctypes.byref(sc), ctypes.byref(d), ctypes.byref(t)))
        self.k, self.seed = k, seed
        return dict(schedule=sc.as_dict(), ms_default=d.value, ms_tuned=t.value)

    def hop_model(self) -> list:
        """Per hop of the last build: edge-merges E, merging vertices A,
        neighbour-delta ranks read, sum of |D_{h-1}(u)| over the edge-merges,
        new entries (the terms of the algorithmic-bytes model of a hop)."""
        H = ctypes.c_int64()
        _check(self._lib.fl_hop_model(self._h, 0, ctypes.byref(H), None, None, None, None, None))
        h = H.value
        cols = [np.zeros(h, np.int64) for _ in range(5)]
        _check(self._lib.fl_hop_model(self._h, h, ctypes.byref(H), *[c.ctypes.data_as(ctypes.c_void_p) for c in cols]))
        names = ("edge_merges", "merging", "delta_read", "delta_sum", "new_entries")
        return [dict(hop=i + 1, **{nm: int(c[i]) for nm, c in zip(names, cols)}) for i in range(h)]

    def profile(self, on: bool = True, census: bool = False):
        """CUDA-event timing of launches; census adds the per-hop counts of
        the sketch build (extra kernels, see fl_hop_stats)."""
        _check(self._lib.fl_profile_enable(self._h, (2 if census else 1) if on else 0))

    def profile_reset(self):
        _check(self._lib.fl_profile_reset(self._h))

    def profile_query(self, kernel_class=-1) -> dict:
        """Launches, kernel milliseconds and algorithmic bytes of one class (name or id)."""
        c = PROF_CLASSES[kernel_class] if isinstance(kernel_class, str) else int(kernel_class)
        l, ms, b = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
        _check(self._lib.fl_profile_query(self._h, c, ctypes.byref(l), ctypes.byref(ms), ctypes.byref(b)))
        return dict(launches=l.value, ms=ms.value, alg_bytes=b.value)

    def _ball_query(self, fn, dtype, src, max_dist, pred, out):
        p_s, k_s, _ = _arg(src, np.int32)
        p_p, k_p, _ = _arg(pred, np.uint8)
        n_src = len(src)
        if out is None and k_s != FL_MEM_DEVICE:
            out = np.zeros((n_src, max_dist + 1), dtype)
        p_o, k_o, _ = _arg(out)
        _check(fn(self._h, n_src, p_s, int(max_dist), p_p, _kind(k_s, k_p, k_o), p_o))
        return out

    def ball_sizes(self, src, max_dist: int, pred=None, out=None):
        """Exact |{w : d(v, w) <= h, pred[w]}| for v in src and h = 0..max_dist
        (int64, one row per source) by bit-parallel BFS (Section 5.1, Fig. 1)."""
        return self._ball_query(self._lib.fl_ball_sizes, np.int64, src, max_dist, pred, out)

    def ball_estimates(self, src, max_dist: int, pred=None, out=None):
        """HIP estimates of the same sizes from the ADS (float64 rows)."""
        return self._ball_query(self._lib.fl_ball_estimates, np.float64, src, max_dist, pred, out)

    def export_sketches(self):
        S = np.zeros((self.n, self.k), np.uint64)
        cnt = np.zeros(self.n, np.int32)
        _check(self._lib.fl_export_sketches(self._h, _arg(S)[0], _arg(cnt)[0], FL_MEM_HOST))
        return S, cnt

    def export_ads(self) -> dict:
        st = self.stats()
        ng, ne = st["ads_groups"], st["ads_entries"]
        out = dict(gofs=np.zeros(self.n + 1, np.int64), eofs=np.zeros(self.n + 1, np.int64),
                   ghop=np.zeros(ng, np.int32), gcnt=np.zeros(ng, np.int32),
                   gcounted=np.zeros(ng, np.int32), gwt=np.zeros(ng, np.float64),
                   eid=np.zeros(ne, np.int32))
        _check(self._lib.fl_export_ads(self._h, *[_arg(out[k])[0] for k in
                                                  ("gofs", "eofs", "ghop", "gcnt", "gcounted", "gwt", "eid")],
                                       FL_MEM_HOST))
        return out


class Solve:
    """fl_solve: one facility-location instance on a built graph."""

    def __init__(self, graph: Graph):
        self._lib = load()
        self.graph = graph
        h = ctypes.c_void_p()
        _check(self._lib.fl_solve_create(graph.handle, ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fl_solve_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def compute_radii(self, cost, client, radii_out=None):
        """Phase (ii).  Returns radii_out (allocated on the host when None)."""
        p_c, k_c, _ = _arg(cost, np.float64)
        p_m, k_m, _ = _arg(client, np.uint8)
        if radii_out is None and k_c != FL_MEM_DEVICE:
            radii_out = np.zeros(self.graph.n, np.float64)
        p_r, k_r, _ = _arg(radii_out)
        _check(self._lib.fl_compute_radii(self._h, p_c, p_m, _kind(k_c, k_m, k_r), p_r))
        return radii_out

    def compute_radii_exact(self, cost, client, radii_out=None):
        """Phase (ii) with exact client counts per distance (BFS) in place of
        the HIP estimates; the later phases then use these radii."""
        p_c, k_c, _ = _arg(cost, np.float64)
        p_m, k_m, _ = _arg(client, np.uint8)
        if radii_out is None and k_c != FL_MEM_DEVICE:
            radii_out = np.zeros(self.graph.n, np.float64)
        p_r, k_r, _ = _arg(radii_out)
        _check(self._lib.fl_compute_radii_exact(self._h, p_c, p_m, _kind(k_c, k_m, k_r), p_r))
        return radii_out

    def open_facilities_eps(self, eps: float, cost, client, open_out=None, fac_iter_out=None, cli_iter_out=None):
        """The opening phase with eps > 0 and the selection of Algorithm 6.
        Returns (open mask, number opened, opening iterations, freezing
        iterations); outputs are allocated on the host when not given and the
        inputs are host arrays."""
        p_c, k_c, _ = _arg(cost, np.float64)
        p_m, k_m, _ = _arg(client, np.uint8)
        if k_c != FL_MEM_DEVICE:
            n = self.graph.n
            open_out = np.zeros(n, np.uint8) if open_out is None else open_out
            fac_iter_out = np.zeros(n, np.int32) if fac_iter_out is None else fac_iter_out
            cli_iter_out = np.zeros(n, np.int32) if cli_iter_out is None else cli_iter_out
        p_o, k_o, _ = _arg(open_out, np.uint8)
        p_f, k_f, _ = _arg(fac_iter_out, np.int32)
        p_i, k_i, _ = _arg(cli_iter_out, np.int32)
        nopen = ctypes.c_int64()
        _check(self._lib.fl_open_facilities_eps(self._h, float(eps), p_c, p_m, _kind(k_c, k_m, k_o, k_f, k_i), p_o,
                                                ctypes.byref(nopen), p_f, p_i))
        return open_out, nopen.value, fac_iter_out, cli_iter_out

    def eps_stats(self) -> dict:
        g, a = ctypes.c_double(), ctypes.c_double()
        it, ev, gr = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(self._lib.fl_eps_stats(self._h, ctypes.byref(g), ctypes.byref(a), ctypes.byref(it), ctypes.byref(ev),
                                      ctypes.byref(gr)))
        return dict(gamma=g.value, alpha0=a.value, iterations=it.value, events=ev.value, groups=gr.value)

    def open_facilities(self, open_out=None):
        """Phase (iii).  Returns (open mask, number opened)."""
        if open_out is None:
            open_out = np.zeros(self.graph.n, np.uint8)
        p, k, _ = _arg(open_out)
        nopen = ctypes.c_int64()
        _check(self._lib.fl_open_facilities(self._h, p, ctypes.byref(nopen), k))
        return open_out, nopen.value

    def assign_clients(self, assign_out=None, dist_out=None):
        if assign_out is None and dist_out is None:
            assign_out = np.zeros(self.graph.n, np.int32)
            dist_out = np.zeros(self.graph.n, np.int32)
        pa, ka, _ = _arg(assign_out)
        pd, kd, _ = _arg(dist_out)
        _check(self._lib.fl_assign_clients(self._h, pa, pd, _kind(ka, kd)))
        return assign_out, dist_out

    def objective(self):
        obj, ds, un = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
        _check(self._lib.fl_objective(self._h, ctypes.byref(obj), ctypes.byref(ds), ctypes.byref(un)))
        return obj.value, ds.value, un.value

    def stats(self) -> dict:
        r, c = ctypes.c_int64(), ctypes.c_int64()
        _check(self._lib.fl_solve_stats(self._h, ctypes.byref(r), ctypes.byref(c)))
        return dict(mis_rounds=r.value, candidates=c.value)

    def mis_log(self) -> np.ndarray:
        """Rounds of the last greedy MIS: int64 rows (greedy round, kind,
        step, frontier, pulled, microseconds); kinds as fl_mis_log."""
        n = ctypes.c_int64()
        _check(self._lib.fl_mis_log(self._h, 0, ctypes.byref(n), None))
        rows = np.zeros((n.value, 6), dtype=np.int64)
        if n.value:
            _check(self._lib.fl_mis_log(self._h, n.value, ctypes.byref(n), rows.ctypes.data_as(ctypes.c_void_p)))
        return rows


class Batch:
    """fl_batch: many instances solved in one pass (see include/fl.h).

    Batch.union(graphs) -- independent graphs [(rowp, cols), ...], one
    instance each; Batch.replicas(graph, n_inst) -- n_inst instances on one
    resident graph with built sketches.  solve() takes the instances' costs
    and client masks concatenated (instance-major)."""

    def __init__(self, handle, keep=None):
        self._lib = load()
        self._h = handle
        self._keep = keep
        n_inst, n_total = ctypes.c_int64(), ctypes.c_int64()
        _check(self._lib.fl_batch_info(self._h, ctypes.byref(n_inst), ctypes.byref(n_total)))
        self.n_inst, self.n_total = n_inst.value, n_total.value

    @classmethod
    def union(cls, graphs, stream=None):
        lib = load()
        ptr_r, ptr_c, kinds, keep = [], [], [], []
        n_of = np.array([len(r) - 1 for r, _ in graphs], np.int64)
        nnz_of = np.array([len(c) for _, c in graphs], np.int64)
        for r, c in graphs:
            pr, kr, a = _arg(r, np.int64)
            pc, kc, b = _arg(c, np.int32)
            ptr_r.append(pr.value or 0)
            ptr_c.append(pc.value or 0)
            kinds += [kr, kc]
            keep += [a, b]
        kind = _kind(*kinds)
        R = (ctypes.c_void_p * len(graphs))(*ptr_r)
        C = (ctypes.c_void_p * len(graphs))(*ptr_c)
        st = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0))
        h = ctypes.c_void_p()
        _check(lib.fl_batch_create_union(len(graphs), n_of.ctypes.data_as(ctypes.c_void_p),
                                         nnz_of.ctypes.data_as(ctypes.c_void_p), R, C, kind, st, ctypes.byref(h)))
        return cls(h)

    @classmethod
    def replicas(cls, graph, n_inst: int, stream=None):
        lib = load()
        st = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0))
        h = ctypes.c_void_p()
        _check(lib.fl_batch_create_replicas(graph.handle, int(n_inst), st, ctypes.byref(h)))
        b = cls(h, keep=graph)
        b.n_per = graph.n
        return b

    def solve(self, k: int, seed: int, cost, client, open_out=None, assign_out=None, dist_out=None,
              n_active=None) -> dict:
        """Solve the first n_active instances (default all; fewer only for a
        replica batch).  Per-vertex outputs (host NumPy arrays unless given)
        and per-instance n_open, objective, dist_sum, n_unserved."""
        I = self.n_inst if n_active is None else int(n_active)
        N = self.n_total if I == self.n_inst else I * self.n_per
        if open_out is None and assign_out is None and dist_out is None and isinstance(cost, np.ndarray):
            open_out = np.zeros(N, np.uint8)
            assign_out = np.zeros(N, np.int32)
            dist_out = np.zeros(N, np.int32)
        pc, kc, _ = _arg(cost, np.float64)
        pm, km, _ = _arg(client, np.uint8)
        po, ko, _ = _arg(open_out, np.uint8)
        pa, ka, _ = _arg(assign_out, np.int32)
        pd, kd, _ = _arg(dist_out, np.int32)
        kind = _kind(kc, km, ko, ka, kd)
        n_open = np.zeros(I, np.int64)
        obj = np.zeros(I, np.float64)
        ds = np.zeros(I, np.int64)
        un = np.zeros(I, np.int64)
        _check(self._lib.fl_batch_solve(self._h, I, int(k), int(seed), pc, pm, po, pa, pd,
                                        n_open.ctypes.data_as(ctypes.c_void_p), obj.ctypes.data_as(ctypes.c_void_p),
                                        ds.ctypes.data_as(ctypes.c_void_p), un.ctypes.data_as(ctypes.c_void_p), kind))
        return dict(open=open_out, assign=assign_out, dist=dist_out, n_open=n_open, objective=obj, dist_sum=ds,
                    n_unserved=un)

    def set_schedule(self, schedule: dict):
        sc = Schedule(**schedule)
        _check(self._lib.fl_batch_set_schedule(self._h, ctypes.byref(sc)))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fl_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def assign_nearest_noalloc(rowp, cols, open_mask, assign_out, dist_out, stream=None):
    """fl_assign_nearest_noalloc: nearest open facility with no device allocation.

    For callers that cannot let the library allocate device memory; all arrays are
    CUDA tensors the caller owns, on the current device: row offsets int64[n+1],
    columns int32[nnz] with nnz = row offsets[-1], open mask uint8 or bool [n],
    outputs int32[n] (either may be None).  Graphs up to 2^20 vertices; calls that
    overlap on the GPU race.  Types, lengths and devices are checked here, before
    anything is launched.
    """
    import torch

    lib = load()
    n = len(rowp) - 1
    want = ((rowp, "row offsets", (torch.int64,), n + 1), (cols, "columns", (torch.int32,), None),
            (open_mask, "open mask", (torch.uint8, torch.bool), n), (assign_out, "assign_out", (torch.int32,), n),
            (dist_out, "dist_out", (torch.int32,), n))
    for a, what, dtypes, length in want:
        if a is None:
            if what in ("assign_out", "dist_out"):
                continue
            raise ValueError(f"{what} is required")
        if not isinstance(a, torch.Tensor):
            raise TypeError(f"{what} must be a torch.Tensor in device memory")
        if a.dtype not in dtypes:
            raise TypeError(f"{what}: expected {' or '.join(str(d) for d in dtypes)}, got {a.dtype}")
        if a.dim() != 1 or not a.is_contiguous():
            raise ValueError(f"{what} must be a contiguous 1-D tensor")
        if length is not None and a.numel() != length:
            raise ValueError(f"{what} has {a.numel()} elements, expected {length}")
    if assign_out is None and dist_out is None:
        raise ValueError("at least one of assign_out, dist_out is required")
    for a, what, _, _ in want:
        if a is not None and not a.is_cuda:
            raise ValueError(f"{what} must be in device memory")
    dev = torch.cuda.current_device()
    for a, what, _, _ in want:
        if a is not None and a.device.index != dev:
            raise ValueError(f"{what} is on cuda:{a.device.index}, the current device is cuda:{dev}")
    nnz = int(rowp[-1].item()) if n >= 0 else 0
    if nnz != cols.numel():
        raise ValueError(f"row offsets end at {nnz} but there are {cols.numel()} columns")
    ptr = [ctypes.c_void_p(a.data_ptr()) if a is not None else None
           for a in (rowp, cols, open_mask, assign_out, dist_out)]
    st = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0))
    _check(lib.fl_assign_nearest_noalloc(n, ptr[0], ptr[1], cols.numel(), ptr[2], ptr[3], ptr[4], st))
    return assign_out, dist_out


def solve(rowp, cols, k, seed, cost, client, stream=None) -> dict:
    """The whole path through the C ABI with host arrays; returns every output."""
    g = Graph(rowp, cols, stream)
    g.build_sketches(k, seed)
    s = Solve(g)
    r = s.compute_radii(cost, client)
    op, nopen = s.open_facilities()
    a, d = s.assign_clients()
    obj, ds, un = s.objective()
    return dict(graph=g, solve=s, stats=g.stats(), radii=r, open=op, n_open=nopen, assign=a, dist=d,
                objective=obj, dist_sum=ds, n_unserved=un, mis=s.stats())


def solve_eps(rowp, cols, k, seed, eps, cost, client, stream=None) -> dict:
    """The eps > 0 path through the C ABI with host arrays: sketches, the
    opening phase and Algorithm 6, assignment, objective."""
    g = Graph(rowp, cols, stream)
    g.build_sketches(k, seed)
    s = Solve(g)
    op, nopen, fi, ci = s.open_facilities_eps(eps, cost, client)
    a, d = s.assign_clients()
    obj, ds, un = s.objective()
    return dict(graph=g, solve=s, open=op, n_open=nopen, fac_iter=fi, cli_iter=ci, assign=a, dist=d, objective=obj,
                dist_sum=ds, n_unserved=un, stats=s.eps_stats())


def autotune_forget():
    """Empty the autotuner's per-process cache."""
    _check(load().fl_autotune_forget())
