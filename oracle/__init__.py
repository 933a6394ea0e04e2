"""CPU oracle for the facility-location hot path -- TEST INFRASTRUCTURE.

A plain, slow implementation of the paper's definitions in C (``fl_oracle.c``),
loaded through ctypes.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the library under
``paper_1503_03635_gb300`` never does, and the two share no code.

Each wrapper names the passage of the paper it follows (see ``fl_oracle.c``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fl_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libfloracle.so")
_lock = threading.Lock()
_lib = None

i64, u64, i32, dbl, vp = (ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32,
                          ctypes.c_double, ctypes.c_void_p)


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, OpenMP, no FP contraction, no fast-math)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            lib.orc_splitmix64_next.restype = u64
            lib.orc_splitmix64_next.argtypes = [ctypes.POINTER(u64)]
            lib.orc_rank.restype = u64
            lib.orc_rank.argtypes = [u64, i64]
            lib.orc_priority.restype = u64
            lib.orc_priority.argtypes = [u64, i64]
            lib.orc_graph_create.restype = vp
            lib.orc_graph_create.argtypes = [i64, vp, vp]
            lib.orc_graph_destroy.restype = None
            lib.orc_graph_destroy.argtypes = [vp]
            lib.orc_build_sketches.restype = ctypes.c_int
            lib.orc_build_sketches.argtypes = [vp, ctypes.c_int, u64]
            lib.orc_build_sketches_hops.restype = ctypes.c_int
            lib.orc_build_sketches_hops.argtypes = [vp, ctypes.c_int, u64, i64]
            lib.orc_threads.restype = ctypes.c_int
            lib.orc_threads.argtypes = []
            for name in ("orc_hops", "orc_edge_merges", "orc_ads_groups", "orc_ads_entries"):
                getattr(lib, name).restype = i64
                getattr(lib, name).argtypes = [vp]
            lib.orc_export_sketch.restype = ctypes.c_int
            lib.orc_export_sketch.argtypes = [vp, vp, vp]
            lib.orc_export_ads.restype = ctypes.c_int
            lib.orc_export_ads.argtypes = [vp] + [vp] * 8
            lib.orc_vertex_ads.restype = i64
            lib.orc_vertex_ads.argtypes = [vp, ctypes.c_int, u64, i64, i64,
                                           vp, vp, vp, vp, vp, vp, ctypes.POINTER(i64)]
            lib.orc_compute_radii.restype = ctypes.c_int
            lib.orc_compute_radii.argtypes = [vp, vp, vp, vp]
            lib.orc_hip_estimate.restype = dbl
            lib.orc_hip_estimate.argtypes = [vp, i64, i64, vp]
            lib.orc_open_facilities.restype = ctypes.c_int
            lib.orc_open_facilities.argtypes = [vp, vp, vp, u64, vp, ctypes.POINTER(i64)]
            lib.orc_check_open_facilities.restype = ctypes.c_int
            lib.orc_check_open_facilities.argtypes = [vp, vp, vp, u64, vp, ctypes.POINTER(i64)]
            lib.orc_assign.restype = ctypes.c_int
            lib.orc_assign.argtypes = [vp, vp, vp, vp]
            lib.orc_radius_of_ads.restype = dbl
            lib.orc_radius_of_ads.argtypes = [i64, vp, vp, vp, vp, vp, vp, dbl]
            lib.orc_nearest_open.restype = ctypes.c_int
            lib.orc_nearest_open.argtypes = [vp, vp, i64, ctypes.POINTER(ctypes.c_int32),
                                             ctypes.POINTER(ctypes.c_int32)]
            lib.orc_ball_sizes.restype = ctypes.c_int
            lib.orc_ball_sizes.argtypes = [vp, i64, vp, i64, vp, vp]
            lib.orc_exact_radii.restype = ctypes.c_int
            lib.orc_exact_radii.argtypes = [vp, vp, vp, vp]
            lib.orc_exact_radii_of.restype = ctypes.c_int
            lib.orc_exact_radii_of.argtypes = [vp, i64, vp, vp, vp, vp]
            lib.orc_fl_optimum.restype = ctypes.c_int
            lib.orc_fl_optimum.argtypes = [vp, vp, vp, vp, ctypes.POINTER(dbl)]
            lib.orc_fl_local_search.restype = ctypes.c_int
            lib.orc_fl_local_search.argtypes = [vp, vp, vp, i64, vp, ctypes.POINTER(dbl), ctypes.POINTER(i64)]
            lib.orc_fl_cost.restype = dbl
            lib.orc_fl_cost.argtypes = [vp, vp, vp, vp]
            lib.orc_eps_gamma.restype = dbl
            lib.orc_eps_gamma.argtypes = [vp, vp, vp]
            lib.orc_eps_open.restype = ctypes.c_int
            lib.orc_eps_open.argtypes = [vp, dbl, vp, vp, ctypes.c_int, vp, vp, vp, ctypes.POINTER(dbl),
                                         ctypes.POINTER(dbl), ctypes.POINTER(i64)]
            lib.orc_eps_select.restype = ctypes.c_int
            lib.orc_eps_select.argtypes = [vp, dbl, dbl, vp, vp, u64, vp, ctypes.POINTER(i64)]
            lib.orc_graph_set_weights.restype = ctypes.c_int
            lib.orc_graph_set_weights.argtypes = [vp, vp]
            lib.orc_build_sketches_weighted.restype = ctypes.c_int
            lib.orc_build_sketches_weighted.argtypes = [vp, ctypes.c_int, u64]
            lib.orc_wads_rounds.restype = ctypes.c_int
            lib.orc_wads_rounds.argtypes = [vp, ctypes.c_int, u64, i64, vp, vp, vp,
                                            ctypes.POINTER(i64), ctypes.POINTER(i64)]
            lib.orc_open_facilities_weighted.restype = ctypes.c_int
            lib.orc_open_facilities_weighted.argtypes = [vp, vp, vp, u64, vp, ctypes.POINTER(i64)]
            lib.orc_assign_weighted.restype = ctypes.c_int
            lib.orc_assign_weighted.argtypes = [vp, vp, vp, vp]
            lib.orc_objective.restype = ctypes.c_int
            lib.orc_objective.argtypes = [i64, vp, vp, vp, vp, ctypes.POINTER(dbl),
                                          ctypes.POINTER(i64), ctypes.POINTER(i64)]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def splitmix64_outputs(state: int, count: int) -> list[int]:
    """The first `count` outputs of SplitMix64 from `state` (Steele et al. 2014)."""
    lib = _load()
    s = u64(state)
    return [int(lib.orc_splitmix64_next(ctypes.byref(s))) for _ in range(count)]


def threads() -> int:
    """OpenMP threads the oracle's parallel loops use."""
    return int(_load().orc_threads())


def rank(seed: int, v: int) -> int:
    """r(v): the hash of vertex v used by the bottom-k sketches (Algorithm 1)."""
    return int(_load().orc_rank(seed, v))


def ranks(seed: int, n: int) -> np.ndarray:
    lib = _load()
    return np.array([lib.orc_rank(seed, v) for v in range(n)], np.uint64)


def priority(seed: int, f: int) -> int:
    """pi(f): the random facility ID of the greedy MIS (Section 4.3)."""
    return int(_load().orc_priority(seed, f))


class Graph:
    """An oracle graph (copies the CSR) with its sketch/ADS state."""

    def __init__(self, rowp: np.ndarray, cols: np.ndarray):
        self._lib = _load()
        self.rowp = np.ascontiguousarray(rowp, np.int64)
        self.cols = np.ascontiguousarray(cols, np.int32)
        self.n = len(self.rowp) - 1
        self._h = self._lib.orc_graph_create(self.n, _p(self.rowp), _p(self.cols))
        if not self._h:
            raise MemoryError("orc_graph_create failed")
        self.k = None
        self.seed = None

    def close(self):
        if self._h:
            self._lib.orc_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- weighted graphs (NEXT f3): Section 3.3 after Algorithm 2 ----------
    def set_weights(self, w: np.ndarray) -> None:
        """Edge lengths, one positive integer per CSR entry, equal for (u, v)
        and (v, u) (Section 5 draws them uniformly in [1, 100])."""
        self.w = np.ascontiguousarray(w, np.int32)
        rc = self._lib.orc_graph_set_weights(self._h, _p(self.w))
        if rc != 0:
            raise ValueError(f"orc_graph_set_weights rc={rc}")

    def build_sketches_weighted(self, k: int, seed: int) -> None:
        """The ADS of every vertex by Algorithm 1 in Dijkstra order; groups
        are per distance ("ghop" holds the distance)."""
        rc = self._lib.orc_build_sketches_weighted(self._h, k, seed)
        if rc != 0:
            raise RuntimeError(f"orc_build_sketches_weighted rc={rc}")
        self.k, self.seed = k, seed

    def wads_rounds(self, k: int, seed: int, cap: int | None = None) -> dict:
        """The ADS by the paper's Algorithm 2 with CleanUp (supersteps in BFS
        order); per vertex its (id, distance) entries in (distance, rank)
        order, the supersteps run and the entries CleanUp removed."""
        cap = cap if cap is not None else max(64, 8 * self.n * k)
        eofs = np.zeros(self.n + 1, np.int64)
        eid = np.zeros(cap, np.int32)
        edist = np.zeros(cap, np.int64)
        steps, cleaned = i64(0), i64(0)
        rc = self._lib.orc_wads_rounds(self._h, k, seed, cap, _p(eofs), _p(eid), _p(edist),
                                       ctypes.byref(steps), ctypes.byref(cleaned))
        if rc != 0:
            raise RuntimeError(f"orc_wads_rounds rc={rc}")
        ne = int(eofs[-1])
        return dict(eofs=eofs, eid=eid[:ne].copy(), edist=edist[:ne].copy(), steps=int(steps.value),
                    cleaned=int(cleaned.value))

    def open_facilities_weighted(self, r: np.ndarray, client: np.ndarray, seed: int):
        r = np.ascontiguousarray(r, np.float64)
        client = np.ascontiguousarray(client, np.uint8)
        op = np.zeros(self.n, np.uint8)
        nopen = i64(0)
        rc = self._lib.orc_open_facilities_weighted(self._h, _p(r), _p(client), seed, _p(op),
                                                    ctypes.byref(nopen))
        if rc != 0:
            raise RuntimeError(f"orc_open_facilities_weighted rc={rc}")
        return op, int(nopen.value)

    def assign_weighted(self, open_: np.ndarray):
        op = np.ascontiguousarray(open_, np.uint8)
        a = np.zeros(self.n, np.int32)
        d = np.zeros(self.n, np.int32)
        rc = self._lib.orc_assign_weighted(self._h, _p(op), _p(a), _p(d))
        if rc != 0:
            raise RuntimeError(f"orc_assign_weighted rc={rc}")
        return a, d

    # -- phase (i): Section 3.3, Algorithms 1-2 ---------------------------
    def build_sketches(self, k: int, seed: int, max_hops: int | None = None) -> None:
        """Phase (i); with max_hops, stop after that many hops (a bounded sample)."""
        if max_hops is None:
            rc = self._lib.orc_build_sketches(self._h, k, seed)
        else:
            rc = self._lib.orc_build_sketches_hops(self._h, k, seed, max_hops)
        if rc != 0:
            raise RuntimeError(f"orc_build_sketches rc={rc}")
        self.k, self.seed = k, seed

    @property
    def hops(self) -> int:
        return int(self._lib.orc_hops(self._h))

    @property
    def edge_merges(self) -> int:
        return int(self._lib.orc_edge_merges(self._h))

    def sketch(self):
        S = np.zeros((self.n, self.k), np.uint64)
        cnt = np.zeros(self.n, np.int32)
        self._lib.orc_export_sketch(self._h, _p(S), _p(cnt))
        return S, cnt

    def ads(self, ranks: bool = True) -> dict:
        """The ADS, vertex-major (ranks=False leaves out the entries' ranks)."""
        ng = int(self._lib.orc_ads_groups(self._h))
        ne = int(self._lib.orc_ads_entries(self._h))
        out = dict(gofs=np.zeros(self.n + 1, np.int64), eofs=np.zeros(self.n + 1, np.int64),
                   ghop=np.zeros(ng, np.int32), gcnt=np.zeros(ng, np.int32),
                   gcounted=np.zeros(ng, np.int32), gwt=np.zeros(ng, np.float64),
                   eid=np.zeros(ne, np.int32))
        if ranks:
            out["erank"] = np.zeros(ne, np.uint64)
        self._lib.orc_export_ads(self._h, _p(out["gofs"]), _p(out["eofs"]), _p(out["ghop"]),
                                 _p(out["gcnt"]), _p(out["gcounted"]), _p(out["gwt"]),
                                 _p(out["eid"]), _p(out["erank"]) if ranks else None)
        return out

    def vertex_ads(self, k: int, seed: int, v: int, cap: int = 1 << 16) -> dict:
        """Algorithm 1 run for the single vertex v (sequential BFS order)."""
        ids = np.zeros(cap, np.int32)
        rk = np.zeros(cap, np.uint64)
        gh = np.zeros(cap, np.int32)
        gn = np.zeros(cap, np.int32)
        gc = np.zeros(cap, np.int32)
        gw = np.zeros(cap, np.float64)
        ng = i64(0)
        ne = self._lib.orc_vertex_ads(self._h, k, seed, v, cap, _p(ids), _p(rk), _p(gh),
                                      _p(gn), _p(gc), _p(gw), ctypes.byref(ng))
        if ne < 0:
            raise RuntimeError("orc_vertex_ads failed (capacity)")
        g = ng.value
        return dict(eid=ids[:ne].copy(), erank=rk[:ne].copy(), ghop=gh[:g].copy(),
                    gcnt=gn[:g].copy(), gcounted=gc[:g].copy(), gwt=gw[:g].copy())

    def nearest_open(self, open_: np.ndarray, v: int):
        """(facility, distance) of v's nearest open facility by BFS from v,
        ties to the smallest id; (-1, -1) when none is reachable."""
        op = np.ascontiguousarray(open_, np.uint8)
        a, d = ctypes.c_int32(), ctypes.c_int32()
        rc = self._lib.orc_nearest_open(self._h, _p(op), v, ctypes.byref(a), ctypes.byref(d))
        if rc != 0:
            raise RuntimeError(f"orc_nearest_open failed ({rc})")
        return a.value, d.value

    def hip_estimate(self, v: int, h: int, client=None) -> float:
        c = None if client is None else np.ascontiguousarray(client, np.uint8)
        return float(self._lib.orc_hip_estimate(self._h, v, h, None if c is None else _p(c)))

    # -- exact sizes and radii (Section 5.1, Fig. 1) ---------------------
    def ball_sizes(self, src, max_dist: int, pred=None) -> np.ndarray:
        """int64 [len(src), max_dist+1]: entry [s, h] = number of vertices w
        with d(src[s], w) <= h and pred[w] (pred None: all), by BFS."""
        src = np.ascontiguousarray(src, np.int32)
        p = None if pred is None else np.ascontiguousarray(pred, np.uint8)
        out = np.zeros((len(src), max_dist + 1), np.int64)
        rc = self._lib.orc_ball_sizes(self._h, len(src), _p(src), max_dist,
                                      None if p is None else _p(p), _p(out))
        if rc != 0:
            raise RuntimeError(f"orc_ball_sizes rc={rc}")
        return out

    def exact_radii(self, cost: np.ndarray, client: np.ndarray, facilities=None) -> np.ndarray:
        """Radii of Eq. 1 at epsilon -> 0 with exact client counts per
        distance (BFS); for all vertices, or for the ids in `facilities`."""
        cost = np.ascontiguousarray(cost, np.float64)
        client = np.ascontiguousarray(client, np.uint8)
        if facilities is None:
            r = np.zeros(self.n, np.float64)
            rc = self._lib.orc_exact_radii(self._h, _p(cost), _p(client), _p(r))
        else:
            fac = np.ascontiguousarray(facilities, np.int32)
            r = np.zeros(len(fac), np.float64)
            rc = self._lib.orc_exact_radii_of(self._h, len(fac), _p(fac), _p(cost), _p(client), _p(r))
        if rc != 0:
            raise RuntimeError(f"orc_exact_radii rc={rc}")
        return r

    # -- quality references (Section 5.2, Table 2) ----------------------
    def fl_cost(self, cost, client, open_) -> float:
        """sum of opening costs + sum of client distances to the open set;
        clients no facility reaches are left out; +inf if a reachable client
        is unserved."""
        c = np.ascontiguousarray(cost, np.float64)
        m = np.ascontiguousarray(client, np.uint8)
        o = np.ascontiguousarray(open_, np.uint8)
        return float(self._lib.orc_fl_cost(self._h, _p(c), _p(m), _p(o)))

    def optimum(self, cost, client):
        """(open mask, cost) of an optimal open set, by enumerating every set
        of at most 24 facilities."""
        c = np.ascontiguousarray(cost, np.float64)
        m = np.ascontiguousarray(client, np.uint8)
        op = np.zeros(self.n, np.uint8)
        obj = dbl(0)
        rc = self._lib.orc_fl_optimum(self._h, _p(c), _p(m), _p(op), ctypes.byref(obj))
        if rc != 0:
            raise RuntimeError(f"orc_fl_optimum rc={rc}")
        return op, float(obj.value)

    def local_search(self, cost, client, start=None, max_moves: int = 1 << 30):
        """(open mask, cost, moves) of add/drop/swap local search from
        `start` (None: the cheapest facility alone)."""
        c = np.ascontiguousarray(cost, np.float64)
        m = np.ascontiguousarray(client, np.uint8)
        op = np.zeros(self.n, np.uint8) if start is None else np.array(start, np.uint8)
        obj, mv = dbl(0), i64(0)
        rc = self._lib.orc_fl_local_search(self._h, _p(c), _p(m), max_moves, _p(op), ctypes.byref(obj),
                                           ctypes.byref(mv))
        if rc != 0:
            raise RuntimeError(f"orc_fl_local_search rc={rc}")
        return op, float(obj.value), int(mv.value)

    # -- phase (ii): Eq. 1 at epsilon -> 0 -------------------------------
    def radii(self, cost: np.ndarray, client: np.ndarray) -> np.ndarray:
        cost = np.ascontiguousarray(cost, np.float64)
        client = np.ascontiguousarray(client, np.uint8)
        r = np.zeros(self.n, np.float64)
        rc = self._lib.orc_compute_radii(self._h, _p(cost), _p(client), _p(r))
        if rc != 0:
            raise RuntimeError(f"orc_compute_radii rc={rc}")
        return r

    # -- phase (iii): lexicographically-first MIS (Section 4.3) -----------
    def open_facilities(self, r: np.ndarray, client: np.ndarray, seed: int):
        r = np.ascontiguousarray(r, np.float64)
        client = np.ascontiguousarray(client, np.uint8)
        op = np.zeros(self.n, np.uint8)
        nopen = i64(0)
        rc = self._lib.orc_open_facilities(self._h, _p(r), _p(client), seed, _p(op),
                                           ctypes.byref(nopen))
        if rc != 0:
            raise RuntimeError(f"orc_open_facilities rc={rc}")
        return op, int(nopen.value)

    def check_open_facilities(self, r: np.ndarray, client: np.ndarray, seed: int, open_: np.ndarray):
        """(ok, witness): whether open_ is the lexicographically-first MIS of
        H-bar under (r_f, pi_f), checked by its characterisation in parallel
        (independent; every other candidate conflicts with an earlier member)."""
        r = np.ascontiguousarray(r, np.float64)
        client = np.ascontiguousarray(client, np.uint8)
        op = np.ascontiguousarray(open_, np.uint8)
        bad = i64(-1)
        rc = self._lib.orc_check_open_facilities(self._h, _p(r), _p(client), seed, _p(op), ctypes.byref(bad))
        if rc < 0:
            raise RuntimeError(f"orc_check_open_facilities rc={rc}")
        return rc == 1, int(bad.value)

    # -- the opening phase with epsilon > 0 (Algorithms 3-6, Eq. 2/3) ------
    def eps_gamma(self, cost, client) -> float:
        """gamma = max over clients reaching a facility of min_f (c(f) + d(c,f))."""
        c = np.ascontiguousarray(cost, np.float64)
        m = np.ascontiguousarray(client, np.uint8)
        return float(self._lib.orc_eps_gamma(self._h, _p(c), _p(m)))

    def eps_open(self, eps: float, cost, client, mode: int = 0) -> dict:
        """Facility opening and client freezing (Algorithms 3-5): per vertex
        the iteration at which it opened (fac_iter) or froze (cli_iter), -1
        for never; q(f) at opening (or at the end); alpha_0, gamma and the
        iterations run.  mode 1 accumulates q by Eq. 2/3 literally."""
        c = np.ascontiguousarray(cost, np.float64)
        m = np.ascontiguousarray(client, np.uint8)
        fi = np.zeros(self.n, np.int32)
        ci = np.zeros(self.n, np.int32)
        q = np.zeros(self.n, np.float64)
        a0, gm, it = dbl(0), dbl(0), i64(0)
        rc = self._lib.orc_eps_open(self._h, float(eps), _p(c), _p(m), int(mode), _p(fi), _p(ci), _p(q),
                                    ctypes.byref(a0), ctypes.byref(gm), ctypes.byref(it))
        if rc != 0:
            raise RuntimeError(f"orc_eps_open rc={rc}")
        return dict(fac_iter=fi, cli_iter=ci, q=q, alpha0=a0.value, gamma=gm.value, iterations=it.value)

    def eps_select(self, eps: float, alpha0: float, fac_iter, cli_iter, seed: int):
        """Algorithm 6: lexicographically-first MIS under pi of H-bar."""
        fi = np.ascontiguousarray(fac_iter, np.int32)
        ci = np.ascontiguousarray(cli_iter, np.int32)
        op = np.zeros(self.n, np.uint8)
        no = i64(0)
        rc = self._lib.orc_eps_select(self._h, float(eps), float(alpha0), _p(fi), _p(ci), seed, _p(op),
                                      ctypes.byref(no))
        if rc != 0:
            raise RuntimeError(f"orc_eps_select rc={rc}")
        return op, int(no.value)

    # -- assignment + objective (Section 3.1) ----------------------------
    def assign(self, open_: np.ndarray):
        op = np.ascontiguousarray(open_, np.uint8)
        a = np.zeros(self.n, np.int32)
        d = np.zeros(self.n, np.int32)
        rc = self._lib.orc_assign(self._h, _p(op), _p(a), _p(d))
        if rc != 0:
            raise RuntimeError(f"orc_assign rc={rc}")
        return a, d


def radius_of_ads(ads: dict, client: np.ndarray, cost: float) -> float:
    """Radius (Eq. 1 at epsilon -> 0) of one vertex from its ADS groups
    (the dict of Graph.vertex_ads: ghop, gcnt, gcounted, gwt, eid)."""
    lib = _load()
    gh = np.ascontiguousarray(ads["ghop"], np.int32)
    gn = np.ascontiguousarray(ads["gcnt"], np.int32)
    gc = np.ascontiguousarray(ads["gcounted"], np.int32)
    gw = np.ascontiguousarray(ads["gwt"], np.float64)
    ids = np.ascontiguousarray(ads["eid"], np.int32)
    cl = np.ascontiguousarray(client, np.uint8)
    return lib.orc_radius_of_ads(len(gh), _p(gh), _p(gn), _p(gc), _p(gw), _p(ids), _p(cl), float(cost))


def objective(open_, cost, client, dist):
    lib = _load()
    op = np.ascontiguousarray(open_, np.uint8)
    cost = np.ascontiguousarray(cost, np.float64)
    client = np.ascontiguousarray(client, np.uint8)
    dist = np.ascontiguousarray(dist, np.int32)
    obj, ds, un = dbl(0), i64(0), i64(0)
    lib.orc_objective(len(op), _p(op), _p(cost), _p(client), _p(dist),
                      ctypes.byref(obj), ctypes.byref(ds), ctypes.byref(un))
    return float(obj.value), int(ds.value), int(un.value)


def solve(rowp, cols, k, seed, cost, client) -> dict:
    """The whole path on the CPU: sketches, radii, MIS, assignment, objective."""
    g = Graph(rowp, cols)
    g.build_sketches(k, seed)
    r = g.radii(cost, client)
    op, nopen = g.open_facilities(r, client, seed)
    a, d = g.assign(op)
    obj, ds, un = objective(op, cost, client, d)
    S, cnt = g.sketch()
    out = dict(graph=g, hops=g.hops, edge_merges=g.edge_merges, S=S, Scnt=cnt,
               ads=g.ads(), radii=r, open=op, n_open=nopen, assign=a, dist=d,
               objective=obj, dist_sum=ds, n_unserved=un)
    return out


def solve_eps(rowp, cols, k, seed, eps, cost, client) -> dict:
    """The epsilon > 0 path on the CPU: sketches, opening phase, Algorithm 6
    selection, assignment, objective."""
    g = Graph(rowp, cols)
    g.build_sketches(k, seed)
    o = g.eps_open(eps, cost, client)
    op, nopen = g.eps_select(eps, o["alpha0"], o["fac_iter"], o["cli_iter"], seed)
    a, d = g.assign(op)
    obj, ds, un = objective(op, cost, client, d)
    return dict(graph=g, opening=o, open=op, n_open=nopen, assign=a, dist=d, objective=obj, dist_sum=ds,
                n_unserved=un)


def solve_weighted(rowp, cols, w, k, seed, cost, client) -> dict:
    """The whole path on a weighted graph (NEXT f3): ADS in Dijkstra order,
    radii (Eq. 1 at epsilon -> 0 over integer distances), the
    lexicographically-first MIS with weighted balls, nearest open facility by
    weighted distance, objective."""
    g = Graph(rowp, cols)
    g.set_weights(w)
    g.build_sketches_weighted(k, seed)
    r = g.radii(cost, client)
    op, nopen = g.open_facilities_weighted(r, client, seed)
    a, d = g.assign_weighted(op)
    obj, ds, un = objective(op, cost, client, d)
    return dict(graph=g, radii=r, open=op, n_open=nopen, assign=a, dist=d, objective=obj, dist_sum=ds,
                n_unserved=un, hops=g.hops)
