"""Seeded synthetic inputs for the facility-location path (graphs, masks, costs).

Shared by the CPU oracle's tests, the CUDA path's tests and the benchmark.  It
holds none of the method's arithmetic: it only draws graphs and per-vertex
inputs from a counter-based hash (see ``synth.c``), so the same call gives the
same arrays on every machine and thread count.

Workload recipes (the paper's social/web graphs and its synthetic R-MAT family,
Section 5 and Table 1, stood in for by seeded R-MAT and Erdos-Renyi graphs):

* ``er10k``  -- G(n=10^4, M=4*10^4), every vertex client and facility, cost 20.0,
  sketch k=16.
* ``rmat20`` -- R-MAT scale 20, 16*2^20 draws, (a,b,c,d)=(.57,.19,.19,.05),
  seeded relabelling, symmetrised and deduplicated; all vertices clients and
  facilities; costs log-uniform in [5, 500]; k=32.
* ``rmat26`` -- the same recipe at scale 26; clients Bernoulli(0.5), facilities
  Bernoulli(0.1) independently, facility costs log-uniform in [10, 10^4], other
  vertices +inf; k=16.
* ``batch`` (``batch_config``): 64 instances on the rmat20 graph with their own
  client sets and costs, plus 256 Erdos-Renyi graphs of uneven size; k=32.
* ``rmatS`` for other scales (tests): the rmat20 recipe at scale S;
  ``rmat26sS``: the rmat26 recipe at scale S (profiling at a smaller footprint).

Seeds: graph seed 42 + config number (er10k=1, rmat20=2, rmat26=3, rmat23=5),
sketch seed 1, mask/cost seed 7, query seed 11.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB_PATH = os.path.join(_HERE, "libflsynth.so")
_lock = threading.Lock()
_lib = None

SKETCH_SEED = 1
MASK_SEED = 7
QUERY_SEED = 11


def build(force: bool = False) -> str:
    """Compile ``synth.c`` into ``libflsynth.so`` (gcc, OpenMP)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            i64, u64, u32, vp = ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p
            lib.syn_er.restype = i64
            lib.syn_er.argtypes = [i64, i64, u64, vp, vp]
            lib.syn_rmat.restype = i64
            lib.syn_rmat.argtypes = [ctypes.c_int, i64, u32, u32, u32, u64, vp, vp]
            lib.syn_bernoulli.restype = None
            lib.syn_bernoulli.argtypes = [i64, u64, u32, vp]
            lib.syn_loguniform.restype = None
            lib.syn_loguniform.argtypes = [i64, u64, ctypes.c_double, ctypes.c_double, vp, vp]
            lib.syn_uniform.restype = None
            lib.syn_uniform.argtypes = [i64, u64, ctypes.c_double, ctypes.c_double, vp]
            lib.syn_hash.restype = None
            lib.syn_hash.argtypes = [i64, u64, vp]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def er(n: int, M: int, seed: int):
    """Erdos-Renyi G(n, M) as symmetric CSR (rowp int64[n+1], cols int32[2M])."""
    lib = _load()
    rowp = np.zeros(n + 1, np.int64)
    cols = np.zeros(max(2 * M, 1), np.int32)
    nnz = lib.syn_er(n, M, seed, _ptr(rowp), _ptr(cols))
    if nnz < 0:
        raise ValueError(f"syn_er failed for n={n} M={M}")
    return rowp, cols[:nnz].copy()


def rmat(scale: int, edgefactor: int, seed: int, a=0.57, b=0.19, c=0.19):
    """R-MAT graph with 2^scale vertices and edgefactor*2^scale draws, as CSR."""
    lib = _load()
    n = 1 << scale
    ndraws = edgefactor * n
    ta = int(a * 65536)
    tb = int((a + b) * 65536)
    tc = int((a + b + c) * 65536)
    rowp = np.zeros(n + 1, np.int64)
    cols = np.empty(max(2 * ndraws, 1), np.int32)
    nnz = lib.syn_rmat(scale, ndraws, ta, tb, tc, seed, _ptr(rowp), _ptr(cols))
    if nnz < 0:
        raise ValueError(f"syn_rmat failed for scale={scale}")
    out = cols[:nnz]
    if nnz < len(cols) // 2:
        out = out.copy()
    return rowp, out


def bernoulli(n: int, seed: int, p: float) -> np.ndarray:
    lib = _load()
    m = np.zeros(n, np.uint8)
    lib.syn_bernoulli(n, seed, min(int(p * 4294967296.0), 0xFFFFFFFF), _ptr(m))
    return m


def loguniform(n: int, seed: int, lo: float, hi: float, facility_mask=None) -> np.ndarray:
    lib = _load()
    out = np.zeros(n, np.float64)
    fm = None if facility_mask is None else np.ascontiguousarray(facility_mask, np.uint8)
    lib.syn_loguniform(n, seed, lo, hi, None if fm is None else _ptr(fm), _ptr(out))
    return out


def uniform(m: int, seed: int, lo: float, hi: float) -> np.ndarray:
    lib = _load()
    out = np.zeros(m, np.float64)
    lib.syn_uniform(m, seed, lo, hi, _ptr(out))
    return out


def hashes(m: int, seed: int) -> np.ndarray:
    lib = _load()
    out = np.zeros(m, np.uint64)
    lib.syn_hash(m, seed, _ptr(out))
    return out


def edge_weights(rowp: np.ndarray, cols: np.ndarray, seed: int, lo: int = 1, hi: int = 100) -> np.ndarray:
    """Integer edge lengths uniform in [lo, hi] (Section 5 draws weights
    between 1 and 100), one per CSR entry and equal for (u, v) and (v, u):
    a hash (the 64-bit finaliser of MurmurHash3) of the unordered pair and
    the seed, reduced modulo the range."""
    rowp = np.asarray(rowp, np.int64)
    n = len(rowp) - 1
    src = np.repeat(np.arange(n, dtype=np.uint64), np.diff(rowp).astype(np.int64))
    dst = np.asarray(cols).astype(np.uint64)
    a, b = np.minimum(src, dst), np.maximum(src, dst)
    x = (a << np.uint64(32)) ^ b ^ np.uint64((seed * 0x9E3779B97F4A7C15) % (1 << 64))
    x ^= x >> np.uint64(33)
    x *= np.uint64(0xFF51AFD7ED558CCD)
    x ^= x >> np.uint64(33)
    x *= np.uint64(0xC4CEB9FE1A85EC53)
    x ^= x >> np.uint64(33)
    return (np.int64(lo) + (x % np.uint64(hi - lo + 1)).astype(np.int64)).astype(np.int32)


@dataclasses.dataclass
class Workload:
    """One facility-location instance: CSR graph + per-vertex inputs."""
    name: str
    n: int
    rowp: np.ndarray          # int64[n+1]
    cols: np.ndarray          # int32[nnz]
    k: int                    # bottom-k sketch size
    seed: int                 # rank seed
    cost: np.ndarray          # float64[n], +inf = not a facility
    client: np.ndarray        # uint8[n], 1 = client

    @property
    def nnz(self) -> int:
        return int(self.rowp[-1])


def from_csr(name, rowp, cols, k, seed, cost, client) -> Workload:
    n = len(rowp) - 1
    return Workload(name, n, np.ascontiguousarray(rowp, np.int64),
                    np.ascontiguousarray(cols, np.int32), k, seed,
                    np.ascontiguousarray(cost, np.float64),
                    np.ascontiguousarray(client, np.uint8))


def config(name: str) -> Workload:
    """Build one of the named workloads (see module docstring)."""
    if name == "er10k":
        n = 10_000
        rowp, cols = er(n, 40_000, 42 + 1)
        return from_csr(name, rowp, cols, 16, SKETCH_SEED,
                        np.full(n, 20.0), np.ones(n, np.uint8))
    if name.startswith("rmat"):
        # "rmat26sS": the rmat26 recipe (masks, costs, k) at scale S
        c3 = name.startswith("rmat26s")
        scale = int(name[7:]) if c3 else int(name[4:])
        rowp, cols = rmat(scale, 16, 42 + {20: 2, 26: 3, 23: 5}.get(scale, scale))
        n = 1 << scale
        if scale == 26 or c3:
            client = bernoulli(n, MASK_SEED, 0.5)
            fac = bernoulli(n, MASK_SEED + 1, 0.1)
            cost = loguniform(n, MASK_SEED + 2, 10.0, 1.0e4, fac)
            return from_csr(name, rowp, cols, 16, SKETCH_SEED, cost, client)
        k = 32
        cost = loguniform(n, MASK_SEED, 5.0, 500.0)
        return from_csr(name, rowp, cols, k, SKETCH_SEED, cost, np.ones(n, np.uint8))
    raise KeyError(name)


@dataclasses.dataclass
class BatchWorkload:
    """The batched workload: instances on one resident graph plus many small
    independent graphs (each a Workload with its own costs and clients)."""
    name: str
    resident: Workload        # the shared graph (its own cost/client unused)
    inst_cost: list           # float64[n] per instance on the resident graph
    inst_client: list         # uint8[n] per instance on the resident graph
    graphs: list              # Workload per independent graph


def _sample_without_replacement(n: int, m: int, seed: int) -> np.ndarray:
    """m distinct vertices of [0, n): the m smallest keys of a seeded hash."""
    key = hashes(n, seed)
    return np.sort(np.argpartition(key, m - 1)[:m]) if m < n else np.arange(n)


def batch_config(n_resident: int = 64, n_graphs: int = 256) -> BatchWorkload:
    """`batch`: n_resident instances on the rmat20 graph (k=32), each with a
    client set of log-uniform size in [10^3, 10^6] sampled without
    replacement, every vertex a facility, one opening cost per instance
    uniform in [5, 500]; plus n_graphs Erdos-Renyi graphs with n log-uniform
    in [10^3, 10^5] and average degree uniform in {4..16}, every vertex a
    client and facility, one cost per graph uniform in [5, 500]; k=32.
    Seeds: graphs 42 + 4, instance parameters 11 (the query seed) + offsets."""
    base = config("rmat20")
    n = base.n
    sizes = loguniform(n_resident, QUERY_SEED, 1.0e3, 1.0e6)
    inst_costs = uniform(n_resident, QUERY_SEED + 1, 5.0, 500.0)
    inst_cost, inst_client = [], []
    for i in range(n_resident):
        m = min(n, int(math.floor(sizes[i])))
        cl = np.zeros(n, np.uint8)
        cl[_sample_without_replacement(n, m, QUERY_SEED + 100 + i)] = 1
        inst_client.append(cl)
        inst_cost.append(np.full(n, inst_costs[i]))
    er_n = loguniform(n_graphs, 42 + 4, 1.0e3, 1.0e5)
    er_deg = uniform(n_graphs, 42 + 5, 4.0, 17.0)
    er_cost = uniform(n_graphs, 42 + 6, 5.0, 500.0)
    graphs = []
    for j in range(n_graphs):
        nj = int(math.floor(er_n[j]))
        dj = min(16, int(math.floor(er_deg[j])))
        rowp, cols = er(nj, nj * dj // 2, 42 + 4 + 1000 * (j + 1))
        graphs.append(from_csr(f"er{nj}", rowp, cols, 32, SKETCH_SEED, np.full(nj, er_cost[j]),
                               np.ones(nj, np.uint8)))
    return BatchWorkload("batch", base, inst_cost, inst_client, graphs)


def small_er(n: int, avg_deg: float, seed: int, k: int = 16, cost: float = 20.0,
             client_p: float = 1.0, fac_p: float = 1.0) -> Workload:
    """Small ER instance for tests (optionally with random client/facility subsets)."""
    M = int(round(n * avg_deg / 2))
    M = min(M, n * (n - 1) // 2)
    rowp, cols = er(n, M, seed)
    client = np.ones(n, np.uint8) if client_p >= 1.0 else bernoulli(n, seed + 1000, client_p)
    fac = np.ones(n, np.uint8) if fac_p >= 1.0 else bernoulli(n, seed + 2000, fac_p)
    c = np.where(fac > 0, cost, np.inf)
    return from_csr(f"er{n}", rowp, cols, k, SKETCH_SEED, c, client)
