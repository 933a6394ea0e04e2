"""Host logic of the serving loop on the CPU (no GPU): queue refusal,
admission by free device memory, and the worker's batching — queries taken
in groups of at most `slots`, each written into its own slice of the batch
and each result mapped back to its own query — with a fake device API and a
fake replica batch whose per-instance result depends only on that
instance's inputs, so a result that went to the wrong query shows."""
import collections
import threading
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1503_03635_gb300 import serve  # noqa: E402


class _FakeCuda:
    def __init__(self, free):
        self.free = free
        self.calls = 0

    def mem_get_info(self, device=None):
        self.calls += 1
        return self.free, 1 << 40

    def set_device(self, device):
        pass

    class _Ctx:
        def __enter__(self):
            return self

        def __exit__(self, *a):
            return False

    def stream(self, s):
        return self._Ctx()


def _fake_torch(free):
    """The calls the worker makes, on CPU tensors, with a fake cuda namespace."""
    t = types.SimpleNamespace()
    t.cuda = _FakeCuda(free)
    t.bool = torch.bool
    t.as_tensor = torch.as_tensor
    t.lt = torch.lt

    def generator(device=None):
        return torch.Generator()

    def rand(n, generator=None, device=None):
        return torch.rand(n, generator=generator)

    t.Generator = generator
    t.rand = rand
    return t


class _FakeStream:
    def synchronize(self):
        pass


class _FakeBatch:
    """Instance i's result depends only on its own cost and clients."""

    def __init__(self, n):
        self.n = n
        self.sizes = []

    def solve(self, k, seed, cost, client, open_out=None, n_active=None):
        n, r = self.n, n_active
        self.sizes.append(r)
        res = {key: np.zeros(r) for key in ("n_open", "objective", "dist_sum", "n_unserved")}
        for i in range(r):
            c = client[i * n:(i + 1) * n].numpy().astype(np.int64)
            f = float(cost[i * n].item())
            res["n_open"][i] = int(c.sum())
            res["objective"][i] = f * int(c.sum()) + k
            res["dist_sum"][i] = int((c * np.arange(n)).sum())
            res["n_unserved"][i] = int(n - c.sum())
            if open_out is not None:
                open_out[i * n:(i + 1) * n].copy_(client[i * n:(i + 1) * n])
        return res


def _server(n, slots, free, query_bytes, max_pending=100):
    s = object.__new__(serve.Server)
    s.torch = _fake_torch(free)
    s.k, s.seed, s.n = 7, 1, n
    s.keep_open_mask = True
    s.device = "cpu"
    s.slots = slots
    s.query_bytes = query_bytes
    s.waited_for_memory = 0
    s.max_pending = max_pending
    s.rejected = 0
    s._q = collections.deque()
    s._cv = threading.Condition()
    s._stop = False
    s._workers = []
    return s


def _bufs(n, slots):
    m = n * slots
    return dict(cost=torch.empty(m, dtype=torch.float64), client=torch.empty(m, dtype=torch.uint8),
                open=torch.empty(m, dtype=torch.uint8), open_h=torch.empty(m, dtype=torch.uint8))


def _expected(q, n, k):
    if q.client_mask is not None:
        c = np.asarray(q.client_mask, np.int64)
    else:
        gen = torch.Generator()
        gen.manual_seed(q.client_seed)
        c = (torch.rand(n, generator=gen) < q.client_frac).numpy().astype(np.int64)
    return dict(n_open=int(c.sum()), objective=q.cost * int(c.sum()) + k, dist_sum=int((c * np.arange(n)).sum()),
                n_unserved=int(n - c.sum()), open=c.astype(np.uint8))


def test_submit_refuses_when_the_queue_is_full():
    s = _server(10, 2, free=1 << 40, query_bytes=1, max_pending=2)
    qs = [s.submit(serve.Query(1.0)) for _ in range(3)]
    assert len(s._q) == 2 and s.rejected == 1
    assert qs[2].error is not None and qs[2]._done.is_set()
    with pytest.raises(RuntimeError):
        qs[2].wait(0)


@pytest.mark.parametrize("free_gb,want,expect", [(10, 4, 4), (5, 4, 3), (3, 2, 1), (2.5, 4, 0), (1, 4, 0)])
def test_admission_by_free_memory(free_gb, want, expect):
    """A query needs query_bytes beyond the reserve kept for the process."""
    s = _server(10, 4, free=int(free_gb * (1 << 30)), query_bytes=1 << 30)
    assert s._admissible(want) == expect


def test_worker_batches_queries_and_maps_results_back():
    n, slots = 64, 3
    s = _server(n, slots, free=1 << 40, query_bytes=1)
    batch = _FakeBatch(n)
    rng = np.random.default_rng(3)
    queries = []
    for i in range(11):
        if i % 3 == 0:
            q = serve.Query(cost=1.5 + i, client_mask=(rng.random(n) < 0.4).astype(np.uint8))
        else:
            q = serve.Query(cost=2.0 + i, client_seed=100 + i, client_frac=0.3)
        queries.append(s.submit(q))  # queued before the worker starts: it takes them in groups
    th = threading.Thread(target=s._run, args=(_FakeStream(), batch, _bufs(n, slots)), daemon=True)
    th.start()
    for q in queries:
        res = q.wait(10)
        want = _expected(q, n, s.k)
        assert res["n_open"] == want["n_open"] and res["dist_sum"] == want["dist_sum"]
        assert res["n_unserved"] == want["n_unserved"] and res["objective"] == pytest.approx(want["objective"])
        assert np.array_equal(res["open"], want["open"])
        assert 1 <= q.batch_size <= slots and q.latency is not None and q.latency >= 0
    with s._cv:
        s._stop = True
        s._cv.notify_all()
    th.join(10)
    assert not th.is_alive()
    assert sum(batch.sizes) == len(queries) and max(batch.sizes) == slots


def test_worker_waits_for_memory_then_serves():
    """With no memory for a query the worker waits (counted) and serves it
    once memory frees up."""
    n, slots = 16, 2
    s = _server(n, slots, free=0, query_bytes=1)
    batch = _FakeBatch(n)
    th = threading.Thread(target=s._run, args=(_FakeStream(), batch, _bufs(n, slots)), daemon=True)
    th.start()
    q = s.submit(serve.Query(cost=3.0, client_mask=np.ones(n, np.uint8)))
    for _ in range(400):
        if s.waited_for_memory > 0:
            break
        threading.Event().wait(0.005)
    assert s.waited_for_memory > 0 and not q._done.is_set()
    s.torch.cuda.free = 1 << 40
    assert q.wait(10)["n_open"] == n
    with s._cv:
        s._stop = True
        s._cv.notify_all()
    th.join(10)
    assert not th.is_alive()


def test_worker_errors_reach_their_queries():
    n = 8

    class _Failing(_FakeBatch):
        def solve(self, *a, **k):
            raise RuntimeError("solve failed")

    s = _server(n, 2, free=1 << 40, query_bytes=1)
    th = threading.Thread(target=s._run, args=(_FakeStream(), _Failing(n), _bufs(n, 2)), daemon=True)
    th.start()
    q = s.submit(serve.Query(cost=1.0, client_mask=np.ones(n, np.uint8)))
    with pytest.raises(RuntimeError, match="solve failed"):
        q.wait(10)
    with s._cv:
        s._stop = True
        s._cv.notify_all()
    th.join(10)


def test_latency_summary():
    qs = []
    for lat in (0.010, 0.020, 0.030, 0.040):
        q = serve.Query(1.0)
        q.t_arrival, q.t_done = 100.0, 100.0 + lat
        qs.append(q)
    bad = serve.Query(1.0)
    bad.t_arrival, bad.t_done, bad.error = 0.0, 5.0, RuntimeError("x")
    out = serve.latency_summary(qs + [bad])
    assert out["max_ms"] == pytest.approx(40.0) and out["mean_ms"] == pytest.approx(25.0)
    assert 10.0 <= out["p50_ms"] <= 40.0 and out["p99_ms"] <= 40.0
    assert serve.latency_summary([]) == {}
