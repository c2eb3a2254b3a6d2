"""Host-side logic of the serving loop (no GPU): the Poisson request trace,
the device-arena allocator that admits requests by memory, and the buffer
layout of one request."""
import numpy as np
import pytest

from paper_2603_20525_gb300 import serve


def test_trace_rates_and_ranges():
    tr = serve.poisson_trace(n_vehicles=32, rate_hz=20.0, duration_s=30.0, seed=3)
    assert all(tr[i].t_arrive <= tr[i + 1].t_arrive for i in range(len(tr) - 1))
    per = np.bincount([r.vehicle for r in tr], minlength=32)
    assert abs(per.mean() - 600) < 3 * np.sqrt(600 / 32)      # 20 Hz x 30 s per vehicle
    assert {r.N for r in tr} == {1024, 4096, 16384, 32768}
    assert min(r.H for r in tr) >= 40 and max(r.H for r in tr) <= 150
    dts = {round(r.dt, 6) for r in tr}
    assert dts <= {round(0.005 * k, 6) for k in range(4, 11)} and len(dts) == 7
    gaps = np.diff([r.t_arrive for r in tr if r.vehicle == 0])
    assert abs(gaps.mean() - 0.05) < 0.01                    # exponential, mean 50 ms


class FakeArena(serve.DeviceArena):
    """The allocator's bookkeeping without device memory."""

    def __init__(self, nbytes):
        self.nbytes = serve._align(nbytes)
        self.free = [(0, self.nbytes)]
        self.used = 0


def test_arena_best_fit_coalesces_and_refuses():
    a = FakeArena(10 * 256)
    x = a.alloc(256 * 3)
    y = a.alloc(256 * 2)
    z = a.alloc(256 * 4)
    assert a.alloc(256 * 2) is None                          # 1 block left
    a.release(y, 256 * 2)
    assert a.alloc(100) == 9 * 256                           # best fit: the 1-block hole
    w = a.alloc(300)                                         # only the 2-block hole fits
    assert w == y
    a.release(9 * 256, 100)
    a.release(x, 256 * 3)
    a.release(w, 300)
    a.release(z, 256 * 4)
    assert a.free == [(0, 10 * 256)] and a.used == 0         # fully coalesced


def test_arena_random_workload_never_overlaps():
    rng = np.random.default_rng(1)
    a = FakeArena(1 << 20)
    live = {}
    for _ in range(3000):
        if live and rng.random() < 0.45:
            off = list(live)[rng.integers(len(live))]
            a.release(off, live.pop(off))
        else:
            n = int(rng.integers(1, 40000))
            off = a.alloc(n)
            if off is not None:
                live[off] = n
        spans = sorted((o, o + serve._align(n)) for o, n in live.items())
        assert all(spans[i][1] <= spans[i + 1][0] for i in range(len(spans) - 1))
        assert a.used == sum(serve._align(n) for n in live.values())
        assert sum(s for _, s in a.free) + a.used == a.nbytes


def test_request_layout_is_aligned_and_disjoint():
    lay, total = serve.request_layout(16384, 100)
    offs = [o for _, o, _, _ in lay]
    assert all(o % 256 == 0 for o in offs) and offs == sorted(offs)
    assert total >= 16384 * 100 * 8              # the candidates' controls


def test_admission_keeps_each_vehicles_order():
    """A request that does not fit (slots, batch size or memory) holds back
    every later request of its vehicle, so a vehicle's plans, and its warm
    starts, always run in arrival order; other vehicles fill the batch."""
    from paper_2603_20525_gb300 import serve

    class V:
        busy = False

    vehicles = [V(), V(), V()]
    q = [serve.Request(0, 0, 4096, 50, 0.02, 0.0),       # fits
         serve.Request(1, 1, 65536, 50, 0.02, 0.0),      # too many candidates now
         serve.Request(2, 1, 1024, 50, 0.02, 0.0),       # same vehicle: must wait behind rid 1
         serve.Request(3, 2, 1024, 50, 0.02, 0.0),       # other vehicle: fits
         serve.Request(4, 0, 1024, 50, 0.02, 0.0)]       # vehicle 0 is now busy
    batch, offs, keep = serve.admit(q, vehicles, 64, 65536, lambda r: 0)
    assert [r.rid for r in batch] == [0, 3] and [r.rid for r in keep] == [1, 2, 4]
    assert vehicles[0].busy and vehicles[2].busy and not vehicles[1].busy
    # memory refusal holds back the vehicle too
    for v in vehicles:
        v.busy = False
    mem = iter([None, 0, 0])
    batch, offs, keep = serve.admit(q[1:4], vehicles, 64, 1 << 20, lambda r: next(mem))
    assert [r.rid for r in batch] == [3] and [r.rid for r in keep] == [1, 2]
    # the batch limit holds back later requests of a vehicle as well
    for v in vehicles:
        v.busy = False
    batch, offs, keep = serve.admit([q[0], q[3], q[4]], vehicles, 1, 1 << 20, lambda r: 0)
    assert [r.rid for r in batch] == [0] and [r.rid for r in keep] == [3, 4]


def test_admission_replays_arrival_order_under_backlog():
    """Against a random backlog with tight slots and memory, every vehicle's
    admitted requests come out in arrival order."""
    import numpy as np
    from paper_2603_20525_gb300 import serve

    class V:
        busy = False

    rng = np.random.default_rng(0)
    vehicles = [V() for _ in range(8)]
    queue = [serve.Request(i, int(rng.integers(0, 8)), int(rng.choice([1024, 4096, 16384, 32768])), 50, 0.02, 0.0)
             for i in range(400)]
    order = {v: [] for v in range(8)}
    free = [5]
    while queue:
        def alloc(r):
            if free[0] > 0 and rng.random() < 0.8:
                free[0] -= 1
                return 0
            return None
        batch, offs, queue = serve.admit(queue, vehicles, 6, 40000, alloc)
        for r in batch:
            order[r.vehicle].append(r.rid)
            vehicles[r.vehicle].busy = False          # completes before the next pass
        free[0] = 5
    for v, rids in order.items():
        assert rids == sorted(rids)
    assert sum(len(r) for r in order.values()) == 400


def test_collector_paused_restores_state():
    import gc
    assert gc.isenabled()
    with serve.collector_paused():
        assert not gc.isenabled()
    assert gc.isenabled()
    with pytest.raises(RuntimeError):
        with serve.collector_paused():
            raise RuntimeError("loop failed")
    assert gc.isenabled()
    gc.disable()
    try:
        with serve.collector_paused():
            assert not gc.isenabled()
        assert not gc.isenabled()          # a caller's own pause is kept
    finally:
        gc.enable()


def test_trace_check_refuses_horizons_beyond_the_warm_start():
    """A plan writes its best controls into its vehicle's warm-start buffer,
    so a horizon longer than that buffer, or an unknown vehicle, is refused
    before anything runs."""
    from types import SimpleNamespace
    from paper_2603_20525_gb300 import serve
    vehicles = [SimpleNamespace(prev=np.zeros((150, 2), np.float32)) for _ in range(2)]
    ok = [serve.Request(0, 0, 1024, 150, 0.02, 0.0), serve.Request(1, 1, 1024, 1, 0.02, 0.0)]
    serve.check_trace(ok, vehicles)
    for bad in (serve.Request(2, 0, 1024, 151, 0.02, 0.0), serve.Request(3, 1, 1024, 0, 0.02, 0.0),
                serve.Request(4, 2, 1024, 40, 0.02, 0.0)):
        with pytest.raises(ValueError):
            serve.check_trace(ok + [bad], vehicles)
