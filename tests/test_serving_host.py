"""Host-side logic of the serving form, on the CPU: what the server refuses
and how it reports a run."""
import pytest

import synth
from paper_1004_1302_gb300 import serve
from paper_1004_1302_gb300 import splotch as S


class _Resident:
    n, dtype = 0, "f16"


@pytest.mark.parametrize("kw", [dict(use_vector=1), dict(modulate=1)])
def test_server_refuses_what_the_region_cut_does_not_carry(kw):
    sp = synth.Species(0, 0, **kw)
    with pytest.raises(ValueError):
        serve.RenderServer(_Resident(), None, sp)


def test_stats_percentiles_and_refusals():
    done = []
    for k, lat in enumerate([0.010, 0.020, 0.030, 0.040]):
        r = serve.Request(k, (0, 0, 0, 1, 1, 1), None, 0, arrival=0.0, n=100)
        r.status, r.done = S.OK, lat
        done.append(r)
    refused = serve.Request(9, (0, 0, 0, 1, 1, 1), None, 0)
    refused.status, refused.done = S.ERR_OOM_ADMISSION, 0.0
    st = serve.RenderServer.stats(done + [refused], wall=2.0)
    assert st["completed"] == 4 and st["refused"] == 1 and st["requests"] == 5
    assert st["p50_ms"] == pytest.approx(20.0) and st["p99_ms"] == pytest.approx(40.0)
    assert st["frames_per_s"] == pytest.approx(2.0) and st["particles_per_s"] == pytest.approx(200.0)


def test_poisson_arrivals_are_increasing_and_seeded():
    a = synth.poisson_times(50, rate=10.0, seed=3)
    b = synth.poisson_times(50, rate=10.0, seed=3)
    assert a == b and all(x < y for x, y in zip(a, a[1:]))
    assert 2.0 < a[-1] < 10.0     # 50 arrivals at 10/s


def test_request_stream_is_seeded_and_inside_the_unit_cube():
    a = synth.request_stream(40, 10**9, seed=5)
    b = synth.request_stream(40, 10**9, seed=5)
    assert [(r[0], r[2]) for r in a] == [(r[0], r[2]) for r in b]
    for box, cam, mode in a:
        assert all(0.0 <= v <= 1.0 for v in box) and mode in (0, 1)
        assert all(lo < hi for lo, hi in zip(box[:3], box[3:]))
        assert 30.0 <= cam.fov_x_deg <= 60.0


# --- watchdog and cancellation, with the device replaced by fakes -------------

class _Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 0.001          # every reading advances the clock by 1 ms
        return self.t


class _Event:
    def __init__(self, clock, end):
        self.clock, self.end = clock, end

    def query(self):
        return self.clock.t >= self.end


class _Info:
    status, tile_entries = S.OK, 0


class _FakeFrame:
    def info(self, stream=None):
        return _Info()


class _FakeServer(serve.RenderServer):
    """The request loop over a device that takes `work[rid]` seconds per
    request (inf: never ends)."""

    def __init__(self, clock, work, max_inflight=2, timeout=None):
        self.request_timeout_s = timeout
        self._cancel, self._cancel_lock = set(), __import__("threading").Lock()
        self.budget, self.in_use, self.peak_in_use = 10_000, 0, 0
        self.keep_images = False
        self.slots = [serve._Slot(None, None, None) for _ in range(max_inflight)]
        self.clock, self.work = clock, work

    def count(self, req):
        return 100

    def _cap(self, req):
        return 1000

    def _bytes(self, req, cap):
        return 1000

    def _launch(self, slot, req, cap):
        slot.req, slot.frame = req, _FakeFrame()
        slot.event = _Event(self.clock, self.clock.t + self.work[req.rid])
        return True


def _reqs(n, gap=0.0):
    return [serve.Request(k, (0, 0, 0, 1, 1, 1), None, 0, arrival=k * gap) for k in range(n)]


def test_watchdog_reports_a_stuck_request_and_keeps_its_slot():
    clk = _Clock()
    srv = _FakeServer(clk, {0: float("inf"), 1: 0.01, 2: 0.01, 3: 0.01}, max_inflight=2, timeout=0.05)
    done, st = srv.serve(_reqs(4), clock=clk, idle_sleep=0.0)
    by = {r.rid: r for r in done}
    assert by[0].status == S.ERR_TIMEOUT and 0.05 < by[0].done - by[0].admitted < 0.06
    assert all(by[k].status == S.OK for k in (1, 2, 3))
    assert st["timed_out"] == 1 and st["completed"] == 3
    # the stuck request still holds its slot and memory until its work ends
    stuck = [s for s in srv.slots if s.req is not None]
    assert len(stuck) == 1 and stuck[0].quarantined and srv.in_use == 1000
    srv.work = {}
    stuck[0].event.end = 0.0                 # the device work finally ends
    srv.serve([], clock=clk, idle_sleep=0.0)
    assert srv.in_use == 0 and all(s.req is None for s in srv.slots)


def test_cancellation_of_waiting_and_running_requests():
    clk = _Clock()
    reqs = _reqs(5)
    reqs[1].cancel_after = 0.0                # cancelled before it starts (one slot, request 0 runs)
    reqs[0].cancel_after = 0.02               # cancelled while it runs
    srv = _FakeServer(clk, {k: 0.05 for k in range(5)}, max_inflight=1)
    srv.cancel(3)
    done, st = srv.serve(reqs, clock=clk, idle_sleep=0.0)
    by = {r.rid: r for r in done}
    assert by[0].status == serve.CANCELLED and by[1].status == serve.CANCELLED and by[3].status == serve.CANCELLED
    assert by[2].status == S.OK and by[4].status == S.OK
    assert by[1].admitted is None and by[3].admitted is None
    assert st["cancelled"] == 3 and st["completed"] == 2 and srv.in_use == 0


def test_one_slot_serves_one_request_at_a_time_and_more_slots_overlap():
    """The serving form's plain arm is the same server with one slot: its
    requests run strictly one after another; with four slots they overlap
    and the same work ends sooner."""
    work = {k: 0.02 for k in range(8)}
    clk = _Clock()
    done1, st1 = _FakeServer(clk, work, max_inflight=1).serve(_reqs(8), clock=clk, idle_sleep=0.0)
    spans = sorted((r.admitted, r.done) for r in done1)
    assert st1["completed"] == 8 and all(a[1] <= b[0] for a, b in zip(spans, spans[1:]))
    clk = _Clock()
    done4, st4 = _FakeServer(clk, work, max_inflight=4).serve(_reqs(8), clock=clk, idle_sleep=0.0)
    spans = sorted((r.admitted, r.done) for r in done4)
    assert st4["completed"] == 8 and any(a[1] > b[0] for a, b in zip(spans, spans[1:]))
    assert st4["wall_s"] < 0.5 * st1["wall_s"]


def test_autotune_signature_separates_builds_and_search_spaces():
    from paper_1004_1302_gb300 import autotune as AT

    class _DP:
        n, dtype = 1000, "f32"

    class _Cam:
        width, height = 64, 32

    space = ((8, 16), (64, 128), (1.0,))
    a = AT.signature(_DP(), _Cam(), 1, "GPU", space=space, lib="aaaa")
    assert a == AT.signature(_DP(), _Cam(), 1, "GPU", space=space, lib="aaaa")
    assert a != AT.signature(_DP(), _Cam(), 1, "GPU", space=space, lib="bbbb")      # another build
    assert a != AT.signature(_DP(), _Cam(), 1, "GPU", space=((16,), (64,), (1.0,)), lib="aaaa")
    assert a != AT.signature(_DP(), _Cam(), 0, "GPU", space=space, lib="aaaa")
