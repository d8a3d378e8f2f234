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
    reqs = [serve.Request(k, (0, 0, 0, 1, 1, 1), None, 0) for k in range(50)]
    a = [r.arrival for r in serve.poisson_arrivals(reqs, rate=10.0, seed=3)]
    reqs2 = [serve.Request(k, (0, 0, 0, 1, 1, 1), None, 0) for k in range(50)]
    b = [r.arrival for r in serve.poisson_arrivals(reqs2, rate=10.0, seed=3)]
    assert a == b and all(x < y for x, y in zip(a, a[1:]))
    assert 2.0 < a[-1] < 10.0     # 50 arrivals at 10/s
