"""GPU tests of the serving form: region-of-interest cut, admission by
memory, and identical results alone and in a concurrent mix."""
import numpy as np
import pytest

import synth
from tests._common import TOL, image_error

pytestmark = pytest.mark.gpu

SIDE = 96   # a 96^3 resident lattice keeps these tests small


@pytest.fixture(scope="module")
def resident():
    import torch
    from paper_1004_1302_gb300 import splotch as S
    S.build()
    S.load()
    x, y, z, h, v = synth.lattice(SIDE)
    host = synth.ParticleSet(x, y, z, h, v, [synth.Species(0, x.size, use_log=1, brightness=0.3, absorption=0.05)])
    dp = S.upload(host, "cuda", "f16")
    torch.cuda.synchronize()
    return host, dp


def _requests(n, count=8, seed=3):
    from paper_1004_1302_gb300.serve import Request
    stream = synth.request_stream(count, n, seed=seed, n_range=(2e4, 3e5),
                                  resolutions=((128, 128), (200, 150), (256, 160)))
    return [Request(k, box, cam, mode) for k, (box, cam, mode) in enumerate(stream)]


def _server(dp, **kw):
    from paper_1004_1302_gb300.serve import RenderServer
    return RenderServer(dp, synth.colormap(), dp.species[0], keep_images=True, **kw)


def test_roi_cut_and_render_match_oracle(resident):
    from paper_1004_1302_gb300 import splotch as S
    from tests._common import oracle_render
    host, dp = resident
    req = _requests(dp.n, count=1, seed=11)[0]
    done, st = _server(dp, max_inflight=1).serve([req])
    assert done[0].status == S.OK and st["completed"] == 1
    lo = np.asarray(req.box[:3], dtype=np.float32)
    hi = np.asarray(req.box[3:], dtype=np.float32)
    p = np.stack([host.x, host.y, host.z], axis=1)
    inside = np.all((p >= lo) & (p < hi), axis=1)
    assert inside.sum() == done[0].n > 0
    idx = np.nonzero(inside)[0]
    sp = synth.Species(0, idx.size, use_log=1, brightness=0.3, absorption=0.05)
    cut = synth.ParticleSet(host.x[idx], host.y[idx], host.z[idx], host.h[idx], host.v[idx], [sp])
    o = oracle_render(cut, req.camera, synth.colormap(), req.mode, dtype="f16")
    assert (image_error(done[0].image.cpu().numpy(), o.image) <= TOL).all()


def test_alone_equals_mixed(resident):
    import torch
    from paper_1004_1302_gb300 import splotch as S
    _, dp = resident
    alone = {}
    for r in _requests(dp.n):
        done, _ = _server(dp, max_inflight=1).serve([r])
        assert done[0].status == S.OK
        alone[r.rid] = done[0].image
    mixed_reqs = _requests(dp.n)
    for k, r in enumerate(mixed_reqs):
        r.arrival = 0.002 * k
    done, st = _server(dp, max_inflight=4).serve(mixed_reqs)
    assert st["completed"] == len(mixed_reqs)
    for r in done:
        assert torch.equal(r.image, alone[r.rid]), r.rid


def test_admission_by_memory(resident):
    from paper_1004_1302_gb300 import splotch as S
    _, dp = resident
    reqs = _requests(dp.n, count=6, seed=5)
    srv = _server(dp, max_inflight=4)
    sizes = []
    for r in reqs:
        r.n = srv.count(r)
        sizes.append(srv._bytes(r, srv._cap(r)))
    # a budget that holds the largest request alone: everything completes, never over budget
    budget = max(sizes)
    srv = _server(dp, max_inflight=4, memory_budget=budget)
    done, st = srv.serve(_requests(dp.n, count=6, seed=5))
    assert st["completed"] == 6 and srv.peak_in_use <= budget
    # a budget below the largest request refuses that one and serves the rest
    big = int(np.argmax(sizes))
    srv = _server(dp, max_inflight=4, memory_budget=max(sizes) - 1)
    done, st = srv.serve(_requests(dp.n, count=6, seed=5))
    by_id = {r.rid: r for r in done}
    assert by_id[big].status == S.ERR_OOM_ADMISSION and st["refused"] == 1 and st["completed"] == 5
