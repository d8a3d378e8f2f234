"""The library built with device index checks (-DSPLOTCH_DEVICE_CHECKS):
every gather and scatter index of the sort, binning and render kernels is
tested against the workspace layout, a failed test records its source line
and SPLOTCH_ERR_STATE and skips the access.  Frames of the parity cases,
including a tile-entry overflow, must pass every check and give the release
build's images bit for bit."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = r'''
import sys
sys.path.insert(0, {root!r})
import numpy as np
import synth
from dataclasses import replace
from tests._common import small_two_species
from paper_1004_1302_gb300 import splotch as S

def frames():
    pal = synth.colormap()
    ps, cam = small_two_species(30_000, 203, 117)
    for mode in (0, 1, 2):
        for tile in (8, 16, 32):
            yield f"m{{mode}}t{{tile}}", ps, cam, dict(mode=mode, tile=tile), None
    vs = synth.vector_fields(ps)
    vs.species = [replace(vs.species[0], use_vector=1, modulate=1), replace(vs.species[1], modulate=1)]
    yield "vector", vs, cam, dict(mode=1, tile=16), None
    yield "split_all", ps, cam, dict(mode=1, tile=16, large_threshold_px=1), None
    yield "overflow", ps, cam, dict(mode=1, tile=16), 2_000

out = {{}}
imgs = {{}}
for name, ps, cam, kw, cap in frames():
    mode = kw.pop("mode")
    fr = S.Frame(S.upload(ps, "cuda", "f32"), cam, synth.colormap(), mode, max_tile_entries=cap, **kw)
    if cap is not None:               # the first frame overflows its capacity
        fr.run()
        inf = fr.info()
        out[name + "_first"] = [int(inf.status), int(inf.check_line)]
    img = fr.render().cpu().numpy()
    inf = fr.info()
    out[name] = [int(inf.status), int(inf.check_line)]
    imgs[name] = img
np.savez({npz!r}, **imgs)
print("RESULT", __import__("json").dumps(out))
'''


def _run(tmp_path, checked: bool, payload: str):
    npz = str(tmp_path / ("checked.npz" if checked else "release.npz"))
    env = dict(os.environ, SPLOTCH_CHECKED="1" if checked else "0", SPLOTCH_TILE_PAYLOAD=payload)
    r = subprocess.run([sys.executable, "-c", CASES.format(root=ROOT, npz=npz)], capture_output=True, text=True,
                       env=env, cwd=ROOT, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):]), np.load(npz)


@pytest.mark.parametrize("payload", ["0", "1"])   # tile boxes gathered by binning, or carried by the sort
def test_checked_build_passes_every_check_and_matches_release(tmp_path, payload):
    from paper_1004_1302_gb300 import splotch as S
    S.build()
    S.build(checked=True)
    res_c, img_c = _run(tmp_path, True, payload)
    res_r, img_r = _run(tmp_path, False, payload)
    assert res_c["overflow_first"] == [S.ERR_WORKSPACE, 0]        # overflow reported, no index out of range
    for name, (status, line) in res_c.items():
        if name.endswith("_first"):
            continue
        assert status == S.OK and line == 0, (name, status, line)
        np.testing.assert_array_equal(img_c[name], img_r[name])
    assert res_r == res_c
