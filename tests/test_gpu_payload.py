"""Both ways binning gets each particle's tile box give the oracle's tile
lists bit for bit: gathered by particle index in render order, or carried
through the depth sort as a payload (chosen by the library for frames whose
boxes do not fit in L2; forced here with SPLOTCH_TILE_PAYLOAD in a child
process so that small frames take it too)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import synth
from tests._common import TOL, image_error, small_two_species

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys
sys.path.insert(0, {root!r})
import numpy as np
import synth
from tests._common import small_two_species
from paper_1004_1302_gb300 import splotch as S
ps, cam = small_two_species(40_000, 330, 190)
out = {{}}
for mode in (0, 1, 2):
    for tile in (8, 16, 32):
        fr = S.Frame(S.upload(ps, "cuda", "f32"), cam, synth.colormap(), mode, tile=tile)
        img = fr.render().cpu().numpy()
        offs, lst = fr.tile_lists()
        out[f"img_{{mode}}_{{tile}}"] = img
        out[f"offs_{{mode}}_{{tile}}"] = offs.cpu().numpy().view(np.uint32)
        out[f"list_{{mode}}_{{tile}}"] = lst.cpu().numpy().view(np.uint32)
        out[f"order_{{mode}}_{{tile}}"] = fr.order().cpu().numpy().view(np.uint32)
np.savez({npz!r}, **out)
print("DONE")
'''


@pytest.mark.parametrize("payload", ["0", "1"])
def test_tile_lists_and_images_match_oracle_with_either_box_source(oracle_mod, tmp_path, payload):
    from paper_1004_1302_gb300 import splotch as S
    O = oracle_mod
    S.build()
    npz = str(tmp_path / "out.npz")
    env = dict(os.environ, SPLOTCH_TILE_PAYLOAD=payload)
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT, npz=npz)], capture_output=True, text=True,
                       env=env, cwd=ROOT, timeout=900)
    assert r.returncode == 0 and "DONE" in r.stdout, r.stderr[-3000:]
    got = np.load(npz)
    ps, cam = small_two_species(40_000, 330, 190)
    pal = synth.colormap()
    for mode in (0, 1, 2):
        for tile in (8, 16, 32):
            ref = O.render_frame(ps, cam, pal, mode, tile=tile)
            np.testing.assert_array_equal(got[f"order_{mode}_{tile}"], ref.order)
            np.testing.assert_array_equal(got[f"offs_{mode}_{tile}"].astype(np.uint64), ref.offsets)
            np.testing.assert_array_equal(got[f"list_{mode}_{tile}"], ref.tile_list)
            err = image_error(got[f"img_{mode}_{tile}"], ref.image)
            assert (err <= TOL).all(), (mode, tile, err)
