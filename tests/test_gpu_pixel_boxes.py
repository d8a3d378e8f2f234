"""The transform stores the pixel boxes only when binning reads them or the
caller asks (splotch_render_params.keep_pixel_boxes): either way the frame
(keys, render order, tile lists, image) is the same bit for bit, a box
request without stored boxes is refused, and the fragment count (taken over
the stored boxes, or over a widened radius clipped to the image) agrees."""
import numpy as np
import pytest

import synth
from tests._common import small_two_species

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_frames_with_and_without_pixel_boxes_agree(mode):
    from paper_1004_1302_gb300 import splotch as S
    S.build()
    ps, cam = small_two_species(60_000, 420, 250)
    pal = synth.colormap()
    out = {}
    for keep in (True, False):
        fr = S.Frame(S.upload(ps, "cuda", "f32"), cam, pal, mode, tile=16, keep_pixel_boxes=keep)
        img = fr.render().cpu().numpy()
        key, box = fr.keys()
        offs, lst = fr.tile_lists()
        out[keep] = (img, key.cpu().numpy(), fr.order().cpu().numpy(), offs.cpu().numpy(), lst.cpu().numpy(),
                     fr.fragments())
        if keep:
            assert box is not None and box.shape == (ps.n, 4)
        else:
            assert box is None
            with pytest.raises(S.SplotchError) as e:
                fr.keys(boxes=True)
            assert e.value.status == S.ERR_STATE
    for a, b in zip(out[True], out[False]):
        if isinstance(a, np.ndarray):
            np.testing.assert_array_equal(a, b)
        else:
            assert a == b and a > 0
