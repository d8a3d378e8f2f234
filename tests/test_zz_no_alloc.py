"""The depth sort for callers that cannot allocate device memory (a renderer
inside a host application that owns all device memory through its own pool,
or a loop that may not call cudaMalloc after start-up).

It is called through the C ABI and must give exactly the order of the
allocating path (splotch_sort, read with splotch_get_order), on two calls in
a row with different inputs, since the second call reuses the fixed scratch
array the first one left behind.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_no_alloc_sort_matches_allocating_sort():
    import torch
    from paper_1004_1302_gb300 import splotch as S
    S.build()
    lib = S.load()
    pal = synth.colormap()
    cases = [synth.two_species(n_gas=120_000, n_dm=80_000, width=640, height=360),
             synth.plummer_mixture(n=S.NO_ALLOC_MAX_KEYS)]
    for ps, cam in cases:
        dp = S.upload(ps, "cuda", "f32")
        fr = S.Frame(dp, cam, pal, S.ABSORPTIVE)
        fr.render()
        ref = fr.order().cpu().numpy()
        key, _ = fr.keys()
        n = ps.n
        order = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        count = torch.zeros(1, dtype=torch.int32, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        for _ in range(2):
            st = lib.splotch_sort_keys_no_alloc(key.data_ptr(), n, order.data_ptr(), count.data_ptr(), stream)
            assert st == S.OK
            torch.cuda.synchronize()
            v = int(count.item())
            assert v == ref.size > 0
            np.testing.assert_array_equal(order[:v].cpu().numpy(), ref)
    # one key more than the fixed scratch holds is refused before anything runs
    big = S.NO_ALLOC_MAX_KEYS + 1
    assert lib.splotch_sort_keys_no_alloc(ctypes.c_void_p(key.data_ptr()), big, ctypes.c_void_p(order.data_ptr()),
                                          ctypes.c_void_p(count.data_ptr()), None) == S.ERR_ARG
    # so is a key pointer off the 16-byte boundary the vector loads need (checked on the host: no launch)
    assert lib.splotch_sort_keys_no_alloc(ctypes.c_void_p(key.data_ptr() + 4), 16, ctypes.c_void_p(order.data_ptr()),
                                          ctypes.c_void_p(count.data_ptr()), None) == S.ERR_ARG
    torch.cuda.synchronize()
