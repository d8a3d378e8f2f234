"""The loader: block slices read on a host thread, staged through pinned
buffers and copied to device arrays on a stream, overlapping the render of
the previous snapshot.  Expected values are numpy's reading of the file and
renders of the same particles uploaded directly."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _arrays(n, nb=5, seed=5):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal(n).astype(np.float32) * (3.0 ** k) for k in range(nb)]


def test_loader_fills_device_arrays(tmp_path):
    import torch
    from paper_1004_1302_gb300 import splotch as S
    S.build()
    S.load()
    n = 1_000_003                                   # 16 chunks of 256 KB per block and a ragged tail
    arrs = _arrays(n)
    path = str(tmp_path / "b.bin")
    synth.write_block_file(path, arrs, big_endian=True, offset_bytes=8)
    f = S.block_file(path, 5, n, True, 8)
    order = [4, 3, 2, 1, 0]
    dst = [torch.full((n,), float("nan"), dtype=torch.float32, device="cuda") for _ in order]
    st = torch.cuda.Stream()
    with S.Loader(chunk_bytes=1 << 18) as L:
        L.start(f, order, dst, 0, n, st.cuda_stream)
        L.wait()
        st.synchronize()
        for d, b in zip(dst, order):
            np.testing.assert_array_equal(d.cpu().numpy(), arrs[b])
        # a slice, and the same loader again
        part = [torch.zeros(1000, dtype=torch.float32, device="cuda")]
        L.start(f, [2], part, 123_456, 1000, st.cuda_stream)
        L.wait()
        st.synchronize()
        np.testing.assert_array_equal(part[0].cpu().numpy(), arrs[2][123_456:124_456])


def test_loader_reports_io_errors(tmp_path):
    import torch
    from paper_1004_1302_gb300 import splotch as S
    S.load()
    path = str(tmp_path / "short.bin")
    synth.write_block_file(path, _arrays(1000, nb=2))
    dst = [torch.zeros(1000, dtype=torch.float32, device="cuda")]
    with S.Loader(chunk_bytes=4096) as L:
        L.start(S.block_file(path, 3, 1000), [2], dst, 0, 1000)      # the third block is not in the file
        with pytest.raises(S.SplotchError) as e:
            L.wait()
        assert e.value.status == S.ERR_IO
        L.start(S.block_file(str(tmp_path / "none.bin"), 1, 10), [0], dst, 0, 10)
        with pytest.raises(S.SplotchError) as e:
            L.wait()
        assert e.value.status == S.ERR_IO
        with pytest.raises(S.SplotchError) as e:
            L.start(S.block_file(path, 2, 1000), [0], dst, 990, 11)
        assert e.value.status == S.ERR_ARG


def test_pipeline_images_equal_direct_uploads(tmp_path):
    """Snapshot k renders on one stream while snapshot k+1 loads on another."""
    import torch
    from paper_1004_1302_gb300 import splotch as S
    S.load()
    snaps, paths = [], []
    for k in range(3):
        ps, cam = synth.two_species(n_gas=120_000, n_dm=80_000, width=320, height=200, seed=synth.SEED + k)
        snaps.append(ps)
        paths.append(str(tmp_path / f"snap{k}.bin"))
        synth.write_block_file(paths[-1], [ps.x, ps.y, ps.z, ps.h, ps.v], big_endian=(k % 2 == 1))
    pal = synth.colormap()
    direct = []
    for ps in snaps:
        fr = S.Frame(S.upload(ps, "cuda", "f32"), cam, pal, S.ABSORPTIVE)
        direct.append(fr.render().cpu().numpy())
    n = snaps[0].n
    bufs = [[torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(5)] for _ in range(2)]
    copy, comp = torch.cuda.Stream(), torch.cuda.Stream()
    got = []
    with S.Loader(chunk_bytes=1 << 20) as L:
        L.start(S.block_file(paths[0], 5, n, False), range(5), bufs[0], 0, n, copy.cuda_stream)
        L.wait()
        for k in range(3):
            comp.wait_stream(copy)                      # snapshot k is on the device
            if k + 1 < 3:                               # load k + 1 while k renders
                copy.wait_stream(comp)                  # its buffers were last read by frame k - 1
                L.start(S.block_file(paths[k + 1], 5, n, (k + 1) % 2 == 1), range(5), bufs[(k + 1) % 2], 0, n,
                        copy.cuda_stream)
            b = bufs[k % 2]
            dp = S.DeviceParticles(*b, "f32", list(snaps[k].species))
            with torch.cuda.stream(comp):
                fr = S.Frame(dp, cam, pal, S.ABSORPTIVE)
                got.append(fr.render(comp).clone())
            if k + 1 < 3:
                L.wait()
    torch.cuda.synchronize()
    for g, d in zip(got, direct):
        np.testing.assert_array_equal(g.cpu().numpy(), d)


def test_host_pipeline_images_equal_direct_renders():
    """Frames from pinned host arrays, the copy of frame k + 1 overlapping the
    render of frame k: each image equals a direct render of its particles."""
    import torch
    from paper_1004_1302_gb300 import splotch as S
    S.load()
    snaps = [synth.two_species(n_gas=90_000, n_dm=60_000, width=300, height=180, seed=synth.SEED + k) for k in range(4)]
    pal = synth.colormap()
    cam = snaps[0][1]
    direct = [S.Frame(S.upload(ps, "cuda", "f32"), cam, pal, S.ABSORPTIVE).render().cpu().numpy() for ps, _ in snaps]
    hosts = [[torch.from_numpy(a).pin_memory() for a in (ps.x, ps.y, ps.z, ps.h, ps.v)] for ps, _ in snaps]
    pipe = S.HostPipeline(snaps[0][0].n, snaps[0][0].species, cam, pal, S.ABSORPTIVE)
    pipe.size(hosts[0])
    got = []
    for k in range(4):
        img = pipe.submit(hosts[k])
        if k % 2 == 1:                     # both host images of the pair are final after a synchronize
            pipe.synchronize()
            got += [pipe.images[0].numpy().copy(), pipe.images[1].numpy().copy()]
    assert pipe.info(0).status == 0 and pipe.info(1).status == 0
    for g, d in zip(got, direct):
        np.testing.assert_array_equal(g, d)
    assert img.shape == (180, 300, 3)
