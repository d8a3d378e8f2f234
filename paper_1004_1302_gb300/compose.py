"""Composition of partial images rendered from depth slabs of one particle set.

Eq. 1 of the paper (Section 2) integrates to an affine map per pixel and
channel: light entering a slab from behind leaves it as I_out = C + T I_in,
where C is the slab's own contribution (rendered front to back with a
background of 0) and T its transmittance.  Two slabs, `front` nearer the
camera than `back`, combine into (C_f + T_f C_b, T_f T_b): an associative but
not commutative operator, so slabs must be combined in depth order.  In
emission mode T = 1 and the operator reduces to a sum (the paper's MPI
reduction of partial images, Section 3.1); with E = A it composes 1 - T.

This is the one exchange step a depth-sharded render needs.  Partial images
on the device compose in the CUDA library (`splotch_compose`); host arrays
(numpy or CPU tensors, as gathered over a CPU process group) compose with the
same operator in host arithmetic.
"""
from __future__ import annotations


def compose_device(front, back, out=None, stream=None):
    """(C, T) of `front` over `back` for float32 CUDA tensors, in the CUDA
    library; `out` = (C, T) tensors to write (may be the inputs)."""
    import torch

    from . import splotch as S
    cf, tf = front
    cb, tb = back
    for t in (cf, tf, cb, tb):
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.numel() == cf.numel()):
            raise ValueError("partial images must be contiguous float32 CUDA tensors of one shape")
    co, to = (torch.empty_like(cf), torch.empty_like(tf)) if out is None else out
    st = (stream or torch.cuda.current_stream(cf.device)).cuda_stream
    S.splotch_compose(cf.data_ptr(), tf.data_ptr(), cb.data_ptr(), tb.data_ptr(), co.data_ptr(),
                      to.data_ptr() if to is not None else None, cf.numel(), st)
    return co, to


def compose_pair(front, back):
    """(C, T) of `front` (nearer the camera) over `back`."""
    cf, tf = front
    cb, tb = back
    if getattr(cf, "is_cuda", False):
        return compose_device(front, back)
    return cf + tf * cb, tf * tb


def compose_slabs(partials):
    """Fold (C, T) partials given nearest slab first."""
    it = iter(partials)
    acc = next(it)
    for p in it:
        acc = compose_pair(acc, p)
    return acc


def gather_compose(c, t, group=None, dst: int = 0):
    """Gather every rank's (C, T) (rank r holds depth slab r, rank 0 the
    nearest) and compose them on rank `dst`; returns (C, T) there and None on
    the other ranks."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    packed = torch.cat([c.reshape(-1), t.reshape(-1)])
    bufs = [torch.empty_like(packed) for _ in range(world)] if rank == dst else None
    dist.gather(packed, bufs, dst=dst, group=group)
    if rank != dst:
        return None
    n = c.numel()
    parts = [(b[:n].reshape(c.shape), b[n:].reshape(t.shape)) for b in bufs]
    return compose_slabs(parts)
