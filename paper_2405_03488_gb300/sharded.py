"""Sharded rounds of Algorithm 3 over several ranks (one process per GPU).

Within every window the 64-sample chunks are dealt round robin (chunk c to
rank c mod world); each rank draws its chunks with ``Graph.sample_partials``,
the ranks' partial arrays are gathered, interleaved back into chunk order and
merged with the device's fixed-order reduction (``gpm_merge_partials``), and
the window test runs on every rank with the same single-rounding FP64 steps
as the device (``gpm_window_update``).  Totals, the stop window and the
estimate are therefore bit-identical to a one-GPU ``gpm_estimate`` with the
same seed, slot and window.  The only exchange is one gather of
32 bytes per chunk per window.
"""
import ctypes as C

import numpy as np

from . import _lib
from ._lib import check


def interleave(parts_by_rank):
    """Chunk-order array from per-rank arrays (rank r holds chunks r, r + W, ...)."""
    world = len(parts_by_rank)
    total = sum(len(p) for p in parts_by_rank)
    out = np.zeros(total, dtype=parts_by_rank[0].dtype)
    for r, p in enumerate(parts_by_rank):
        out[r::world][:len(p)] = p
    return out


def merge_partials(parts):
    """Totals of chunk partials in chunk order, bit-identical to the device's reduction."""
    parts = np.ascontiguousarray(parts)
    out = _lib.Sums()
    check(_lib.load().gpm_merge_partials(C.c_void_p(parts.ctypes.data), len(parts), C.byref(out)),
          "gpm_merge_partials")
    return out


def window_update(state, sums, z, eps, n_min, n_max):
    check(_lib.load().gpm_window_update(C.byref(state), C.byref(sums), z, eps, n_min, n_max), "gpm_window_update")
    return state


def torch_gather(group=None):
    """A gather over torch.distributed (gloo or NCCL): every rank receives
    every rank's partial array, in rank order."""
    import torch
    import torch.distributed as dist

    def gather(local):
        world = dist.get_world_size(group)
        dev = torch.device("cuda") if dist.get_backend(group) == "nccl" else torch.device("cpu")
        raw = torch.from_numpy(local.view(np.uint8).copy()).to(dev)
        size = torch.tensor([raw.numel()], dtype=torch.int64, device=dev)
        sizes = [torch.zeros_like(size) for _ in range(world)]
        dist.all_gather(sizes, size, group=group)
        cap = int(max(s.item() for s in sizes))
        buf = torch.zeros(cap, dtype=torch.uint8, device=dev)
        buf[:raw.numel()] = raw
        bufs = [torch.zeros_like(buf) for _ in range(world)]
        dist.all_gather(bufs, buf, group=group)
        return [b[:int(s.item())].cpu().numpy().view(local.dtype) for b, s in zip(bufs, sizes)]

    return gather


def estimate_sharded(partials_fn, eps, delta, window, rank, world, gather, n_min=None, n_max=1 << 40, state=None,
                     max_rounds=None):
    """Algorithm 3 with each window's chunks split over ``world`` ranks.

    partials_fn(first, count, rank, world) returns this rank's chunk partials
    of samples [first, first + count) (``Graph.sample_partials`` with the
    pattern, seed and slot bound); gather(local) returns every rank's array in
    rank order.  Returns the fields of a one-GPU estimate and, under "state",
    the running window state.

    Checkpoint and resume: ``max_rounds`` stops after that many windows of
    this call; the returned state (a ``gpm_window``, 72 bytes, ``bytes(state)``
    to save, ``_lib.Window.from_buffer_copy`` to load) passed back as ``state``
    continues the run.  Window r always covers samples [r W, (r+1) W) of the
    counter-based streams, so a resumed run equals the uninterrupted one bit
    for bit."""
    if not (eps > 0 and 0 < delta < 1 and window > 0):
        raise ValueError("eps > 0, 0 < delta < 1 and window > 0 are required")
    z = _lib.load().gpm_normal_quantile(1.0 - delta / 2.0)
    n_min = window if n_min is None else n_min
    if state is None:
        st = _lib.Window()
        st.active = 1
    else:
        st = _lib.Window.from_buffer_copy(state)
    done = 0
    while st.active and (max_rounds is None or done < max_rounds):
        first = st.rounds * window
        local = partials_fn(first, window, rank, world)
        merged = merge_partials(interleave(gather(local)))
        window_update(st, merged, z, eps, n_min, n_max)
        done += 1
    return {"estimate": st.mu, "ci_half_width": st.half, "eps_hat": st.eps_hat, "samples": st.n,
            "hits": st.hits, "rounds": st.rounds, "converged": st.converged, "sum": st.sum, "sumsq": st.sumsq,
            "active": st.active, "state": st}


def torch_allreduce_sum(group=None):
    """Integer sum over torch.distributed ranks (gloo or NCCL)."""
    import torch
    import torch.distributed as dist

    def allreduce(x):
        dev = torch.device("cuda") if dist.get_backend(group) == "nccl" else torch.device("cpu")
        t = torch.tensor([int(x)], dtype=torch.int64, device=dev)
        dist.all_reduce(t, group=group)
        return int(t.item())

    return allreduce


def gs_estimate_sharded(count_fn, colors, k, rank, world, allreduce):
    """GS over ranks by colour class: count_fn(rank, world) is this rank's
    exact count over its classes (``Graph.gs_count_classes``), allreduce sums
    the integers; the estimate is the total times colors^(k-1)."""
    total = allreduce(count_fn(rank, world))
    return {"exact_count": total, "estimate": float(total) * float(colors) ** (k - 1)}
