"""Sharded rounds of Algorithm 3 over several ranks (one process per GPU).

A window's chunk-order reduction adds 1024 contiguous runs of chunks left to
right and then folds the runs pairwise.  Rank r of ``world`` takes the runs
[r B, (r + 1) B), B = ceil(1024 / world): one contiguous block of samples.
Each rank samples its block and reduces it to run sums on its GPU
(``Graph.sample_runs``); one all-gather of B x 32 bytes per window gives every
rank all 1024 run sums, which it folds (``gpm_merge_runs``) and feeds to the
window test (``gpm_window_update``, the device's single-rounding FP64 steps).
Totals, the stop window and the estimate are therefore bit-identical to a
one-GPU ``gpm_estimate`` with the same seed, slot and window.

``Graph.estimate_sharded`` runs that loop inside libgpm
(``gpm_estimate_sharded``) with the all-gather supplied as a callback;
``estimate_sharded`` below is the same loop in Python over any source of run
sums (the tests feed it the CPU oracle's).  The older round-robin chunk
deal (``Graph.sample_partials``, ``interleave``, ``merge_partials``) stays
available.
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


RUNS = 1024


def run_block(world):
    """Runs per rank, B = ceil(1024 / world)."""
    return (RUNS + world - 1) // world


def merge_runs(runs):
    """Totals of the first 1024 run sums (in run order), folded pairwise as
    the device does; bit-identical to the one-GPU reduction of the window."""
    runs = np.ascontiguousarray(runs[:RUNS])
    if len(runs) < RUNS:
        pad = np.zeros(RUNS, dtype=runs.dtype)
        pad[:len(runs)] = runs
        runs = pad
    out = _lib.Sums()
    check(_lib.load().gpm_merge_runs(C.c_void_p(runs.ctypes.data), C.byref(out)), "gpm_merge_runs")
    return out


def runs_from_partials(parts, count, rank, world):
    """The run sums rank `rank` computes from its chunks' partials (chunk
    order, the rank's block only): run t adds chunks [t per, (t + 1) per)
    left to right.  Host mirror of the device's reduce_runs, for sources of
    chunk partials other than the GPU (the CPU oracle in the tests)."""
    nch = (count + 63) // 64
    per = (nch + RUNS - 1) // RUNS
    B = run_block(world)
    out = np.zeros(B, dtype=parts.dtype)
    lo = rank * B
    for t in range(B):
        g = lo + t
        if g >= RUNS:
            break
        a, b = g * per - lo * per, min((g + 1) * per, nch) - lo * per
        acc_s = acc_q = 0.0
        hits = n = 0
        for i in range(max(a, 0), max(b, 0)):
            acc_s += float(parts["sum"][i])
            acc_q += float(parts["sumsq"][i])
            hits += int(parts["hits"][i])
            n += int(parts["n"][i])
        out[t] = (acc_s, acc_q, hits, n)
    return out


def rank_samples(count, rank, world):
    """The contiguous sample range [lo, hi) of rank's run block in a window of count."""
    nch = (count + 63) // 64
    per = (nch + RUNS - 1) // RUNS
    B = run_block(world)
    c_lo = min(rank * B * per, nch)
    c_hi = min(min((rank + 1) * B, RUNS) * per, nch)
    return min(64 * c_lo, count), min(64 * c_hi, count)


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


def estimate_sharded(runs_fn, eps, delta, window, rank, world, gather, n_min=None, n_max=1 << 40, state=None,
                     max_rounds=None):
    """Algorithm 3 with each window split over ``world`` ranks by run blocks.

    runs_fn(first, count, rank, world) returns this rank's B run sums of
    samples [first, first + count) (``Graph.sample_runs`` with the pattern,
    seed and slot bound); gather(local) returns every rank's array in rank
    order.  Returns the fields of a one-GPU estimate and, under "state", the
    running window state.

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
        local = runs_fn(first, window, rank, world)
        merged = merge_runs(np.concatenate(gather(local)))
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


def torch_allgather_bytes(group=None):
    """Fixed-size all-gather of byte blocks over torch.distributed (gloo or
    NCCL), for ``Graph.estimate_sharded``: gather(block) returns the ranks'
    blocks concatenated in rank order."""
    import torch
    import torch.distributed as dist

    def gather(block):
        world = dist.get_world_size(group)
        dev = torch.device("cuda") if dist.get_backend(group) == "nccl" else torch.device("cpu")
        t = torch.from_numpy(block).to(dev)
        outs = [torch.empty_like(t) for _ in range(world)]
        dist.all_gather(outs, t, group=group)
        return torch.cat(outs).cpu().numpy()

    return gather
