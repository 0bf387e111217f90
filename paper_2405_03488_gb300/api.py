"""Python face of libgpm for PyTorch users: graphs held in torch tensors (or
host numpy arrays), calls on torch's current CUDA stream.  Marshalling only;
the work runs in libgpm.so."""
import ctypes as C

import numpy as np
import torch

from . import _lib
from . import graphs as _graphs
from ._lib import (DEVICE_PTRS, EXACT, GS, HYBRID, NS, NS_LEARNED, RELABEL_DEGREE,  # noqa: F401
                   VALIDATE, VERIFY_CHECK, VERIFY_INTERSECT, VERIFY_LAZY, check, make_pattern)

RECORD_DTYPE = np.dtype([("factor", np.uint64, _lib.MAX_K), ("w_u64", np.uint64), ("w_f64", np.float64),
                         ("vert", np.uint32, _lib.MAX_K), ("aux", np.uint32, _lib.MAX_K), ("hit", np.uint8),
                         ("depth", np.uint8), ("overflow", np.uint8), ("pad", np.uint8), ("sectors", np.uint32)])
assert RECORD_DTYPE.itemsize == C.sizeof(_lib.SampleRecord)
PARTIAL_DTYPE = np.dtype([("sum", np.float64), ("sumsq", np.float64), ("hits", np.uint64), ("n", np.uint64)])
assert PARTIAL_DTYPE.itemsize == C.sizeof(_lib.Partial)


def pattern(spec, induced=None):
    """A gpm_pattern from a name ('4-clique', 'house', ...) or (k, edges[, induced])."""
    if isinstance(spec, _lib.Pattern):
        return spec
    if isinstance(spec, str):
        k, edges = _graphs.pattern(spec)
        ind = False
    else:
        k, edges = spec[0], spec[1]
        ind = bool(spec[2]) if len(spec) > 2 else False
    if induced is not None:
        ind = induced
    return make_pattern(k, edges, ind)


def config(**kw):
    cfg = _lib.Config()
    mlp = kw.pop("mlp", None)
    selector = kw.pop("selector", None)
    for key, val in kw.items():
        if val is None:
            continue
        if key == "verify" and isinstance(val, str):
            val = {"intersect": VERIFY_INTERSECT, "check": VERIFY_CHECK, "lazy": VERIFY_LAZY}[val]
        setattr(cfg, key, val)
    keep = []
    if mlp is not None:
        st = mlp.c_struct()
        cfg.mlp = C.pointer(st)
        keep += [mlp, st]
    if selector is not None:
        ss = selector.c_struct()
        cfg.selector = C.pointer(ss)
        keep += [selector, ss]
    cfg._keep = keep
    return cfg


def _stream_ptr():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class Graph:
    """A resident data graph.

    ``row_ptr`` (int64 / uint64, n + 1) and ``col`` (int32 / uint32, 2m) are
    either CUDA tensors, which the handle borrows (kept alive here), or host
    arrays, which the library copies to the device."""

    def __init__(self, row_ptr, col, validate=False, relabel=False):
        L = _lib.load()
        self._keep = None
        flags = (VALIDATE if validate else 0) | (RELABEL_DEGREE if relabel else 0)
        h = C.c_void_p()
        if isinstance(row_ptr, torch.Tensor) and row_ptr.is_cuda:
            row_ptr = row_ptr.contiguous().to(torch.int64)
            col = col.contiguous().to(torch.int32)
            self._keep = (row_ptr, col)
            n = row_ptr.numel() - 1
            code = L.gpm_load_csr(n, C.c_void_p(row_ptr.data_ptr()), C.c_void_p(col.data_ptr()),
                                  flags | DEVICE_PTRS, _stream_ptr(), C.byref(h))
        else:
            if isinstance(row_ptr, torch.Tensor):
                row_ptr, col = row_ptr.numpy(), col.numpy()
            rp = np.ascontiguousarray(row_ptr, dtype=np.uint64)
            cc = np.ascontiguousarray(col, dtype=np.uint32)
            n = len(rp) - 1
            code = L.gpm_load_csr(n, C.c_void_p(rp.ctypes.data), C.c_void_p(cc.ctypes.data if len(cc) else 0),
                                  flags, _stream_ptr(), C.byref(h))
        check(code, "gpm_load_csr")
        self.h = h
        n_, m_, nnz_, md_ = C.c_uint64(), C.c_uint64(), C.c_uint64(), C.c_uint64()
        check(L.gpm_graph_info(h, C.byref(n_), C.byref(m_), C.byref(nnz_), C.byref(md_)), "gpm_graph_info")
        self.n, self.m, self.nnz, self.max_degree = n_.value, m_.value, nnz_.value, md_.value

    def relabel_map(self):
        """New id of every loaded vertex (a graph loaded with relabel=True)."""
        out = np.zeros(max(self.n, 1), dtype=np.uint32)
        check(_lib.load().gpm_relabel_map(self.h, C.c_void_p(out.ctypes.data)), "gpm_relabel_map")
        return out[:self.n]

    def close(self):
        if getattr(self, "h", None):
            _lib.load().gpm_free_graph(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def estimate(self, pat, scheme=NS, eps=0.01, delta=0.01, seed=1, allow_unconverged=True, **cfg):
        res = _lib.Result()
        pp = pattern(pat)
        c = config(**cfg)
        code = _lib.load().gpm_estimate(self.h, C.byref(pp), scheme, eps, delta, seed, C.byref(c), C.byref(res))
        # NOT_CONVERGED and ABORTED still fill the result
        ok = (_lib.GPM_OK, _lib.GPM_ERR_NOT_CONVERGED, _lib.GPM_ERR_ABORTED) if allow_unconverged else (_lib.GPM_OK,)
        check(code, "gpm_estimate", ok)
        d = res.as_dict()
        d["status"] = code
        return d

    def estimate_batch(self, pats, eps, delta=0.01, seed=1, **cfg):
        L = _lib.load()
        arr = (_lib.Pattern * len(pats))(*[pattern(p) for p in pats])
        e = (C.c_double * len(pats))(*eps)
        res = (_lib.Result * len(pats))()
        c = config(**cfg)
        code = L.gpm_estimate_batch(self.h, len(pats), arr, e, delta, seed, C.byref(c), res)
        check(code, "gpm_estimate_batch", (_lib.GPM_OK, _lib.GPM_ERR_NOT_CONVERGED))
        return [r.as_dict() for r in res]

    def hybrid_model(self, pat, eps=0.01, delta=0.01, seed=1, **cfg):
        """The hybrid choice's inputs and decisions (no engine run)."""
        info = _lib.HybridInfo()
        pp = pattern(pat)
        c = config(**cfg)
        check(_lib.load().gpm_hybrid_model(self.h, C.byref(pp), eps, delta, seed, C.byref(c), C.byref(info)),
              "gpm_hybrid_model")
        return info.as_dict()

    def profile(self, pat, kind="pilot", frac=0.1, eps=0.01, delta=0.01, seed=1, **cfg):
        """Predicted NS sample count: kind "pilot" (a window on G) or
        "sparsified" (the paper's profiler on a frac-edge-sparsified G')."""
        info = _lib.ProfileInfo()
        pp = pattern(pat)
        c = config(**cfg)
        k = {"pilot": 0, "sparsified": 1}[kind]
        check(_lib.load().gpm_profile(self.h, C.byref(pp), k, frac, eps, delta, seed, C.byref(c), C.byref(info)),
              "gpm_profile")
        return info.as_dict()

    def autotune(self, pats, seed=1, **cfg):
        """Fastest launch shape for these patterns: dict(block_warps, cap)."""
        arr = (_lib.Pattern * len(pats))(*[pattern(p) for p in pats])
        c = config(**cfg)
        check(_lib.load().gpm_autotune(self.h, len(pats), arr, seed, C.byref(c)), "gpm_autotune")
        return {"block_warps": c.block_warps, "cap": c.cap}

    def sample_sums(self, pat, seed, first, count, **cfg):
        out = _lib.Sums()
        pp = pattern(pat)
        c = config(**cfg)
        check(_lib.load().gpm_sample_sums(self.h, C.byref(pp), seed, first, count, C.byref(c), C.byref(out)),
              "gpm_sample_sums")
        return out

    def sample_partials(self, pat, seed, first, count, rank=0, world=1, **cfg):
        """Per-chunk partials of the 64-sample chunks c = rank (mod world) of
        [first, first + count), in chunk order (a structured array with fields
        sum, sumsq, hits, n)."""
        nchunks = (count + 63) // 64
        mine = max(0, (nchunks - rank + world - 1) // world) if nchunks > rank else 0
        out = np.zeros(max(mine, 1), dtype=PARTIAL_DTYPE)
        n = C.c_uint64()
        pp = pattern(pat)
        c = config(**cfg)
        check(_lib.load().gpm_sample_partials(self.h, C.byref(pp), seed, first, count, rank, world, C.byref(c),
                                              C.c_void_p(out.ctypes.data), C.byref(n)), "gpm_sample_partials")
        assert n.value == mine
        return out[:mine]

    def sample_runs(self, pat, seed, first, count, rank=0, world=1, **cfg):
        """This rank's B = ceil(1024 / world) run sums of samples [first, first +
        count) (a structured array with fields sum, sumsq, hits, n)."""
        B = (1024 + world - 1) // world
        out = np.zeros(B, dtype=PARTIAL_DTYPE)
        pp = pattern(pat)
        c = config(**cfg)
        check(_lib.load().gpm_sample_runs(self.h, C.byref(pp), seed, first, count, rank, world, C.byref(c),
                                          C.c_void_p(out.ctypes.data)), "gpm_sample_runs")
        return out

    def estimate_sharded(self, pat, rank, world, gather, eps=0.01, delta=0.01, seed=1, state=None, max_rounds=0,
                         **cfg):
        """gpm_estimate_sharded: this rank's part of an estimate over `world`
        ranks.  gather(block) receives this rank's bytes (numpy uint8) and
        returns all ranks' blocks concatenated in rank order.  state: a
        _lib.Window to continue (written back) or None."""
        res = _lib.Result()
        pp = pattern(pat)
        c = config(**cfg)
        err = []

        def cb(ctx, send, recv, nbytes):
            try:
                blk = np.ctypeslib.as_array(C.cast(send, C.POINTER(C.c_uint8)), shape=(nbytes,)).copy()
                allb = np.ascontiguousarray(gather(blk), dtype=np.uint8)
                if allb.size != nbytes * world:
                    raise ValueError("gather returned %d bytes, expected %d" % (allb.size, nbytes * world))
                C.memmove(recv, allb.ctypes.data, allb.size)
                return 0
            except Exception as e:  # reported to the library as a failed collective
                err.append(e)
                return 1

        fn = _lib.ALLGATHER_FN(cb)
        code = _lib.load().gpm_estimate_sharded(self.h, C.byref(pp), eps, delta, seed, rank, world, C.byref(c),
                                                C.cast(fn, C.c_void_p), None,
                                                C.byref(state) if state is not None else None, max_rounds,
                                                C.byref(res))
        if err:
            raise err[0]
        check(code, "gpm_estimate_sharded", (_lib.GPM_OK, _lib.GPM_ERR_NOT_CONVERGED, _lib.GPM_ERR_ABORTED))
        d = res.as_dict()
        d["status"] = code
        return d

    def trace(self, pat, seed, first, count, **cfg):
        recs = np.zeros(count, dtype=RECORD_DTYPE)
        pp = pattern(pat)
        c = config(**cfg)
        check(_lib.load().gpm_trace(self.h, C.byref(pp), seed, first, count, C.byref(c),
                                    C.c_void_p(recs.ctypes.data)), "gpm_trace")
        return recs

    def exact_count(self, pat):
        out = C.c_uint64()
        pp = pattern(pat)
        check(_lib.load().gpm_exact_count(self.h, C.byref(pp), C.byref(out)), "gpm_exact_count")
        return out.value

    def sparsify(self, colors, seed, colouring=0, slot=0):
        """Colour sparsification into new CUDA tensors (row_ptr, col)."""
        row = torch.empty(self.n + 1, dtype=torch.int64, device="cuda")
        col = torch.empty(max(self.nnz, 1), dtype=torch.int32, device="cuda")
        kept = C.c_uint64()
        check(_lib.load().gpm_sparsify(self.h, colors, seed, colouring, slot, C.c_void_p(row.data_ptr()),
                                       C.c_void_p(col.data_ptr()), C.byref(kept)), "gpm_sparsify")
        return row, col[:kept.value]

    def gs_count_classes(self, pat, colors, seed, rank, world, colouring=0, slot=0, max_seconds=0.0):
        """Exact count, on the colour-sparsified graph, of the matches in the colour
        classes c = rank (mod world): one rank's share of a sharded GS count."""
        out = C.c_uint64()
        pp = pattern(pat)
        check(_lib.load().gpm_gs_count_classes(self.h, C.byref(pp), colors, seed, colouring, slot, rank, world,
                                               max_seconds, C.byref(out)), "gpm_gs_count_classes")
        return out.value

    def sparsify_edges(self, p, seed, colouring=0, slot=0):
        """Bernoulli edge sparsification (keep probability p) into new CUDA tensors (row_ptr, col)."""
        row = torch.empty(self.n + 1, dtype=torch.int64, device="cuda")
        col = torch.empty(max(self.nnz, 1), dtype=torch.int32, device="cuda")
        kept = C.c_uint64()
        check(_lib.load().gpm_sparsify_edges(self.h, p, seed, colouring, slot, C.c_void_p(row.data_ptr()),
                                             C.c_void_p(col.data_ptr()), C.byref(kept)), "gpm_sparsify_edges")
        return row, col[:kept.value]

    def abort(self):
        check(_lib.load().gpm_abort(self.h), "gpm_abort")


def gather_probe(nbytes, chain=4, hops=1 << 28):
    """Random 32-byte-sector gather throughput (bytes/s) over a buffer of nbytes,
    chains of `chain` dependent hops (the sampler's access pattern)."""
    out = C.c_double()
    check(_lib.load().gpm_gather_probe(nbytes, chain, hops, C.byref(out)), "gpm_gather_probe")
    return out.value


def plan(pat):
    """(order, restrictions, oriented) from the library's host planner."""
    pp = pattern(pat)
    order = (C.c_int32 * _lib.MAX_K)()
    lo = (C.c_int32 * 64)()
    hi = (C.c_int32 * 64)()
    nres = C.c_int32()
    ori = C.c_int32()
    check(_lib.load().gpm_plan(C.byref(pp), order, lo, hi, C.byref(nres), C.byref(ori)), "gpm_plan")
    return list(order[:pp.k]), [(lo[i], hi[i]) for i in range(nres.value)], ori.value


def normal_quantile(p):
    return _lib.load().gpm_normal_quantile(p)


# ------------------------------------------------------------------ learned proposal
MLP_SIZES = (("w1", 192), ("b1", 64), ("w2", 4096), ("b2", 64), ("w3", 64), ("b3", 1))
MLP_FLOATS = 4481


class Proposal:
    """Weights of the learned proposal on the GPU: FP32 master copy ``w32`` and
    the BF16 bit patterns ``w16`` the sampler reads (gpm_mlp order)."""

    def __init__(self, seed=0, device="cuda"):
        g = torch.Generator()
        g.manual_seed(int(seed))
        parts = []
        for name, n in MLP_SIZES:
            fan_in = {"w1": 3, "w2": 64, "w3": 64}.get(name)
            if fan_in:
                parts.append(torch.randn(n, generator=g) * (2.0 / fan_in) ** 0.5)
            else:
                parts.append(torch.zeros(n))
        self.w32 = torch.cat(parts).float().to(device).contiguous()
        self.w16 = self.w32.to(torch.bfloat16).view(torch.int16).contiguous()

    def c_struct(self):
        base = self.w16.data_ptr()
        ptrs, off = {}, 0
        for name, n in MLP_SIZES:
            ptrs[name] = C.c_void_p(base + 2 * off)
            off += n
        return _lib.MLP(**{k: v.value for k, v in ptrs.items()})

    def arrays16(self):
        """Host uint16 arrays (w1 [64,3], b1, w2 [64,64], b2, w3, b3)."""
        h = self.w16.cpu().numpy().view(np.uint16)
        out, off = [], 0
        for name, n in MLP_SIZES:
            a = h[off:off + n].copy()
            out.append(a.reshape(64, 3) if name == "w1" else a.reshape(64, 64) if name == "w2" else a)
            off += n
        return out

    def train(self, graph, pat, seed=1, samples=1 << 20, epochs=4, batch=8192, lr=3e-3):
        loss, rows = C.c_double(), C.c_uint64()
        pp = pattern(pat)
        check(_lib.load().gpm_train_proposal(graph.h, C.byref(pp), seed, samples, epochs, batch, lr,
                                             C.c_void_p(self.w32.data_ptr()), C.c_void_p(self.w16.data_ptr()),
                                             C.byref(loss), C.byref(rows)), "gpm_train_proposal")
        return loss.value, rows.value

    def train_rows(self, graph, feat, label, epochs=200, batch=4096, lr=1e-2):
        """Adam on given rows (CUDA float tensors feat [n, 3], label [n])."""
        feat = feat.contiguous().float()
        label = label.contiguous().float()
        loss = C.c_double()
        check(_lib.load().gpm_mlp_train(graph.h, C.c_void_p(feat.data_ptr()), C.c_void_p(label.data_ptr()),
                                        feat.shape[0], epochs, batch, lr, C.c_void_p(self.w32.data_ptr()),
                                        C.c_void_p(self.w16.data_ptr()), C.byref(loss)), "gpm_mlp_train")
        return loss.value

    def scores(self, graph, feat, tensor=False):
        """Sampler scores a_x of feature rows (CUDA float tensor [n, 3]);
        tensor=True scores them as the sampler does with mlp_tensor=1."""
        feat = feat.contiguous().float()
        out = torch.empty(feat.shape[0], dtype=torch.int32, device=feat.device)
        m = self.c_struct()
        fn = _lib.load().gpm_mlp_scores_tc if tensor else _lib.load().gpm_mlp_scores
        check(fn(graph.h, C.byref(m), C.c_void_p(feat.data_ptr()), feat.shape[0], C.c_void_p(out.data_ptr())),
              "gpm_mlp_scores_tc" if tensor else "gpm_mlp_scores")
        return out

    def loss_grad(self, graph, feat, label, w32=None):
        w = (self.w32 if w32 is None else w32).contiguous()
        grad = torch.empty(MLP_FLOATS, dtype=torch.float32, device=w.device)
        loss = C.c_double()
        check(_lib.load().gpm_mlp_loss_grad(graph.h, C.c_void_p(w.data_ptr()), C.c_void_p(feat.data_ptr()),
                                            C.c_void_p(label.data_ptr()), feat.shape[0],
                                            C.c_void_p(grad.data_ptr()), C.byref(loss)), "gpm_mlp_loss_grad")
        return loss.value, grad


def proposal_features(graph, pat, recs_dev, n):
    """Training rows from device records (torch uint8 buffer of n records)."""
    pp = pattern(pat)
    k = pp.k
    feat = torch.empty((max(n * max(k - 3, 0), 1), 3), dtype=torch.float32, device="cuda")
    label = torch.empty(max(n * max(k - 3, 0), 1), dtype=torch.float32, device="cuda")
    rows = C.c_uint64()
    check(_lib.load().gpm_proposal_features(graph.h, C.byref(pp), C.c_void_p(recs_dev.data_ptr()), n,
                                            C.c_void_p(feat.data_ptr()), C.c_void_p(label.data_ptr()),
                                            C.byref(rows)), "gpm_proposal_features")
    return feat[:rows.value], label[:rows.value]
