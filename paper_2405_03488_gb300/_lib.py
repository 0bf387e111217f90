"""Thin ctypes binding of libgpm.so (include/gpm.h): argument marshalling only.

Every computation runs in the library's CUDA kernels.  Importing this module
does not need a GPU; calling an entry point that touches the device does.
If libgpm.so is missing the import fails loudly (there is no CPU fallback).
"""
import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libgpm_san.so" if os.environ.get("GPM_SANITIZE") == "1" else "libgpm.so")

MAX_K = 12

GPM_OK = 0
GPM_ERR_ARG = -1
GPM_ERR_GRAPH = -2
GPM_ERR_OOM = -3
GPM_ERR_CUDA = -4
GPM_ERR_NOT_CONVERGED = -5
GPM_ERR_ABORTED = -6
GPM_ERR_UNSUPPORTED = -8
GPM_ERR_COMM = -9

NS, GS, HYBRID, NS_LEARNED, EXACT = 0, 1, 2, 3, 4
VERIFY_INTERSECT, VERIFY_CHECK, VERIFY_LAZY = 0, 1, 2
DEVICE_PTRS, VALIDATE, RELABEL_DEGREE = 1, 2, 4

STATUS_NAMES = {0: "OK", -1: "ERR_ARG", -2: "ERR_GRAPH", -3: "ERR_OOM", -4: "ERR_CUDA",
                -5: "ERR_NOT_CONVERGED", -6: "ERR_ABORTED", -8: "ERR_UNSUPPORTED", -9: "ERR_COMM"}


class Pattern(C.Structure):
    _fields_ = [("k", C.c_uint8), ("induced", C.c_uint8), ("adj", C.c_uint16 * 16)]


class MLP(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("w1", "b1", "w2", "b2", "w3", "b3")]


class Config(C.Structure):
    _fields_ = [("window", C.c_uint64), ("n_min", C.c_uint64), ("n_max", C.c_uint64),
                ("max_seconds", C.c_double), ("colors", C.c_uint32), ("slot", C.c_uint32),
                ("verify", C.c_uint32), ("grid_blocks", C.c_uint32), ("block_warps", C.c_uint32),
                ("cap", C.c_uint32), ("mlp", C.POINTER(MLP)), ("selector", C.POINTER(MLP)),
                ("edge_p", C.c_double), ("samplers", C.c_uint32), ("bytes_sample", C.c_uint32),
                ("mlp_tensor", C.c_uint32), ("pad_", C.c_uint32)]


class HybridInfo(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("n_s", "t_lo", "t_hi", "t_gs", "t_pre", "t_search", "c_step",
                                           "triangles")] + \
               [("features", C.c_float * 3), ("cost_model_gs", C.c_int32), ("selector_gs", C.c_int32)]

    def as_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_ if name != "features"}
        d["features"] = list(self.features)
        return d


class ProfileInfo(C.Structure):
    _fields_ = [("n_s", C.c_double), ("seconds", C.c_double), ("n_o", C.c_double), ("eps_o", C.c_double),
                ("rho_g", C.c_double), ("rho_gp", C.c_double), ("samples_used", C.c_uint64),
                ("kind", C.c_int32), ("pad_", C.c_int32)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "pad_"}


class Result(C.Structure):
    _fields_ = [("estimate", C.c_double), ("ci_half_width", C.c_double), ("eps_hat", C.c_double),
                ("sum", C.c_double), ("sumsq", C.c_double), ("samples", C.c_uint64),
                ("hits", C.c_uint64), ("rounds", C.c_uint64), ("scheme_used", C.c_int32),
                ("converged", C.c_int32), ("t_total_s", C.c_double), ("t_pilot_s", C.c_double),
                ("t_preproc_s", C.c_double), ("t_sample_s", C.c_double), ("exact_count", C.c_uint64),
                ("kernel_launches", C.c_uint64), ("algo_bytes_per_sample", C.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class SampleRecord(C.Structure):
    _fields_ = [("factor", C.c_uint64 * MAX_K), ("w_u64", C.c_uint64), ("w_f64", C.c_double),
                ("vert", C.c_uint32 * MAX_K), ("aux", C.c_uint32 * MAX_K), ("hit", C.c_uint8),
                ("depth", C.c_uint8), ("overflow", C.c_uint8), ("pad", C.c_uint8), ("sectors", C.c_uint32)]


class Sums(C.Structure):
    _fields_ = [("n", C.c_uint64), ("hits", C.c_uint64), ("sum", C.c_double), ("sumsq", C.c_double)]


class Partial(C.Structure):
    _fields_ = [("sum", C.c_double), ("sumsq", C.c_double), ("hits", C.c_uint64), ("n", C.c_uint64)]


class Window(C.Structure):
    _fields_ = [("sum", C.c_double), ("sumsq", C.c_double), ("hits", C.c_uint64), ("n", C.c_uint64),
                ("rounds", C.c_uint64), ("mu", C.c_double), ("half", C.c_double), ("eps_hat", C.c_double),
                ("converged", C.c_uint32), ("active", C.c_uint32)]


# (name, restype, argtypes): every exported entry point of include/gpm.h
P = C.POINTER
_V = C.c_void_p
_u64, _u32, _i32, _dbl = C.c_uint64, C.c_uint32, C.c_int32, C.c_double
# int gather(void *ctx, const void *send, void *recv, size_t bytes)
ALLGATHER_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t)

SIGNATURES = [
    ("gpm_load_csr", _i32, [_u64, _V, _V, _u32, _V, P(_V)]),
    ("gpm_free_graph", None, [_V]),
    ("gpm_graph_info", _i32, [_V, P(_u64), P(_u64), P(_u64), P(_u64)]),
    ("gpm_relabel_map", _i32, [_V, _V]),
    ("gpm_estimate", _i32, [_V, P(Pattern), _i32, _dbl, _dbl, _u64, P(Config), P(Result)]),
    ("gpm_estimate_batch", _i32, [_V, _u32, P(Pattern), P(_dbl), _dbl, _u64, P(Config), P(Result)]),
    ("gpm_autotune", _i32, [_V, _u32, P(Pattern), _u64, P(Config)]),
    ("gpm_hybrid_model", _i32, [_V, P(Pattern), _dbl, _dbl, _u64, P(Config), P(HybridInfo)]),
    ("gpm_profile", _i32, [_V, P(Pattern), _i32, _dbl, _dbl, _dbl, _u64, P(Config), P(ProfileInfo)]),
    ("gpm_mlp_train", _i32, [_V, _V, _V, _u64, _u32, _u32, C.c_float, _V, _V, P(_dbl)]),
    ("gpm_sample_sums", _i32, [_V, P(Pattern), _u64, _u64, _u64, P(Config), P(Sums)]),
    ("gpm_sample_sums_static", _i32, [_V, P(Pattern), _u64, _u64, _u64, P(Config), P(Sums)]),
    ("gpm_sample_partials", _i32, [_V, P(Pattern), _u64, _u64, _u64, _u32, _u32, P(Config), _V, P(_u64)]),
    ("gpm_merge_partials", _i32, [_V, _u64, P(Sums)]),
    ("gpm_window_update", _i32, [P(Window), P(Sums), _dbl, _dbl, _u64, _u64]),
    ("gpm_sample_runs", _i32, [_V, P(Pattern), _u64, _u64, _u64, _u32, _u32, P(Config), _V]),
    ("gpm_merge_runs", _i32, [_V, P(Sums)]),
    ("gpm_estimate_sharded", _i32, [_V, P(Pattern), _dbl, _dbl, _u64, _u32, _u32, P(Config), _V, _V,
                                    P(Window), _u64, P(Result)]),
    ("gpm_trace", _i32, [_V, P(Pattern), _u64, _u64, _u64, P(Config), _V]),
    ("gpm_exact_count", _i32, [_V, P(Pattern), P(_u64)]),
    ("gpm_mlp_scores", _i32, [_V, P(MLP), _V, _u64, _V]),
    ("gpm_mlp_scores_tc", _i32, [_V, P(MLP), _V, _u64, _V]),
    ("gpm_mlp_loss_grad", _i32, [_V, _V, _V, _V, _u64, _V, P(_dbl)]),
    ("gpm_proposal_features", _i32, [_V, P(Pattern), _V, _u64, _V, _V, P(_u64)]),
    ("gpm_train_proposal", _i32, [_V, P(Pattern), _u64, _u64, _u32, _u32, C.c_float, _V, _V, P(_dbl), P(_u64)]),
    ("gpm_sparsify", _i32, [_V, _u32, _u64, _u32, _u32, _V, _V, P(_u64)]),
    ("gpm_sparsify_edges", _i32, [_V, _dbl, _u64, _u32, _u32, _V, _V, P(_u64)]),
    ("gpm_gs_count_classes", _i32, [_V, P(Pattern), _u32, _u64, _u32, _u32, _u32, _u32, _dbl, P(_u64)]),
    ("gpm_abort", _i32, [_V]),
    ("gpm_gather_probe", _i32, [_u64, _u32, _u64, P(_dbl)]),
    ("gpm_plan", _i32, [P(Pattern), P(_i32), P(_i32), P(_i32), P(_i32), P(_i32)]),
    ("gpm_normal_quantile", _dbl, [_dbl]),
    ("gpm_last_error", C.c_char_p, []),
    ("gpm_version", C.c_char_p, []),
]

_lib = None


def load():
    """Load libgpm.so (built by ``build.py``); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libgpm.so is not built: run python -c 'import __graft_entry__ as g; g.build()'")
        L = C.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        assert C.sizeof(SampleRecord) == 216
        _lib = L
    return _lib


class GpmError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = load().gpm_last_error().decode(errors="replace")
        super().__init__("%s failed: %s (%s)" % (where, STATUS_NAMES.get(code, code), msg))


def check(code, where, ok=(GPM_OK,)):
    if code not in ok:
        raise GpmError(code, where)
    return code


def make_pattern(k, edges, induced=False):
    p = Pattern()
    p.k = k
    p.induced = 1 if induced else 0
    for a, b in edges:
        p.adj[a] |= 1 << b
        p.adj[b] |= 1 << a
    return p
