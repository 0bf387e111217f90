"""ctypes binding of the plain C oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product package.  It shares no code
with the CUDA path.  ``build()`` compiles ``oracle.c`` with gcc; nothing here
touches a GPU.
"""
import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")
MAXK = 12
MAXRES = 66

INTERSECT, CHECK, LEARNED, LAZY = 0, 1, 2, 3


class Plan(C.Structure):
    _fields_ = [("k", C.c_int32), ("induced", C.c_int32), ("oriented", C.c_int32),
                ("nres", C.c_int32), ("order", C.c_int32 * MAXK), ("adj", C.c_uint32 * MAXK),
                ("res_lo", C.c_int32 * MAXRES), ("res_hi", C.c_int32 * MAXRES),
                ("aut_size", C.c_int64)]

    def restrictions(self):
        return [(self.res_lo[i], self.res_hi[i]) for i in range(self.nres)]


class Record(C.Structure):
    _fields_ = [("factor", C.c_uint64 * MAXK), ("w_u64", C.c_uint64), ("w_f64", C.c_double),
                ("vert", C.c_uint32 * MAXK), ("aux", C.c_uint32 * MAXK),
                ("hit", C.c_uint8), ("depth", C.c_uint8), ("overflow", C.c_uint8),
                ("pad", C.c_uint8 * 5)]


class Sums(C.Structure):
    _fields_ = [("n", C.c_uint64), ("hits", C.c_uint64), ("sum", C.c_double),
                ("sumsq", C.c_double), ("bytes", C.c_double)]


class Online(C.Structure):
    _fields_ = [("estimate", C.c_double), ("ci_half_width", C.c_double), ("eps_hat", C.c_double),
                ("sum", C.c_double), ("sumsq", C.c_double), ("samples", C.c_uint64),
                ("hits", C.c_uint64), ("rounds", C.c_uint64), ("converged", C.c_int32),
                ("pad", C.c_int32)]


class MLP16(C.Structure):
    _fields_ = [(n, C.POINTER(C.c_uint16)) for n in ("w1", "b1", "w2", "b2", "w3", "b3")]


class MLP32(C.Structure):
    _fields_ = [("w1", C.c_float * 192), ("b1", C.c_float * 64), ("w2", C.c_float * 4096),
                ("b2", C.c_float * 64), ("w3", C.c_float * 64), ("b3", C.c_float * 1)]


# the numpy dtype mirror of Record, for bulk traces
RECORD_DTYPE = np.dtype([("factor", np.uint64, MAXK), ("w_u64", np.uint64), ("w_f64", np.float64),
                         ("vert", np.uint32, MAXK), ("aux", np.uint32, MAXK), ("hit", np.uint8),
                         ("depth", np.uint8), ("overflow", np.uint8), ("pad", np.uint8, 5)])

_lock = threading.Lock()
_lib = None


# OG_SANITIZE=1 builds and loads a separate copy instrumented with gcc's
# AddressSanitizer and UndefinedBehaviorSanitizer (errors abort the process;
# run under LD_PRELOAD=$(gcc -print-file-name=libasan.so) ASAN_OPTIONS=detect_leaks=0)
SANITIZE = os.environ.get("OG_SANITIZE") == "1"
if SANITIZE:
    LIB = LIB.replace("liboracle.so", "liboracle_san.so")


def build(force=False):
    """Compile oracle.c into liboracle.so (gcc, no fast-math, no FMA contraction)."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    san = ["-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer"] \
        if SANITIZE else []
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
                           "-fno-fast-math"] + san + ["-o", tmp, SRC, "-lm"])
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            P = C.POINTER
            u64, u32, i32, dbl = C.c_uint64, C.c_uint32, C.c_int, C.c_double
            L.og_philox4x32_10.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
            L.og_choice_word.restype = u64
            L.og_choice_word.argtypes = [u64, u64, u32, u32, u32]
            L.og_index_map.restype = u64
            L.og_index_map.argtypes = [u64, u64]
            L.og_validate.restype = i32
            L.og_validate.argtypes = [u64, C.c_void_p, C.c_void_p]
            L.og_graph_new.restype = C.c_void_p
            L.og_graph_new.argtypes = [u64, C.c_void_p, C.c_void_p]
            L.og_graph_free.argtypes = [C.c_void_p]
            L.og_graph_m.restype = u64
            L.og_graph_m.argtypes = [C.c_void_p]
            L.og_plan_build.restype = i32
            L.og_plan_build.argtypes = [i32, P(C.c_uint32), i32, P(Plan)]
            L.og_sample.restype = i32
            L.og_sample.argtypes = [C.c_void_p, P(Plan), P(C.c_uint64), i32, P(MLP16),
                                    C.c_void_p, C.c_void_p, P(Record)]
            L.og_sample_bytes.restype = dbl
            L.og_sample_bytes.argtypes = [C.c_void_p, P(Plan), i32, P(Record)]
            L.og_ns_run.restype = i32
            L.og_ns_run.argtypes = [C.c_void_p, P(Plan), i32, P(MLP16), u64, u32, u64, u64,
                                    P(Sums), C.c_void_p, i32]
            L.og_welford_run.restype = i32
            L.og_welford_run.argtypes = [C.c_void_p, P(Plan), i32, P(MLP16), u64, u32, u64, u64, P(dbl), P(dbl)]
            L.og_ns_bytes.restype = i32
            L.og_ns_bytes.argtypes = [C.c_void_p, P(Plan), i32, P(MLP16), u64, u32, u64, u64, C.c_void_p]
            L.og_phi_inv.restype = dbl
            L.og_phi_inv.argtypes = [dbl]
            L.og_error_of.argtypes = [dbl, dbl, u64, dbl, P(dbl), P(dbl), P(dbl)]
            L.og_ns_online.restype = i32
            L.og_ns_online.argtypes = [C.c_void_p, P(Plan), i32, P(MLP16), dbl, dbl, u64, u32,
                                       u64, u64, u64, P(Online)]
            L.og_color.restype = u32
            L.og_color.argtypes = [u64, u64, u32, u32, u32]
            L.og_sparsify.restype = u64
            L.og_sparsify.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            L.og_bes_threshold.restype = u64
            L.og_bes_threshold.argtypes = [dbl]
            L.og_bes_keep.restype = i32
            L.og_bes_keep.argtypes = [u64, u32, u32, u32, u32, u64]
            L.og_bes_sparsify.restype = u64
            L.og_bes_sparsify.argtypes = [C.c_void_p, u64, u32, u32, u64, C.c_void_p, C.c_void_p]
            L.og_exact_count.restype = u64
            L.og_exact_count.argtypes = [C.c_void_p, P(Plan)]
            L.og_flog2p1.restype = C.c_float
            L.og_flog2p1.argtypes = [u64]
            L.og_mlp_logit.restype = C.c_float
            L.og_mlp_logit.argtypes = [P(MLP16), P(C.c_float)]
            L.og_score.restype = u32
            L.og_score.argtypes = [C.c_float]
            L.og_mlp_loss_grad.restype = dbl
            L.og_mlp_loss_grad.argtypes = [P(MLP32), C.c_void_p, C.c_void_p, u64, P(MLP32)]
            for name in ("og_sizeof_plan", "og_sizeof_record", "og_sizeof_online", "og_sizeof_sums"):
                getattr(L, name).restype = u64
            assert L.og_sizeof_plan() == C.sizeof(Plan)
            assert L.og_sizeof_record() == C.sizeof(Record) == RECORD_DTYPE.itemsize
            assert L.og_sizeof_online() == C.sizeof(Online)
            assert L.og_sizeof_sums() == C.sizeof(Sums)
            _lib = L
    return _lib


# --------------------------------------------------------------------------
def philox(ctr, key):
    L = lib()
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    L.og_philox4x32_10(c, k, o)
    return tuple(o)


def choice_word(seed, s, t, slot=0, purpose=0):
    return lib().og_choice_word(seed, s, slot, purpose, t)


def index_map(r, n):
    return lib().og_index_map(r, n)


def phi_inv(p):
    return lib().og_phi_inv(p)


def error_of(total, total_sq, n, z):
    mu, half, eh = C.c_double(), C.c_double(), C.c_double()
    lib().og_error_of(total, total_sq, n, z, C.byref(mu), C.byref(half), C.byref(eh))
    return mu.value, half.value, eh.value


def validate(row_ptr, col):
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.uint64)
    col = np.ascontiguousarray(col, dtype=np.uint32)
    return lib().og_validate(len(row_ptr) - 1, row_ptr.ctypes.data, col.ctypes.data)


class Graph:
    """Oracle view of a host CSR (keeps the numpy arrays alive)."""

    def __init__(self, row_ptr, col):
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.uint64)
        self.col = np.ascontiguousarray(col, dtype=np.uint32)
        self.n = len(self.row_ptr) - 1
        self.h = lib().og_graph_new(self.n, self.row_ptr.ctypes.data, self.col.ctypes.data)
        self.m = lib().og_graph_m(self.h)
        self.nnz = int(self.row_ptr[-1])

    def __del__(self):
        try:
            if self.h:
                lib().og_graph_free(self.h)
                self.h = None
        except Exception:
            pass

    @property
    def max_degree(self):
        return int(np.max(np.diff(self.row_ptr))) if self.n else 0


def pattern_adj(k, edges):
    adj = [0] * MAXK
    for a, b in edges:
        adj[a] |= 1 << b
        adj[b] |= 1 << a
    return adj


def plan(k, edges, induced=False):
    p = Plan()
    adj = (C.c_uint32 * MAXK)(*pattern_adj(k, edges))
    rc = lib().og_plan_build(k, adj, 1 if induced else 0, C.byref(p))
    if rc != 0:
        raise ValueError("pattern rejected by the plan builder (code %d)" % rc)
    return p


class Weights16:
    """BF16 MLP weights as uint16 arrays, with the ctypes view the oracle reads."""

    def __init__(self, w1, b1, w2, b2, w3, b3):
        self.arrs = [np.ascontiguousarray(a, dtype=np.uint16).ravel() for a in (w1, b1, w2, b2, w3, b3)]
        ptrs = [a.ctypes.data_as(C.POINTER(C.c_uint16)) for a in self.arrs]
        self.c = MLP16(*ptrs)


def sample(g, p, r, mode=INTERSECT, mlp=None):
    """One sample from explicit choice words r[0..k-2]."""
    L = lib()
    rr = (C.c_uint64 * MAXK)(*([int(x) for x in r] + [0] * (MAXK - len(r))))
    md = (g.max_degree + 1) * MAXK      # an NS-base union spans up to k - 1 lists
    buf = np.zeros(md, dtype=np.uint32)
    buf2 = np.zeros(md, dtype=np.uint32)
    rec = Record()
    L.og_sample(g.h, C.byref(p), rr, mode, C.byref(mlp.c) if mlp else None,
                buf.ctypes.data, buf2.ctypes.data, C.byref(rec))
    return rec


def sample_bytes(g, p, rec, mode=INTERSECT):
    return lib().og_sample_bytes(g.h, C.byref(p), mode, C.byref(rec))


def ns_run(g, p, seed, first, count, mode=INTERSECT, mlp=None, slot=0, trace=False, want_bytes=False):
    """Samples [first, first+count): returns (Sums, records or None)."""
    acc = Sums()
    recs = np.zeros(count, dtype=RECORD_DTYPE) if trace else None
    rc = lib().og_ns_run(g.h, C.byref(p), mode, C.byref(mlp.c) if mlp else None, seed, slot,
                         first, count, C.byref(acc), recs.ctypes.data if trace else None,
                         1 if want_bytes else 0)
    if rc != 0:
        raise MemoryError("oracle run failed")
    return acc, recs


def welford(g, p, seed, first, count, mode=INTERSECT, mlp=None, slot=0):
    """(mean, M2) of samples [first, first+count) by Welford's update."""
    mu, m2 = C.c_double(), C.c_double()
    rc = lib().og_welford_run(g.h, C.byref(p), mode, C.byref(mlp.c) if mlp else None, seed, slot, first, count,
                              C.byref(mu), C.byref(m2))
    if rc != 0:
        raise MemoryError("oracle run failed")
    return mu.value, m2.value


def ns_bytes(g, p, seed, first, count, mode=INTERSECT, mlp=None, slot=0):
    """Algorithmic bytes of each sample of [first, first+count) (float64 array)."""
    out = np.zeros(count, dtype=np.float64)
    rc = lib().og_ns_bytes(g.h, C.byref(p), mode, C.byref(mlp.c) if mlp else None, seed, slot, first, count,
                           out.ctypes.data)
    if rc != 0:
        raise MemoryError("oracle run failed")
    return out


def ns_online(g, p, eps, delta, seed, window, n_min=None, n_max=10**9, mode=INTERSECT, mlp=None, slot=0):
    out = Online()
    rc = lib().og_ns_online(g.h, C.byref(p), mode, C.byref(mlp.c) if mlp else None, eps, delta, seed,
                            slot, window, n_min if n_min is not None else window, n_max, C.byref(out))
    if rc != 0:
        raise MemoryError("oracle run failed")
    return out


def colors(n, c, seed, colouring=0, slot=0):
    L = lib()
    return np.array([L.og_color(seed, v, colouring, slot, c) for v in range(n)], dtype=np.uint32)


def sparsify(g, cols):
    cols = np.ascontiguousarray(cols, dtype=np.uint32)
    row = np.zeros(g.n + 1, dtype=np.uint64)
    col = np.zeros(max(g.nnz, 1), dtype=np.uint32)
    kept = lib().og_sparsify(g.h, cols.ctypes.data, row.ctypes.data, col.ctypes.data)
    return row, col[:kept].copy()


def bes_threshold(p):
    """t with keep probability t / 2^32 (Algorithm 2's p)."""
    return lib().og_bes_threshold(p)


def bes_keep(seed, u, w, t, colouring=0, slot=0):
    return bool(lib().og_bes_keep(seed, u, w, colouring, slot, t))


def bes_sparsify(g, seed, t, colouring=0, slot=0):
    """Bernoulli edge sparsification (Algorithm 2): the kept CSR."""
    row = np.zeros(g.n + 1, dtype=np.uint64)
    col = np.zeros(max(g.nnz, 1), dtype=np.uint32)
    kept = lib().og_bes_sparsify(g.h, seed, colouring, slot, t, row.ctypes.data, col.ctypes.data)
    return row, col[:kept].copy()


def exact_count(g, p):
    return lib().og_exact_count(g.h, C.byref(p))


def gs_estimate(g, p, c, seed, colouring=0, slot=0):
    """Colour sparsification estimate C' * c^(k-1) and the exact count C'."""
    cols = colors(g.n, c, seed, colouring, slot)
    row, col = sparsify(g, cols)
    gp = Graph(row, col)
    cp = exact_count(gp, p)
    return float(cp) * float(c) ** (p.k - 1), cp


def flog2p1(d):
    return lib().og_flog2p1(d)


def mlp_logit(mlp, f):
    arr = (C.c_float * 3)(*f)
    return lib().og_mlp_logit(C.byref(mlp.c), arr)


def score(z):
    return lib().og_score(z)


def mlp_loss_grad(w32, feat, label):
    """w32: dict of float32 arrays (w1 [64,3], b1, w2 [64,64], b2, w3 [64], b3 [1])."""
    W = MLP32()
    for name in ("w1", "b1", "w2", "b2", "w3", "b3"):
        a = np.ascontiguousarray(w32[name], dtype=np.float32).ravel()
        C.memmove(getattr(W, name), a.ctypes.data, a.nbytes)
    G = MLP32()
    feat = np.ascontiguousarray(feat, dtype=np.float32)
    label = np.ascontiguousarray(label, dtype=np.float32)
    loss = lib().og_mlp_loss_grad(C.byref(W), feat.ctypes.data, label.ctypes.data, len(label), C.byref(G))
    grads = {}
    for name, shape in (("w1", (64, 3)), ("b1", (64,)), ("w2", (64, 64)), ("b2", (64,)),
                        ("w3", (64,)), ("b3", (1,))):
        grads[name] = np.frombuffer(getattr(G, name), dtype=np.float32).reshape(shape).copy()
    return loss, grads
