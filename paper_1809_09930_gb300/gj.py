"""Python binding of the C ABI in include/gj.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of the join: points go in as numpy arrays or torch tensors (host or
CUDA), pairs come back in caller-provided or freshly allocated buffers.  The
library must have been built (``__graft_entry__.build()`` or
``python -m paper_1809_09930_gb300._build``); importing this module without it
raises, there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgj.so")

GJ_OK = 0
GJ_ERR_INVALID_ARG = -1
GJ_ERR_NONFINITE = -2
GJ_ERR_OOM = -3
GJ_ERR_CUDA = -4
GJ_ERR_CAPACITY = -5
GJ_ERR_TIMEOUT = -6
GJ_ERR_UNSUPPORTED = -7
GJ_ERR_TOO_LARGE = -8
GJ_MAX_DIMS = 1024

GJ_REORDER = 1 << 0
GJ_SORTIDU = 1 << 1
GJ_SHORTC = 1 << 2
GJ_TC_FILTER = 1 << 3
GJ_AUTOTUNE = 1 << 4
GJ_TUNE_FORM = 1 << 5
GJ_HOST_BATCHED = 1 << 6
GJ_DEFAULT_FLAGS = GJ_REORDER | GJ_SORTIDU | GJ_SHORTC


class GJError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {gj_status_string(status)} ({status})" if what else gj_status_string(status))


class gj_config(C.Structure):
    _fields_ = [("k", C.c_int32), ("flags", C.c_uint32), ("stream", C.c_void_p),
                ("batch_pairs", C.c_uint64), ("device", C.c_int32), ("query_block", C.c_int32),
                ("tile", C.c_int32), ("reserved", C.c_uint32 * 5)]


class gj_tune_result(C.Structure):
    _fields_ = [("k", C.c_int32), ("flags", C.c_uint32), ("query_block", C.c_int32), ("tile", C.c_int32),
                ("batch_pairs", C.c_uint64), ("est_pairs", C.c_uint64), ("build_ms", C.c_double),
                ("join_ms", C.c_double), ("trials", C.c_int32), ("reserved", C.c_int32)]


class gj_job(C.Structure):
    _fields_ = [("points", C.c_void_p), ("n", C.c_int64), ("d", C.c_int32), ("k", C.c_int32),
                ("eps", C.c_double)]


class gj_index_info_t(C.Structure):
    _fields_ = [("n", C.c_int64), ("d", C.c_int32), ("k", C.c_int32), ("eps", C.c_double),
                ("nonempty_cells", C.c_int64), ("work_items", C.c_int64),
                ("candidate_pairs", C.c_uint64), ("window_pairs", C.c_uint64),
                ("flags", C.c_uint32), ("sortidu_dim", C.c_int32),
                ("perm", C.c_int32 * GJ_MAX_DIMS)]


class gj_join_stats(C.Structure):
    _fields_ = [("pairs", C.c_uint64), ("launches", C.c_uint32), ("batches_planned", C.c_uint32),
                ("batch_pairs", C.c_uint64), ("estimate", C.c_uint64), ("tc_survivors", C.c_uint64),
                ("evaluated", C.c_uint64), ("dims", C.c_uint64), ("join_ms", C.c_double),
                ("estimate_ms", C.c_double), ("total_ms", C.c_double), ("busy_ms", C.c_double),
                ("candidates", C.c_uint64)]


EXPORTS = ["gj_config_init", "gj_index_build", "gj_index_build_ex", "gj_self_join",
           "gj_self_join_part", "gj_index_get_info", "gj_last_join_stats", "gj_free",
           "gj_last_status", "gj_status_string", "gj_version", "gj_probe_fp64_tflops",
           "gj_kernel_launches", "gj_debug_tc_tile", "gj_self_join_noalloc", "gj_batch_build",
           "gj_batch_self_join", "gj_batch_get_info", "gj_batch_free", "gj_autotune", "gj_batch_get_k",
           "gj_neighbor_table", "gj_join_qe", "gj_tc_threshold", "gj_debug_set_wait_limit"]

_lib = None


def load(path: str | None = None):
    """Load libgj.so and declare the C signatures."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"the CUDA library {p} is not built; run __graft_entry__.build()")
    lib = C.CDLL(p)
    V = C.c_void_p
    lib.gj_config_init.restype = None
    lib.gj_config_init.argtypes = [C.POINTER(gj_config)]
    lib.gj_index_build.restype = V
    lib.gj_index_build.argtypes = [V, C.c_int64, C.c_int32, C.c_double, C.c_int32]
    lib.gj_index_build_ex.restype = V
    lib.gj_index_build_ex.argtypes = [V, C.c_int64, C.c_int32, C.c_double, C.POINTER(gj_config)]
    lib.gj_self_join.restype = C.c_int
    lib.gj_self_join.argtypes = [V, V, C.c_uint64, C.POINTER(C.c_uint64)]
    lib.gj_self_join_part.restype = C.c_int
    lib.gj_self_join_part.argtypes = [V, C.c_int32, C.c_int32, V, C.c_uint64, C.POINTER(C.c_uint64)]
    lib.gj_index_get_info.restype = C.c_int
    lib.gj_index_get_info.argtypes = [V, C.POINTER(gj_index_info_t)]
    lib.gj_last_join_stats.restype = C.c_int
    lib.gj_last_join_stats.argtypes = [V, C.POINTER(gj_join_stats)]
    lib.gj_free.restype = None
    lib.gj_free.argtypes = [V]
    lib.gj_last_status.restype = C.c_int
    lib.gj_last_status.argtypes = []
    lib.gj_status_string.restype = C.c_char_p
    lib.gj_status_string.argtypes = [C.c_int]
    lib.gj_version.restype = C.c_char_p
    lib.gj_version.argtypes = []
    lib.gj_probe_fp64_tflops.restype = C.c_int
    lib.gj_probe_fp64_tflops.argtypes = [C.c_int32, C.POINTER(C.c_double)]
    lib.gj_kernel_launches.restype = C.c_ulonglong
    lib.gj_kernel_launches.argtypes = []
    lib.gj_debug_tc_tile.restype = C.c_int
    lib.gj_debug_tc_tile.argtypes = [V, V, C.c_int32, V]
    lib.gj_debug_set_wait_limit.restype = C.c_int
    lib.gj_debug_set_wait_limit.argtypes = [C.c_uint64]
    lib.gj_tc_threshold.restype = C.c_int
    lib.gj_tc_threshold.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int32, C.POINTER(C.c_float)]
    lib.gj_self_join_noalloc.restype = C.c_int
    lib.gj_batch_build.restype = V
    lib.gj_batch_build.argtypes = [C.POINTER(gj_job), C.c_int32, C.POINTER(gj_config)]
    lib.gj_batch_self_join.restype = C.c_int
    lib.gj_batch_self_join.argtypes = [V, V, V, V]
    lib.gj_batch_get_info.restype = C.c_int
    lib.gj_batch_get_info.argtypes = [V, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_uint64)]
    lib.gj_batch_free.restype = None
    lib.gj_batch_free.argtypes = [V]
    lib.gj_self_join_noalloc.argtypes = [V, C.c_int32, C.c_int32, V, C.c_uint64, C.POINTER(C.c_uint64)]
    lib.gj_autotune.restype = C.c_int
    lib.gj_autotune.argtypes = [V, C.c_int64, C.c_int32, C.c_double, C.POINTER(gj_config),
                                C.POINTER(gj_tune_result)]
    lib.gj_join_qe.restype = C.c_int
    lib.gj_join_qe.argtypes = [V, V, C.c_int64, V, C.c_uint64, C.POINTER(C.c_uint64)]
    lib.gj_neighbor_table.restype = C.c_int
    lib.gj_neighbor_table.argtypes = [V, V, V, C.c_uint64, C.POINTER(C.c_uint64)]
    lib.gj_batch_get_k.restype = C.c_int
    lib.gj_batch_get_k.argtypes = [V, C.POINTER(C.c_int32)]
    if path is None:
        _lib = lib
    return lib


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def _ptr_points(points):
    """(pointer, n, d, keepalive) for an (n, d) float64 array or tensor."""
    try:
        import torch
        if isinstance(points, torch.Tensor):
            if points.dtype != torch.float64 or points.dim() != 2:
                raise TypeError("points must be a 2-D float64 tensor")
            t = points.contiguous()
            return t.data_ptr(), t.shape[0], t.shape[1], t
    except ImportError:  # pragma: no cover
        pass
    a = np.ascontiguousarray(points, dtype=np.float64)
    if a.ndim != 2:
        raise TypeError("points must be a 2-D array")
    return a.ctypes.data, a.shape[0], a.shape[1], a


def _ptr_pairs(out):
    """(pointer, capacity in pairs, keepalive) for a (cap, 2) uint32 buffer."""
    if out is None:
        return None, 0, None
    try:
        import torch
        if isinstance(out, torch.Tensor):
            if out.dtype not in (torch.int32, torch.uint32) or out.dim() != 2 or out.shape[1] != 2 \
                    or not out.is_contiguous():
                raise TypeError("pair buffer must be a contiguous (cap, 2) int32/uint32 tensor")
            return out.data_ptr(), out.shape[0], out
    except ImportError:  # pragma: no cover
        pass
    if not (isinstance(out, np.ndarray) and out.dtype == np.uint32 and out.ndim == 2
            and out.shape[1] == 2 and out.flags.c_contiguous):
        raise TypeError("pair buffer must be a C-contiguous (cap, 2) uint32 array")
    return out.ctypes.data, out.shape[0], out


# ---------------------------------------------------------------------------
# the C entry points, by name
# ---------------------------------------------------------------------------

def gj_config_init() -> gj_config:
    cfg = gj_config()
    load().gj_config_init(C.byref(cfg))
    return cfg


def gj_index_build(points, eps: float, k: int = 0) -> int:
    p, n, d, keep = _ptr_points(points)
    h = load().gj_index_build(p, n, d, float(eps), int(k))
    del keep
    if not h:
        raise GJError(gj_last_status(), "gj_index_build")
    return h


def gj_index_build_ex(points, eps: float, cfg: gj_config) -> int:
    p, n, d, keep = _ptr_points(points)
    h = load().gj_index_build_ex(p, n, d, float(eps), C.byref(cfg))
    del keep
    if not h:
        raise GJError(gj_last_status(), "gj_index_build_ex")
    return h


def gj_autotune(points, eps: float, cfg: gj_config | None = None) -> dict:
    """The autotuner's pick for these points (timed trials on the device)."""
    p, n, d, keep = _ptr_points(points)
    cfg = cfg if cfg is not None else gj_config_init()
    r = gj_tune_result()
    st = load().gj_autotune(p, n, d, float(eps), C.byref(cfg), C.byref(r))
    del keep
    if st != GJ_OK:
        raise GJError(st, "gj_autotune")
    return {f: getattr(r, f) for f, _ in gj_tune_result._fields_ if f != "reserved"}


def gj_self_join(h: int, out=None) -> tuple[int, int]:
    """Returns (status, |R|); pairs land in ``out`` when it is large enough."""
    p, cap, keep = _ptr_pairs(out)
    cnt = C.c_uint64(0)
    st = load().gj_self_join(h, p, cap, C.byref(cnt))
    del keep
    return st, int(cnt.value)


def gj_self_join_part(h: int, part: int, nparts: int, out=None) -> tuple[int, int]:
    p, cap, keep = _ptr_pairs(out)
    cnt = C.c_uint64(0)
    st = load().gj_self_join_part(h, int(part), int(nparts), p, cap, C.byref(cnt))
    del keep
    return st, int(cnt.value)


def gj_join_qe(h: int, queries, out=None) -> tuple[int, int]:
    """Q join_eps E against the index h (over E); returns (status, count)."""
    q, nq, d, keepq = _ptr_points(queries)
    p, cap, keep = _ptr_pairs(out)
    cnt = C.c_uint64(0)
    st = load().gj_join_qe(h, q, nq, p, cap, C.byref(cnt))
    del keep, keepq
    return st, int(cnt.value)


def gj_neighbor_table(h: int, row_start, nbr) -> tuple[int, int]:
    """CSR neighbour table into CUDA tensors: row_start int64 (n+1,), nbr
    int32/uint32 (cap,).  Returns (status, |R|)."""
    cnt = C.c_uint64(0)
    st = load().gj_neighbor_table(h, row_start.data_ptr(), nbr.data_ptr() if nbr is not None else None,
                                  int(nbr.numel()) if nbr is not None else 0, C.byref(cnt))
    return st, int(cnt.value)


def gj_self_join_noalloc(h: int, out=None, part: int = 0, nparts: int = 1) -> tuple[int, int]:
    """The allocation-free join into a device buffer; returns (status, |R|)."""
    p, cap, keep = _ptr_pairs(out)
    cnt = C.c_uint64(0)
    st = load().gj_self_join_noalloc(h, int(part), int(nparts), p, cap, C.byref(cnt))
    del keep
    return st, int(cnt.value)


def gj_index_get_info(h: int) -> dict:
    info = gj_index_info_t()
    st = load().gj_index_get_info(h, C.byref(info))
    if st != GJ_OK:
        raise GJError(st, "gj_index_get_info")
    out = {f: getattr(info, f) for f, _ in gj_index_info_t._fields_ if f != "perm"}
    out["perm"] = [int(info.perm[j]) for j in range(info.d)]
    return out


def gj_last_join_stats(h: int) -> dict:
    st_ = gj_join_stats()
    st = load().gj_last_join_stats(h, C.byref(st_))
    if st != GJ_OK:
        raise GJError(st, "gj_last_join_stats")
    return {f: getattr(st_, f) for f, _ in gj_join_stats._fields_}


def gj_free(h: int) -> None:
    if h:
        load().gj_free(h)


def gj_last_status() -> int:
    return int(load().gj_last_status())


def gj_status_string(status: int) -> str:
    return load().gj_status_string(int(status)).decode()


def gj_version() -> str:
    return load().gj_version().decode()


def gj_probe_fp64_tflops(device: int = -1) -> float:
    v = C.c_double(0.0)
    st = load().gj_probe_fp64_tflops(int(device), C.byref(v))
    if st != GJ_OK:
        raise GJError(st, "gj_probe_fp64_tflops")
    return float(v.value)


def gj_debug_set_wait_limit(ns: int) -> int:
    """Limit of every bounded device wait of later tensor-core joins (0: default)."""
    return int(load().gj_debug_set_wait_limit(int(ns)))


def gj_kernel_launches() -> int:
    return int(load().gj_kernel_launches())


def gj_tc_threshold(eps: float, sigma: float, R0: float, d: int) -> tuple[int, float]:
    """(status, T): the fp32 survivor threshold of the tensor-core filter."""
    t = C.c_float(0.0)
    st = load().gj_tc_threshold(float(eps), float(sigma), float(R0), int(d), C.byref(t))
    return st, t.value


def gj_debug_tc_tile(A, B) -> np.ndarray:
    """D = A @ B.T on the tensor cores for (128, Kp) float16 arrays."""
    A = np.ascontiguousarray(A, dtype=np.float16)
    B = np.ascontiguousarray(B, dtype=np.float16)
    if A.shape != B.shape or A.shape[0] != 128:
        raise ValueError("A and B must both be (128, Kp) float16")
    D = np.empty((128, 128), dtype=np.float32)
    st = load().gj_debug_tc_tile(A.ctypes.data, B.ctypes.data, A.shape[1], D.ctypes.data)
    if st != GJ_OK:
        raise GJError(st, "gj_debug_tc_tile")
    return D


def gj_batch_build(jobs, cfg: gj_config | None = None) -> int:
    """jobs: list of (points, eps, k) with points as for gj_index_build."""
    arr = (gj_job * len(jobs))()
    keep = []
    for i, (pts, eps, k) in enumerate(jobs):
        p, n, d, kp = _ptr_points(pts)
        keep.append(kp)
        arr[i].points = p
        arr[i].n = n
        arr[i].d = d
        arr[i].k = int(k)
        arr[i].eps = float(eps)
    cfg = cfg if cfg is not None else gj_config_init()
    h = load().gj_batch_build(arr, len(jobs), C.byref(cfg))
    del keep
    if not h:
        raise GJError(gj_last_status(), "gj_batch_build")
    return h


def gj_batch_self_join(b: int, njobs: int, outs=None) -> tuple[int, list[int]]:
    """outs: None (count only) or a list of (cap, 2) int32 CUDA tensors / None."""
    counts = (C.c_uint64 * njobs)()
    if outs is None:
        st = load().gj_batch_self_join(b, None, None, counts)
    else:
        ptrs = (C.c_void_p * njobs)()
        caps = (C.c_uint64 * njobs)()
        for j, o in enumerate(outs):
            p, cap, _ = _ptr_pairs(o)
            ptrs[j] = p
            caps[j] = cap
        st = load().gj_batch_self_join(b, ptrs, caps, counts)
    return st, [int(c) for c in counts]


def gj_batch_get_info(b: int) -> dict:
    wi, tp, cp = C.c_int64(), C.c_int64(), C.c_uint64()
    st = load().gj_batch_get_info(b, C.byref(wi), C.byref(tp), C.byref(cp))
    if st != GJ_OK:
        raise GJError(st, "gj_batch_get_info")
    return {"work_items": wi.value, "total_points": tp.value, "candidate_pairs": cp.value}


def gj_batch_get_k(b: int, njobs: int) -> list[int]:
    ks = (C.c_int32 * njobs)()
    st = load().gj_batch_get_k(b, ks)
    if st != GJ_OK:
        raise GJError(st, "gj_batch_get_k")
    return [int(k) for k in ks]


def gj_batch_free(b: int) -> None:
    if b:
        load().gj_batch_free(b)


# ---------------------------------------------------------------------------
# convenience
# ---------------------------------------------------------------------------

class Index:
    """Owns a gj_index handle."""

    def __init__(self, points, eps: float, k: int = 0, flags: int = GJ_DEFAULT_FLAGS,
                 stream=None, batch_pairs: int = 0, device: int = -1, query_block: int = 0,
                 tile: int = 0):
        cfg = gj_config_init()
        cfg.k = int(k)
        cfg.flags = int(flags)
        cfg.stream = int(stream) if stream else None
        cfg.batch_pairs = int(batch_pairs)
        cfg.device = int(device)
        cfg.query_block = int(query_block)
        cfg.tile = int(tile)
        self.h = gj_index_build_ex(points, eps, cfg)
        self._sizes = {}   # |R| of (part, nparts) once known: R is fixed for an index

    def close(self):
        if self.h:
            gj_free(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def info(self) -> dict:
        return gj_index_get_info(self.h)

    def stats(self) -> dict:
        return gj_last_join_stats(self.h)

    def count(self) -> int:
        """|R| by a count-only join (remembered for join())."""
        st, n = gj_self_join(self.h, None)
        if st != GJ_OK:
            raise GJError(st, "gj_self_join (count)")
        self._sizes[(None, 1)] = n
        return n

    def join_qe(self, queries):
        """The pairs (query row, entry row) within eps as a (m, 2) uint32 array.
        Two launches: a count-only join sizes the array, then the join fills it
        (call gj_join_qe with a buffer of your own to join once)."""
        st, m = gj_join_qe(self.h, queries, None)
        if st != GJ_OK:
            raise GJError(st, "gj_join_qe (count)")
        out = np.empty((max(m, 1), 2), dtype=np.uint32)
        st, m2 = gj_join_qe(self.h, queries, out)
        if st != GJ_OK:
            raise GJError(st, "gj_join_qe")
        return out[:m2]

    def neighbor_table(self):
        """(row_start, nbr) as CUDA tensors (int64 (n+1,), int32 (|R|,))."""
        import torch
        n = self.info()["n"]
        m = self.count()
        row_start = torch.empty(n + 1, dtype=torch.int64, device="cuda")
        nbr = torch.empty(max(m, 1), dtype=torch.int32, device="cuda")
        st, c = gj_neighbor_table(self.h, row_start, nbr)
        if st != GJ_OK:
            raise GJError(st, "gj_neighbor_table")
        return row_start, nbr[:c]

    def join(self, out=None, part: int | None = None, nparts: int = 1):
        """Pairs as a (|R|, 2) uint32 numpy array (or the given buffer's prefix).
        Without a buffer the array is sized by |R|: known after count() or an
        earlier join of this index, else found by one count-only join first
        (then the call runs the join twice; pass ``out`` to join once)."""
        key = (part, nparts if part is not None else 1)
        if out is None:
            n = self._sizes.get(key)
            if n is None:
                n = self.count() if part is None else gj_self_join_part(self.h, part, nparts, None)[1]
            out = np.empty((max(n, 1), 2), dtype=np.uint32)
        if part is None:
            st, n = gj_self_join(self.h, out)
        else:
            st, n = gj_self_join_part(self.h, part, nparts, out)
        if st != GJ_OK:
            raise GJError(st, "gj_self_join")
        self._sizes[key] = n
        return out[:n]
