"""ctypes binding of libballmapper's C-ABI (``include/ballmapper.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Device inputs are torch CUDA tensors; the library's outputs and
scratch are allocated through a callback into torch's caching allocator, so
the returned device arrays are torch tensors that own their memory.  Host
inputs (numpy arrays or CPU tensors) select the library's host I/O mode.

There is no CPU fallback: if the library is not built, or no GB300 is
present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libballmapper.so")

BM_OK, BM_ERR_ARG, BM_ERR_CUDA, BM_ERR_NOMEM, BM_ERR_CAPACITY, BM_ERR_TIMEOUT, BM_ERR_UNSUPPORTED = range(7)
BM_PATH_TC_SPLIT3, BM_PATH_FP32, BM_PATH_TC_FP16, BM_PATH_TC_AUTO = 0, 1, 2, 3
PATHS = {"tc": BM_PATH_TC_SPLIT3, "fp32": BM_PATH_FP32, "tc16": BM_PATH_TC_FP16, "auto": BM_PATH_TC_AUTO}
BM_CENTRE_AUTO, BM_CENTRE_ALWAYS, BM_CENTRE_OFF = 0, 1, 2

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class bm_options(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_void_p), ("path", ctypes.c_int32), ("host_io", ctypes.c_int32),
                ("batch", ctypes.c_int32), ("skip_edges", ctypes.c_int32), ("alloc", ALLOC_FN),
                ("free", FREE_FN), ("alloc_ctx", ctypes.c_void_p), ("want_dists", ctypes.c_int32),
                ("centring", ctypes.c_int32)]


class bm_stats(ctypes.Structure):
    _fields_ = [("distance_evals", ctypes.c_int64), ("tile_pairs", ctypes.c_int64), ("band_pairs", ctypes.c_int64),
                ("greedy_steps", ctypes.c_int64), ("candidates", ctypes.c_int64), ("edge_pairs", ctypes.c_int64),
                ("ms_prep", ctypes.c_double), ("ms_greedy", ctypes.c_double), ("ms_members", ctypes.c_double),
                ("ms_edges", ctypes.c_double), ("ms_total", ctypes.c_double), ("band_delta", ctypes.c_float),
                ("path", ctypes.c_int32), ("ms_sweep", ctypes.c_double), ("sweep_launches", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("recheck_rate", ctypes.c_double),
                ("dist_max_rel_err", ctypes.c_double), ("truncated", ctypes.c_int32), ("centred", ctypes.c_int32)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class bm_csr(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("nnz", ctypes.c_int64), ("offsets", ctypes.c_void_p),
                ("ids", ctypes.c_void_p), ("on_host", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("dists", ctypes.c_void_p)]


class bm_graph(ctypes.Structure):
    _fields_ = [("n_landmarks", ctypes.c_int64), ("landmarks", ctypes.c_void_p), ("members", bm_csr),
                ("n_edges", ctypes.c_int64), ("edges", ctypes.c_void_p), ("on_host", ctypes.c_int32),
                ("reserved0", ctypes.c_int32), ("stats", bm_stats)]


class bm_instance(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("n", ctypes.c_int64), ("d", ctypes.c_int32), ("eps", ctypes.c_float),
                ("batch", ctypes.c_int32), ("reserved0", ctypes.c_int32)]


class bm_tile_config(ctypes.Structure):
    _fields_ = [("d_pad", ctypes.c_int32), ("ck", ctypes.c_int32), ("nt", ctypes.c_int32), ("bbuf", ctypes.c_int32),
                ("astg", ctypes.c_int32)]

    def as_dict(self):
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


class BallMapperError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


STATUS_NAMES = {BM_OK: "BM_OK", BM_ERR_ARG: "BM_ERR_ARG", BM_ERR_CUDA: "BM_ERR_CUDA", BM_ERR_NOMEM: "BM_ERR_NOMEM",
                BM_ERR_CAPACITY: "BM_ERR_CAPACITY", BM_ERR_TIMEOUT: "BM_ERR_TIMEOUT",
                BM_ERR_UNSUPPORTED: "BM_ERR_UNSUPPORTED"}

_lib = None
_lib_lock = threading.Lock()


def load(path: str = LIB_PATH):
    """Load libballmapper.so (raises if it has not been built)."""
    global _lib
    with _lib_lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError("libballmapper.so is not built (%s); run __graft_entry__.build()" % path)
        lib = ctypes.CDLL(path)
        lib.bm_options_init.argtypes = [ctypes.POINTER(bm_options)]
        lib.bm_options_init.restype = None
        lib.bm_range_query.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_int64, ctypes.c_float, ctypes.POINTER(bm_options),
                                       ctypes.POINTER(bm_csr), ctypes.POINTER(bm_stats)]
        lib.bm_range_query.restype = ctypes.c_int
        lib.bm_build.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_float,
                                 ctypes.POINTER(bm_options), ctypes.POINTER(bm_graph)]
        lib.bm_build.restype = ctypes.c_int
        lib.bm_csr_free.argtypes = [ctypes.POINTER(bm_csr), ctypes.POINTER(bm_options)]
        lib.bm_csr_free.restype = None
        lib.bm_graph_free.argtypes = [ctypes.POINTER(bm_graph), ctypes.POINTER(bm_options)]
        lib.bm_graph_free.restype = None
        lib.bm_status_string.argtypes = [ctypes.c_int]
        lib.bm_status_string.restype = ctypes.c_char_p
        lib.bm_last_error.argtypes = []
        lib.bm_last_error.restype = ctypes.c_char_p
        lib.bm_version.argtypes = []
        lib.bm_version.restype = ctypes.c_int32
        lib.bm_range_count_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                                               ctypes.c_int64, ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p]
        lib.bm_range_count_noalloc.restype = ctypes.c_int
        lib.bm_ivf_train.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_int64, ctypes.c_uint64, ctypes.POINTER(bm_options),
                                     ctypes.POINTER(ctypes.c_void_p)]
        lib.bm_ivf_train.restype = ctypes.c_int
        lib.bm_ivf_free.argtypes = [ctypes.c_void_p]
        lib.bm_ivf_free.restype = None
        lib.bm_ivf_info.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32),
                                    ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_void_p),
                                    ctypes.POINTER(ctypes.c_void_p)]
        lib.bm_ivf_info.restype = ctypes.c_int
        lib.bm_ivf_range_query.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_float,
                                           ctypes.c_int32, ctypes.POINTER(bm_options), ctypes.POINTER(bm_csr),
                                           ctypes.c_void_p, ctypes.POINTER(bm_stats)]
        lib.bm_ivf_range_query.restype = ctypes.c_int
        lib.bm_build_ivf.argtypes = [ctypes.c_void_p, ctypes.c_float, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64,
                                     ctypes.POINTER(bm_options), ctypes.POINTER(bm_graph)]
        lib.bm_build_ivf.restype = ctypes.c_int
        lib.bm_build_batched.argtypes = [ctypes.POINTER(bm_instance), ctypes.c_int32, ctypes.POINTER(bm_options),
                                         ctypes.POINTER(bm_graph), ctypes.POINTER(ctypes.c_int32)]
        lib.bm_build_batched.restype = ctypes.c_int
        lib.bm_tile_shapes.argtypes = [ctypes.POINTER(bm_tile_config), ctypes.c_int32]
        lib.bm_tile_shapes.restype = ctypes.c_int32
        lib.bm_get_tile_config.argtypes = [ctypes.c_int32, ctypes.POINTER(bm_tile_config)]
        lib.bm_get_tile_config.restype = ctypes.c_int
        lib.bm_set_tile_config.argtypes = [ctypes.c_int32, ctypes.POINTER(bm_tile_config)]
        lib.bm_set_tile_config.restype = ctypes.c_int
        lib.bm_build_fps.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_float, ctypes.c_int64,
                                     ctypes.POINTER(bm_options), ctypes.POINTER(bm_graph)]
        lib.bm_build_fps.restype = ctypes.c_int
        lib.bm_color.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                 ctypes.c_int32, ctypes.POINTER(bm_options), ctypes.c_void_p]
        lib.bm_color.restype = ctypes.c_int
        lib.bm_gidx_build.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.POINTER(bm_options), ctypes.POINTER(ctypes.c_void_p)]
        lib.bm_gidx_build.restype = ctypes.c_int
        lib.bm_gidx_free.argtypes = [ctypes.c_void_p]
        lib.bm_gidx_free.restype = None
        lib.bm_gidx_info.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32),
                                     ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_void_p),
                                     ctypes.POINTER(ctypes.c_void_p)]
        lib.bm_gidx_info.restype = ctypes.c_int
        lib.bm_gidx_range_query.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_float,
                                            ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(bm_options),
                                            ctypes.POINTER(bm_csr), ctypes.POINTER(bm_stats)]
        lib.bm_gidx_range_query.restype = ctypes.c_int
        lib.bm_build_gidx.argtypes = [ctypes.c_void_p, ctypes.c_float, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
                                      ctypes.c_int64, ctypes.POINTER(bm_options), ctypes.POINTER(bm_graph)]
        lib.bm_build_gidx.restype = ctypes.c_int
        lib.bm_knn_dist.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.POINTER(bm_options), ctypes.c_void_p, ctypes.POINTER(bm_stats)]
        lib.bm_knn_dist.restype = ctypes.c_int
        lib.bm_occupancy_eps.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.POINTER(bm_options), ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(bm_stats)]
        lib.bm_occupancy_eps.restype = ctypes.c_int
        lib.bm_set_nerve_bitmap_bytes.argtypes = [ctypes.c_int64]
        lib.bm_set_nerve_bitmap_bytes.restype = ctypes.c_int64
        lib.bm_band_halfwidth.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_double]
        lib.bm_band_halfwidth.restype = ctypes.c_double
        _lib = lib
        return lib


def _check(lib, status):
    if status != BM_OK:
        raise BallMapperError(status, lib.bm_last_error().decode(errors="replace"))


class _TorchAllocator:
    """Routes the library's device allocations to torch's caching allocator."""

    def __init__(self, device):
        import torch
        self._torch = torch
        self._device = device
        self.live = {}
        self.failed = False

        def _alloc(nbytes, stream, ctx):
            try:
                t = torch.empty(int(nbytes), dtype=torch.uint8, device=self._device)
            except Exception:
                self.failed = True
                return None
            p = t.data_ptr()
            self.live[p] = t
            return p

        def _free(ptr, stream, ctx):
            self.live.pop(ptr, None)

        self.alloc_cb = ALLOC_FN(_alloc)
        self.free_cb = FREE_FN(_free)

    def peek(self, ptr, count, dtype):
        """A view of a buffer the library still owns (e.g. an index's arrays)."""
        return self.live[ptr].view(dtype)[:count]

    def tensor(self, ptr, count, dtype):
        """Adopt a library output as a torch tensor of `count` elements."""
        torch = self._torch
        if not ptr:
            return torch.empty(0, dtype=dtype, device=self._device)
        raw = self.live.pop(ptr)
        return raw.view(dtype)[:count]


def _is_torch_cuda(x) -> bool:
    try:
        import torch
    except ImportError:
        return False
    return isinstance(x, torch.Tensor) and x.is_cuda


CENTRING = {"auto": BM_CENTRE_AUTO, "always": BM_CENTRE_ALWAYS, "off": BM_CENTRE_OFF}


def _options(lib, path: str, batch: int, stream, host_io: bool, alloc: Optional[_TorchAllocator],
             skip_edges: bool = False, want_dists: bool = False, centring: str = "auto"):
    opt = bm_options()
    lib.bm_options_init(ctypes.byref(opt))
    opt.centring = CENTRING[centring]
    opt.skip_edges = 1 if skip_edges else 0
    opt.want_dists = 1 if want_dists else 0
    opt.path = PATHS[path]
    opt.batch = int(batch)
    opt.host_io = 1 if host_io else 0
    opt.stream = stream or None
    if alloc is not None:
        opt.alloc = alloc.alloc_cb
        opt.free = alloc.free_cb
    return opt


def _current_stream(device):
    import torch
    return torch.cuda.current_stream(device).cuda_stream


def _as_input(x, d_expected=None):
    """(pointer, rows, d, keepalive, host) for a float32 matrix."""
    if _is_torch_cuda(x):
        import torch
        if x.dtype != torch.float32 or x.dim() != 2:
            raise ValueError("expected a 2-D float32 CUDA tensor")
        x = x.contiguous()
        return x.data_ptr(), x.shape[0], x.shape[1], x, False
    try:
        import torch
        if isinstance(x, torch.Tensor):
            x = x.numpy()
    except ImportError:
        pass
    a = np.ascontiguousarray(x, dtype=np.float32)
    if a.ndim != 2:
        raise ValueError("expected a 2-D array")
    return (a.ctypes.data if a.size else None), a.shape[0], a.shape[1], a, True


def bm_range_query(X, Q, eps: float, path: str = "auto", stream=None, want_dists: bool = False,
                   centring: str = "auto"):
    """Exact range query R_eps(q) for every row q of Q over the points X.

    Device tensors in -> torch CUDA tensors out; host arrays in -> numpy out.
    Returns (offsets int64 [m+1], ids int32 [nnz], stats dict); with want_dists,
    (offsets, ids, stats, dists float32 [nnz]) where dists[e] = d(Q_row, X[ids[e]]).
    centring: "auto", "always" or "off" (bm_options.centring: whether the tensor-core
    tiles take the points and queries translated by the points' sample mean)."""
    lib = load()
    px, n, d, kx, hx = _as_input(X)
    pq, m, dq, kq, hq = _as_input(Q)
    if dq != d and m and n:
        raise ValueError("dimension mismatch")
    if hx != hq:
        raise ValueError("X and Q must both be device tensors or both host arrays")
    out = bm_csr()
    st = bm_stats()
    if hx:
        opt = _options(lib, path, 0, stream, True, None, want_dists=want_dists, centring=centring)
        _check(lib, lib.bm_range_query(px, n, d, pq, m, ctypes.c_float(eps), ctypes.byref(opt), ctypes.byref(out),
                                       ctypes.byref(st)))
        own = _HostResult(lib.bm_csr_free, bm_csr.from_buffer_copy(out), opt)
        off = own.view(out.offsets, ctypes.c_int64, m + 1)
        ids = own.view(out.ids, ctypes.c_int32, out.nnz)
        if want_dists:
            return off, ids, st.as_dict(), own.view(out.dists, ctypes.c_float, out.nnz)
        return off, ids, st.as_dict()
    import torch
    dev = kx.device
    alloc = _TorchAllocator(dev)
    opt = _options(lib, path, 0, stream or _current_stream(dev), False, alloc, want_dists=want_dists,
                   centring=centring)
    _check(lib, lib.bm_range_query(px, n, d, pq, m, ctypes.c_float(eps), ctypes.byref(opt), ctypes.byref(out),
                                   ctypes.byref(st)))
    off = alloc.tensor(out.offsets, m + 1, torch.int64)
    ids = alloc.tensor(out.ids, out.nnz, torch.int32)
    if want_dists:
        return off, ids, st.as_dict(), alloc.tensor(out.dists, out.nnz, torch.float32)
    return off, ids, st.as_dict()


def bm_build(X, eps: float, path: str = "auto", batch: int = 0, stream=None, skip_edges: bool = False,
             want_dists: bool = False, centring: str = "auto"):
    """Exact Ball Mapper: landmarks (greedy index order), CSR memberships, nerve edges.

    Device tensor in -> dict of torch CUDA tensors; host array in -> dict of numpy arrays.
    Keys: landmarks int32 [L], offsets int64 [L+1], ids int32 [nnz], edges int32 [E, 2], stats;
    with want_dists also dists float32 [nnz] (distance of each member to its landmark).
    centring: "auto", "always" or "off" (bm_options.centring)."""
    lib = load()
    px, n, d, kx, host = _as_input(X)
    g = bm_graph()
    if host:
        opt = _options(lib, path, batch, stream, True, None, skip_edges, want_dists, centring)
        _check(lib, lib.bm_build(px, n, d, ctypes.c_float(eps), ctypes.byref(opt), ctypes.byref(g)))
        return _host_graph(lib, g, opt, want_dists)
    dev = kx.device
    # scratch and outputs from the library's own pool (no Python call per buffer); the
    # outputs come back as zero-copy tensors that release them when the last one is gone
    opt = _options(lib, path, batch, stream or _current_stream(dev), False, None, skip_edges, want_dists, centring)
    _check(lib, lib.bm_build(px, n, d, ctypes.c_float(eps), ctypes.byref(opt), ctypes.byref(g)))
    return _device_graph(lib, g, opt, dev, want_dists)


def _graph_dict(alloc, g, want_dists=False):
    """A device bm_graph adopted as a dict of torch tensors."""
    import torch
    L, nnz, E = g.n_landmarks, g.members.nnz, g.n_edges
    res = {"landmarks": alloc.tensor(g.landmarks, L, torch.int32),
           "offsets": alloc.tensor(g.members.offsets, L + 1, torch.int64),
           "ids": alloc.tensor(g.members.ids, nnz, torch.int32),
           "edges": alloc.tensor(g.edges, 2 * E, torch.int32).view(E, 2),
           "stats": g.stats.as_dict()}
    if want_dists:
        res["dists"] = alloc.tensor(g.members.dists, nnz, torch.float32)
    return res


class _HostResult:
    """Owns the host buffers of one library result; the numpy arrays returned to the caller
    are views of them, and the buffers go back to the library (bm_graph_free / bm_csr_free)
    once the last view is gone."""

    def __init__(self, free_fn, obj, opt):
        self._free, self._obj, self._opt = free_fn, obj, opt

    def view(self, ptr, ctype, count):
        buf = (ctype * max(count, 1)).from_address(ptr)
        buf._owner = self   # the array's base chain keeps the owner alive
        return np.ctypeslib.as_array(buf)[:count]

    def __del__(self):
        try:
            self._free(ctypes.byref(self._obj), ctypes.byref(self._opt))
        except Exception:
            pass


class _CudaSpan:
    """__cuda_array_interface__ of a span of a library-owned device buffer (keeps its owner)."""

    def __init__(self, owner, ptr, count, typestr):
        self._owner = owner
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None, "stream": None}


class _DeviceResult:
    """Owns the device buffers of one library result (allocated from the library's own
    stream-ordered pool, with no call into Python per buffer); the torch tensors returned
    are views of them, and the buffers go back to the library (bm_graph_free) once the last
    tensor is gone."""

    _TYPESTR = {"int32": "<i4", "int64": "<i8", "float32": "<f4"}

    def __init__(self, free_fn, obj, opt, device):
        self._free, self._obj, self._opt, self._device = free_fn, obj, opt, device

    def tensor(self, ptr, count, dtype):
        import torch
        if count == 0 or not ptr:
            return torch.empty(0, dtype=dtype, device=self._device)
        span = _CudaSpan(self, ptr, count, self._TYPESTR[str(dtype).replace("torch.", "")])
        t = torch.as_tensor(span, device=self._device)
        t._bm_owner = span   # besides the storage's own reference to the span
        return t

    def __del__(self):
        try:
            self._free(ctypes.byref(self._obj), ctypes.byref(self._opt))
        except Exception:
            pass


def _device_graph(lib, g, opt, device, want_dists=False):
    """A device bm_graph from the library's pool as a dict of torch tensors (no copy)."""
    import torch
    own = _DeviceResult(lib.bm_graph_free, bm_graph.from_buffer_copy(g), opt, device)
    L, nnz, E = g.n_landmarks, g.members.nnz, g.n_edges
    res = {"landmarks": own.tensor(g.landmarks, L, torch.int32),
           "offsets": own.tensor(g.members.offsets, L + 1, torch.int64),
           "ids": own.tensor(g.members.ids, nnz, torch.int32),
           "edges": own.tensor(g.edges, 2 * E, torch.int32).view(E, 2),
           "stats": g.stats.as_dict()}
    if want_dists:
        res["dists"] = own.tensor(g.members.dists, nnz, torch.float32)
    return res


def _host_graph(lib, g, opt, want_dists):
    """A host bm_graph as numpy arrays (views of the library's buffers, no copy)."""
    own = _HostResult(lib.bm_graph_free, bm_graph.from_buffer_copy(g), opt)
    L, nnz, E = g.n_landmarks, g.members.nnz, g.n_edges
    res = {"landmarks": own.view(g.landmarks, ctypes.c_int32, L),
           "offsets": own.view(g.members.offsets, ctypes.c_int64, L + 1),
           "ids": own.view(g.members.ids, ctypes.c_int32, nnz),
           "edges": own.view(g.edges, ctypes.c_int32, 2 * E).reshape(E, 2),
           "stats": g.stats.as_dict()}
    if want_dists:
        res["dists"] = own.view(g.members.dists, ctypes.c_float, nnz)
    return res


def bm_build_fps(X, eps: float, first: int = 0, path: str = "auto", stream=None, want_dists: bool = False):
    """Ball Mapper on farthest-point landmarks (Sec. 2.2) starting at point `first`;
    landmarks in selection order.  Same result layout as bm_build."""
    lib = load()
    px, n, d, kx, host = _as_input(X)
    g = bm_graph()
    if host:
        opt = _options(lib, path, 0, stream, True, None, want_dists=want_dists)
        _check(lib, lib.bm_build_fps(px, n, d, ctypes.c_float(eps), int(first), ctypes.byref(opt), ctypes.byref(g)))
        return _host_graph(lib, g, opt, want_dists)
    alloc = _TorchAllocator(kx.device)
    opt = _options(lib, path, 0, stream or _current_stream(kx.device), False, alloc, want_dists=want_dists)
    _check(lib, lib.bm_build_fps(px, n, d, ctypes.c_float(eps), int(first), ctypes.byref(opt), ctypes.byref(g)))
    return _graph_dict(alloc, g, want_dists)


COLOR_STATS = {"mean": 0, "median": 1, "min": 2, "max": 3}


def bm_color(offsets, ids, f, stat: str = "mean", stream=None):
    """Coloring (Sec. 2.3): stat of f over every CSR row.  All CUDA tensors (int64 offsets,
    int32 ids, float32 f) -> float64 CUDA tensor; all numpy arrays -> numpy array."""
    lib = load()
    rows = int(offsets.shape[0]) - 1
    n = int(f.shape[0])
    if _is_torch_cuda(offsets):
        import torch
        offsets = offsets.to(torch.int64).contiguous()
        ids = ids.to(torch.int32).contiguous()
        f = f.to(torch.float32).contiguous()
        out = torch.empty(max(rows, 1), dtype=torch.float64, device=offsets.device)
        alloc = _TorchAllocator(offsets.device)
        opt = _options(lib, "auto", 0, stream or _current_stream(offsets.device), False, alloc)
        _check(lib, lib.bm_color(offsets.data_ptr(), ids.data_ptr() if ids.numel() else None, rows,
                                 f.data_ptr() if n else None, n, COLOR_STATS[stat], ctypes.byref(opt),
                                 out.data_ptr()))
        return out[:rows]
    o = np.ascontiguousarray(offsets, dtype=np.int64)
    i = np.ascontiguousarray(ids, dtype=np.int32)
    fv = np.ascontiguousarray(f, dtype=np.float32)
    out = np.empty(max(rows, 1), dtype=np.float64)
    opt = _options(lib, "auto", 0, stream, True, None)
    _check(lib, lib.bm_color(o.ctypes.data, i.ctypes.data if i.size else None, rows, fv.ctypes.data if n else None,
                             n, COLOR_STATS[stat], ctypes.byref(opt), out.ctypes.data))
    return out[:rows]


def bm_knn_dist(X, k: int, path: str = "auto", stream=None, centring: str = "auto"):
    """Distance from every point to its k-th nearest neighbour, itself counted first
    (Sec. 6.1).  Device tensor in -> float64 CUDA tensor [n]; host array in -> numpy.
    Returns (kdist, stats)."""
    lib = load()
    px, n, d, kx, host = _as_input(X)
    st = bm_stats()
    if host:
        out = np.empty(max(n, 1), dtype=np.float64)
        opt = _options(lib, path, 0, stream, True, None, centring=centring)
        _check(lib, lib.bm_knn_dist(px, n, d, int(k), ctypes.byref(opt), out.ctypes.data, ctypes.byref(st)))
        return out[:n], st.as_dict()
    import torch
    out = torch.empty(max(n, 1), dtype=torch.float64, device=kx.device)
    alloc = _TorchAllocator(kx.device)
    opt = _options(lib, path, 0, stream or _current_stream(kx.device), False, alloc, centring=centring)
    _check(lib, lib.bm_knn_dist(px, n, d, int(k), ctypes.byref(opt), out.data_ptr(), ctypes.byref(st)))
    return out[:n], st.as_dict()


def bm_occupancy_eps(X, k: int, path: str = "auto", stream=None, centring: str = "auto"):
    """Target-occupancy scale (Sec. 6.1): median over the points of the k-th NN distance.
    Returns (eps as a Python float, stats)."""
    lib = load()
    px, n, d, kx, host = _as_input(X)
    st = bm_stats()
    eps = ctypes.c_double(0.0)
    if host:
        opt = _options(lib, path, 0, stream, True, None, centring=centring)
    else:
        alloc = _TorchAllocator(kx.device)
        opt = _options(lib, path, 0, stream or _current_stream(kx.device), False, alloc, centring=centring)
    _check(lib, lib.bm_occupancy_eps(px, n, d, int(k), ctypes.byref(opt), ctypes.byref(eps), ctypes.byref(st)))
    return eps.value, st.as_dict()


def bm_build_batched(instances, path: str = "auto", batch: int = 0, stream=None, skip_edges: bool = False,
                     batches=None, centring: str = "auto"):
    """Many independent exact builds in one call; the greedy loops of all instances
    run inside one CUDA graph.  instances: sequence of (X, eps), all CUDA tensors
    (results as torch tensors) or all host arrays (results as numpy arrays).
    batches: optional per-instance largest greedy batch (0 = `batch`), e.g. from
    autotune.batches_for.  Returns a list of dicts shaped like bm_build's."""
    lib = load()
    ins = [_as_input(X) for X, _ in instances]
    hosts = {h for _, _, _, _, h in ins}
    if len(hosts) > 1:
        raise ValueError("instances must all be device tensors or all host arrays")
    host = hosts.pop() if hosts else False
    count = len(ins)
    if batches is not None and len(batches) != count:
        raise ValueError("batches needs one entry per instance")
    arr_in = (bm_instance * max(count, 1))()
    for k, ((px, n, d, _, _), (_, eps)) in enumerate(zip(ins, instances)):
        arr_in[k].X = px
        arr_in[k].n = n
        arr_in[k].d = d
        arr_in[k].eps = float(eps)
        arr_in[k].batch = int(batches[k]) if batches is not None else 0
    outs = (bm_graph * max(count, 1))()
    statuses = (ctypes.c_int32 * max(count, 1))()
    if host:
        opt = _options(lib, path, batch, stream, True, None, skip_edges, centring=centring)
        _check(lib, lib.bm_build_batched(arr_in, count, ctypes.byref(opt), outs, statuses))
        return [_host_graph(lib, outs[k], opt, False) for k in range(count)]
    import torch
    dev = ins[0][3].device if count else torch.device("cuda", torch.cuda.current_device())
    opt = _options(lib, path, batch, stream or _current_stream(dev), False, None, skip_edges, centring=centring)
    _check(lib, lib.bm_build_batched(arr_in, count, ctypes.byref(opt), outs, statuses))
    return [_device_graph(lib, outs[k], opt, dev) for k in range(count)]


def tile_shapes():
    """The compiled tensor-core tile shapes, as dicts (d_pad = 0)."""
    lib = load()
    n = lib.bm_tile_shapes(None, 0)
    arr = (bm_tile_config * max(n, 1))()
    lib.bm_tile_shapes(arr, n)
    return [arr[i].as_dict() for i in range(n)]


def get_tile_config(d: int) -> dict:
    """Tile configuration used for point dimension d."""
    lib = load()
    c = bm_tile_config()
    _check(lib, lib.bm_get_tile_config(int(d), ctypes.byref(c)))
    return c.as_dict()


def set_tile_config(d: int, cfg: Optional[dict]) -> None:
    """Override the tile configuration for dimension d (None: the built-in choice)."""
    lib = load()
    if cfg is None:
        _check(lib, lib.bm_set_tile_config(int(d), None))
        return
    c = bm_tile_config(**{k: int(cfg[k]) for k in ("d_pad", "ck", "nt", "bbuf", "astg")})
    _check(lib, lib.bm_set_tile_config(int(d), ctypes.byref(c)))


def set_nerve_bitmap_bytes(nbytes: int) -> int:
    """Bitmap budget of the nerve-edge deduplication (0 = default, < 0 = always
    sort); returns the previous setting."""
    return int(load().bm_set_nerve_bitmap_bytes(int(nbytes)))


def version() -> int:
    return int(load().bm_version())


def bm_range_count_noalloc(X, Q, eps: float, counts, stream=None):
    """|R_eps(q)| for every row q of Q, written into the caller's int64 CUDA tensor
    `counts` (length m).  The library allocates nothing for this call: it works in
    a fixed scratch area compiled into it (see the C header for limits)."""
    import torch
    lib = load()
    if not (_is_torch_cuda(X) and _is_torch_cuda(Q) and _is_torch_cuda(counts)):
        raise ValueError("X, Q and counts must be CUDA tensors")
    if counts.dtype != torch.int64 or not counts.is_contiguous() or counts.numel() != Q.shape[0]:
        raise ValueError("counts must be a contiguous int64 tensor with one entry per query")
    px, n, d, kx, _ = _as_input(X)
    pq, m, dq, kq, _ = _as_input(Q)
    if m and n and dq != d:
        raise ValueError("dimension mismatch")
    st = stream or _current_stream(kx.device)
    _check(lib, lib.bm_range_count_noalloc(px, n, d, pq, m, ctypes.c_float(eps), st, counts.data_ptr()))
    return counts


class IvfIndex:
    """Inverted-file index over device points X (bm_ivf_train).  The index refers to X,
    which must stay alive and unchanged; its own buffers come from torch's allocator."""

    def __init__(self, X, nlist: int = 1024, iters: int = 20, sample: int = 0, seed: int = 0, path: str = "auto"):
        """path: the scan's arithmetic for queries and builds (auto / tc: bf16-split tensor-core
        tiles over the cells laid out in whole tiles; fp32: CUDA-core tiles)."""
        import torch
        self._path = path
        self._lib = load()
        if not _is_torch_cuda(X):
            raise ValueError("X must be a CUDA tensor")
        px, n, d, kx, _ = _as_input(X)
        self._X = kx
        self._alloc = _TorchAllocator(kx.device)
        self._opt = _options(self._lib, "fp32", 0, _current_stream(kx.device), False, self._alloc)
        h = ctypes.c_void_p()
        _check(self._lib, self._lib.bm_ivf_train(px, n, d, int(nlist), int(iters), int(sample), int(seed),
                                                 ctypes.byref(self._opt), ctypes.byref(h)))
        self._h = h
        n_ = ctypes.c_int64()
        d_ = ctypes.c_int32()
        nl = ctypes.c_int32()
        co = ctypes.c_void_p()
        ce = ctypes.c_void_p()
        _check(self._lib, self._lib.bm_ivf_info(h, ctypes.byref(n_), ctypes.byref(d_), ctypes.byref(nl),
                                                ctypes.byref(co), ctypes.byref(ce)))
        self.n, self.d, self.nlist = n_.value, d_.value, nl.value
        self.cell_of = self._alloc.peek(co.value, self.n, torch.int32)
        self.centroids = self._alloc.peek(ce.value, self.nlist * self.d, torch.float32).view(self.nlist, self.d)

    def range_query(self, Q, eps: float, nprobe: int, want_dists: bool = False, path: Optional[str] = None):
        """(offsets, ids, probes, stats): conservative range sets over the nprobe nearest cells;
        with want_dists, (offsets, ids, probes, stats, dists)."""
        import torch
        pq, m, dq, kq, _ = _as_input(Q)
        if not _is_torch_cuda(Q):
            raise ValueError("Q must be a CUDA tensor")
        probes = torch.empty((m, nprobe), dtype=torch.int32, device=kq.device)
        alloc = _TorchAllocator(kq.device)
        opt = _options(self._lib, path or self._path, 0, _current_stream(kq.device), False, alloc,
                       want_dists=want_dists)
        out = bm_csr()
        st = bm_stats()
        _check(self._lib, self._lib.bm_ivf_range_query(self._h, pq, m, ctypes.c_float(eps), int(nprobe),
                                                       ctypes.byref(opt), ctypes.byref(out),
                                                       probes.data_ptr() if m else None, ctypes.byref(st)))
        res = (alloc.tensor(out.offsets, m + 1, torch.int64), alloc.tensor(out.ids, out.nnz, torch.int32), probes,
               st.as_dict())
        if want_dists:
            res = res + (alloc.tensor(out.dists, out.nnz, torch.float32),)
        return res

    def build(self, eps: float, nprobe: int, landmarks=None, batch: int = 0, want_dists: bool = False,
              path: Optional[str] = None):
        """Ball Mapper through the index: fixed-landmark mode (landmarks = CUDA int32 tensor)
        or end-to-end mode (landmarks None)."""
        import torch
        dev = self._X.device
        alloc = _TorchAllocator(dev)
        opt = _options(self._lib, path or self._path, batch, _current_stream(dev), False, alloc,
                       want_dists=want_dists)
        g = bm_graph()
        lm_ptr, nl = None, 0
        if landmarks is not None:
            landmarks = landmarks.to(device=dev, dtype=torch.int32).contiguous()
            lm_ptr, nl = landmarks.data_ptr() if landmarks.numel() else None, landmarks.numel()
        _check(self._lib, self._lib.bm_build_ivf(self._h, ctypes.c_float(eps), int(nprobe), lm_ptr, nl,
                                                 ctypes.byref(opt), ctypes.byref(g)))
        return _graph_dict(alloc, g, want_dists)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.bm_ivf_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GraphIndex:
    """Proximity-graph index over device points X (bm_gidx_build): every point's M nearest
    other points, made undirected.  The index refers to X, which must stay alive and
    unchanged; its own buffers come from torch's allocator."""

    def __init__(self, X, M: int = 16, n_entries: int = 0, path: str = "auto"):
        import torch
        self._lib = load()
        if not _is_torch_cuda(X):
            raise ValueError("X must be a CUDA tensor")
        px, n, d, kx, _ = _as_input(X)
        self._X = kx
        self._alloc = _TorchAllocator(kx.device)
        self._opt = _options(self._lib, path, 0, _current_stream(kx.device), False, self._alloc)
        h = ctypes.c_void_p()
        _check(self._lib, self._lib.bm_gidx_build(px, n, d, int(M), int(n_entries), ctypes.byref(self._opt),
                                                  ctypes.byref(h)))
        self._h = h
        n_ = ctypes.c_int64()
        d_ = ctypes.c_int32()
        na = ctypes.c_int64()
        ao = ctypes.c_void_p()
        aj = ctypes.c_void_p()
        _check(self._lib, self._lib.bm_gidx_info(h, ctypes.byref(n_), ctypes.byref(d_), ctypes.byref(na),
                                                 ctypes.byref(ao), ctypes.byref(aj)))
        self.n, self.d, self.n_adj = n_.value, d_.value, na.value
        self.adj_off = self._alloc.peek(ao.value, self.n + 1, torch.int64)
        self.adj = self._alloc.peek(aj.value, self.n_adj, torch.int32)

    def range_query(self, Q, eps: float, ef: int, max_visits: int = 0, want_dists: bool = False):
        """(offsets, ids, stats): conservative range sets through the graph search."""
        import torch
        pq, m, dq, kq, _ = _as_input(Q)
        if not _is_torch_cuda(Q):
            raise ValueError("Q must be a CUDA tensor")
        alloc = _TorchAllocator(kq.device)
        opt = _options(self._lib, "auto", 0, _current_stream(kq.device), False, alloc, want_dists=want_dists)
        out = bm_csr()
        st = bm_stats()
        _check(self._lib, self._lib.bm_gidx_range_query(self._h, pq, m, ctypes.c_float(eps), int(ef), int(max_visits),
                                                        ctypes.byref(opt), ctypes.byref(out), ctypes.byref(st)))
        res = (alloc.tensor(out.offsets, m + 1, torch.int64), alloc.tensor(out.ids, out.nnz, torch.int32),
               st.as_dict())
        if want_dists:
            res = res + (alloc.tensor(out.dists, out.nnz, torch.float32),)
        return res

    def build(self, eps: float, ef: int, max_visits: int = 0, landmarks=None, batch: int = 0,
              want_dists: bool = False):
        """Ball Mapper through the graph: fixed-landmark mode (landmarks = CUDA int32 tensor)
        or end-to-end mode (landmarks None)."""
        import torch
        dev = self._X.device
        alloc = _TorchAllocator(dev)
        opt = _options(self._lib, "auto", batch, _current_stream(dev), False, alloc, want_dists=want_dists)
        g = bm_graph()
        lm_ptr, nl = None, 0
        if landmarks is not None:
            landmarks = landmarks.to(device=dev, dtype=torch.int32).contiguous()
            lm_ptr, nl = landmarks.data_ptr() if landmarks.numel() else None, landmarks.numel()
        _check(self._lib, self._lib.bm_build_gidx(self._h, ctypes.c_float(eps), int(ef), int(max_visits), lm_ptr, nl,
                                                  ctypes.byref(opt), ctypes.byref(g)))
        return _graph_dict(alloc, g, want_dists)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.bm_gidx_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def band_halfwidth(path: str, d: int, d_pad: int, n_a: float, n_b: float, phi_a: float, phi_b: float) -> float:
    """The proven error-band half-width of a tile path (bm_band_halfwidth), in units of
    v = (eps^2 - D)/2; path: "tc", "tc16" or "fp32"."""
    return float(load().bm_band_halfwidth(PATHS[path], int(d), int(d_pad), float(n_a), float(n_b), float(phi_a),
                                          float(phi_b)))
