"""Python binding of libffm_gb300.so (C ABI in include/ffm.h): argument marshalling only.

Every step of the computation runs in the library's CUDA kernels.  There is no CPU path:
if the shared library is missing or a CUDA device is not available, calls raise.

Arrays may be torch tensors (CUDA or CPU) or numpy arrays (host memory); host arrays are
staged to the device by the library.  Densities are laid out (nrhs, N) row-major, which
is the ABI's column-major N x nrhs.
"""
import ctypes as C
import os

import numpy as np

try:
    import torch
except ImportError:  # pragma: no cover - torch is part of the environment
    torch = None

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libffm_gb300.so")

LAPLACE, HELMHOLTZ, LAPLACE_DL, LAPLACE_GRAD = 0, 1, 2, 3
F32, F64, C64, C128 = 0, 1, 2, 3
# plane-wave level arithmetic (ffm_precision)
PREC_AUTO, PREC_F32, PREC_F32C, PREC_F64, PREC_F32X2 = 0, 1, 2, 3, 4
# Lagrange transfer variants (ffm_opts.lagrange_transfer)
LAG_DEFAULT, LAG_CUDA_CORES, LAG_TC_TRANSLATION, LAG_TC_TARGET = 0, 1, 2, 3
# plane-wave source / target steps (ffm_opts.pw_transform)
PW_AUTO, PW_DIRECT, PW_NUFFT, PW_DIRECT_TC = 0, 1, 2, 3
EXPORT_PERM_X, EXPORT_PERM_Y, EXPORT_ADM, EXPORT_NEAR = 0, 1, 2, 3
STATUS = {0: "FFM_OK", 1: "FFM_EINVAL", 2: "FFM_ENOMEM", 3: "FFM_ECUDA", 4: "FFM_ETIMEOUT", 5: "FFM_EUNSUPPORTED"}

# Every symbol include/ffm.h declares.
ABI_SYMBOLS = ("ffm_plan", "ffm_apply", "ffm_destroy", "ffm_plan_bytes", "ffm_plan_info", "ffm_plan_export",
               "ffm_launch_count", "ffm_profile_enable", "ffm_profile_reset", "ffm_profile_read", "ffm_status_str",
               "ffm_last_error", "ffm_morton_order_noalloc", "ffm_graph_create", "ffm_graph_launch",
               "ffm_graph_kernels", "ffm_graph_destroy", "ffm_autotune", "ffm_bem_create", "ffm_bem_apply",
               "ffm_bem_solve", "ffm_bem_products", "ffm_bem_destroy")


class FFMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class Opts(C.Structure):
    _fields_ = [("n_leaf", C.c_int), ("l_cap", C.c_int), ("kappa_switch", C.c_double), ("r1_override", C.c_int),
                ("precision", C.c_int), ("weights", C.c_void_p), ("weights_dtype", C.c_int),
                ("autotune_cache", C.c_char_p), ("lagrange_transfer", C.c_int), ("normals", C.c_void_p),
                ("normals_dtype", C.c_int), ("pw_transform", C.c_int), ("aca_eps", C.c_double),
                ("wait_tries", C.c_int)]


class Info(C.Structure):
    _fields_ = [("l_stop", C.c_int), ("root_admissible", C.c_int), ("d0", C.c_double), ("oX", C.c_double * 3),
                ("oY", C.c_double * 3), ("nboxX", C.c_int64 * 22), ("nboxY", C.c_int64 * 22),
                ("n_adm", C.c_int64 * 22), ("n_near", C.c_int64 * 22), ("n_trans", C.c_int64 * 22),
                ("mode", C.c_int * 22), ("r1", C.c_int * 22), ("L", C.c_int * 22), ("nQ", C.c_int * 22),
                ("nx", C.c_int64), ("ny", C.c_int64), ("src_points", C.c_int64 * 22),
                ("tgt_points", C.c_int64 * 22), ("p2p_pairs", C.c_int64), ("pw_prec", C.c_int * 22),
                ("cancel", C.c_double * 22), ("device_errors", C.c_int), ("autotuned", C.c_int),
                ("p2p_tchunk", C.c_int), ("p2p_smax", C.c_int), ("tune_tc", C.c_int * 22),
                ("tune_pw", (C.c_int * 3) * 22), ("nufft", C.c_int * 22), ("nufft_w", C.c_int * 22),
                ("nufft_n2", C.c_int * 22), ("n_src_boxes", C.c_int64 * 22), ("n_tgt_boxes", C.c_int64 * 22),
                ("pw_recurrences", C.c_int64 * 22), ("aca_rank", C.c_int * 22), ("aca_terms", C.c_int64 * 22),
                ("aca_pair_terms", C.c_int64 * 22)]

    def as_dict(self):
        d = {"l_stop": self.l_stop, "root_admissible": self.root_admissible, "d0": self.d0, "oX": list(self.oX),
             "oY": list(self.oY), "nx": self.nx, "ny": self.ny, "p2p_pairs": self.p2p_pairs,
             "device_errors": self.device_errors, "autotuned": self.autotuned, "p2p_tchunk": self.p2p_tchunk,
             "p2p_smax": self.p2p_smax, "tune_pw": [list(r) for r in self.tune_pw]}
        for f in ("nboxX", "nboxY", "n_adm", "n_near", "n_trans", "mode", "r1", "L", "nQ", "src_points",
                  "tgt_points", "pw_prec", "cancel", "tune_tc", "nufft", "nufft_w", "nufft_n2",
                  "n_src_boxes", "n_tgt_boxes", "pw_recurrences", "aca_rank", "aca_terms", "aca_pair_terms"):
            d[f] = list(getattr(self, f))
        return d


_lib = None


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libffm_gb300.so is not built (run __graft_entry__.build() or "
                               "python -m paper_1909_05600_gb300.build); there is no CPU fallback")
        L = C.CDLL(LIB_PATH)
        vp, i64 = C.c_void_p, C.c_int64
        L.ffm_plan.argtypes = [vp, C.c_int, i64, vp, C.c_int, i64, C.c_int, C.c_double, C.c_double, C.POINTER(Opts),
                               vp, C.POINTER(vp)]
        L.ffm_plan.restype = C.c_int
        L.ffm_apply.argtypes = [vp, vp, C.c_int, C.c_int, vp, vp]
        L.ffm_apply.restype = C.c_int
        L.ffm_destroy.argtypes = [vp]
        L.ffm_destroy.restype = None
        L.ffm_plan_bytes.argtypes = [vp, C.POINTER(C.c_size_t)]
        L.ffm_plan_bytes.restype = C.c_int
        L.ffm_plan_info.argtypes = [vp, C.POINTER(Info)]
        L.ffm_plan_info.restype = C.c_int
        L.ffm_plan_export.argtypes = [vp, C.c_int, C.c_int, vp, C.POINTER(i64)]
        L.ffm_plan_export.restype = C.c_int
        L.ffm_launch_count.restype = C.c_uint64
        L.ffm_profile_enable.argtypes = [C.c_int]
        L.ffm_profile_enable.restype = None
        L.ffm_profile_reset.restype = None
        L.ffm_profile_read.argtypes = [C.c_char_p, C.POINTER(C.c_uint64), C.POINTER(C.c_double), C.c_int]
        L.ffm_profile_read.restype = C.c_int
        L.ffm_status_str.argtypes = [C.c_int]
        L.ffm_status_str.restype = C.c_char_p
        L.ffm_last_error.restype = C.c_char_p
        L.ffm_morton_order_noalloc.argtypes = [vp, C.c_int, i64, vp, vp]
        L.ffm_morton_order_noalloc.restype = C.c_int
        L.ffm_graph_create.argtypes = [vp, vp, C.c_int, C.c_int, vp, C.POINTER(vp)]
        L.ffm_graph_create.restype = C.c_int
        L.ffm_graph_launch.argtypes = [vp, vp]
        L.ffm_graph_launch.restype = C.c_int
        L.ffm_graph_kernels.argtypes = [vp]
        L.ffm_graph_kernels.restype = i64
        L.ffm_graph_destroy.argtypes = [vp]
        L.ffm_graph_destroy.restype = None
        L.ffm_autotune.argtypes = [vp, C.c_int, C.c_char_p, vp]
        L.ffm_autotune.restype = C.c_int
        L.ffm_bem_create.argtypes = [vp, i64, vp, i64, C.c_int, C.c_double, C.c_double, C.POINTER(Opts), vp,
                                     C.POINTER(vp)]
        L.ffm_bem_create.restype = C.c_int
        L.ffm_bem_apply.argtypes = [vp, vp, vp, vp]
        L.ffm_bem_apply.restype = C.c_int
        L.ffm_bem_solve.argtypes = [vp, vp, vp, C.c_double, C.c_int, C.c_int, C.POINTER(C.c_int),
                                    C.POINTER(C.c_double), vp]
        L.ffm_bem_solve.restype = C.c_int
        L.ffm_bem_products.argtypes = [vp, C.POINTER(C.c_int64)]
        L.ffm_bem_products.restype = C.c_int
        L.ffm_bem_destroy.argtypes = [vp]
        L.ffm_bem_destroy.restype = None
        _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        raise FFMError(rc, lib().ffm_last_error().decode())


def launch_count():
    return int(lib().ffm_launch_count())


def profile_enable(on=True):
    """Bracket every kernel launch of the library with CUDA events (per-kernel device time)."""
    lib().ffm_profile_enable(1 if on else 0)


def profile_reset():
    lib().ffm_profile_reset()


def profile_read(cap=256):
    """{kernel name: (launches, total device ms)} since the last reset."""
    names = C.create_string_buffer(64 * cap)
    n_l = (C.c_uint64 * cap)()
    ms = (C.c_double * cap)()
    n = lib().ffm_profile_read(names, n_l, ms, cap)
    out = {}
    for i in range(n):
        nm = names.raw[64 * i:64 * (i + 1)].split(b"\0", 1)[0].decode()
        out[nm] = (int(n_l[i]), float(ms[i]))
    return out


_TORCH_DT = None


def _dtype_code(a):
    global _TORCH_DT
    if torch is not None and isinstance(a, torch.Tensor):
        if _TORCH_DT is None:
            _TORCH_DT = {torch.float32: F32, torch.float64: F64, torch.complex64: C64, torch.complex128: C128}
        return _TORCH_DT[a.dtype]
    return {np.dtype(np.float32): F32, np.dtype(np.float64): F64, np.dtype(np.complex64): C64,
            np.dtype(np.complex128): C128}[a.dtype]


def _ptr(a):
    if torch is not None and isinstance(a, torch.Tensor):
        assert a.is_contiguous(), "tensors must be contiguous"
        return a.data_ptr()
    assert a.flags["C_CONTIGUOUS"], "arrays must be C-contiguous"
    return a.ctypes.data


def _stream_of(*arrays, stream=None):
    if stream is not None:
        return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    if torch is not None:
        for a in arrays:
            if isinstance(a, torch.Tensor) and a.is_cuda:
                return torch.cuda.current_stream(a.device).cuda_stream
    return 0


NOALLOC_MAX_POINTS = 262144


class Graph:
    """ffm_graph_create / ffm_graph_launch / ffm_graph_destroy.  Keeps the plan and the
    two buffers alive while it exists."""

    def __init__(self, plan, u, out):
        self._h = None
        one = u.ndim == 1
        nrhs = 1 if one else int(u.shape[0])
        self._keep = (plan, u, out)
        h = C.c_void_p()
        _check(lib().ffm_graph_create(plan._h, _ptr(u), _dtype_code(u), nrhs, _ptr(out), C.byref(h)))
        self._h = h
        self.kernels = int(lib().ffm_graph_kernels(h))

    def launch(self, stream=None):
        s = _stream_of(self._keep[1], self._keep[2], stream=stream)
        _check(lib().ffm_graph_launch(self._h, s))

    def close(self):
        if self._h:
            lib().ffm_graph_destroy(self._h)
            self._h = None
        self._keep = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def morton_order_noalloc(X, perm_out, stream=None):
    """ffm_morton_order_noalloc: Morton ordering of X (n x 3, device) into perm_out (n int32 or
    uint32 entries, device), without any device allocation inside the library.  Every entry
    of perm_out is 0xFFFFFFFF once the stream has run if a coordinate was not finite."""
    if torch is None or not isinstance(X, torch.Tensor) or not isinstance(perm_out, torch.Tensor):
        raise TypeError("X and perm_out must be CUDA tensors")
    n = int(X.shape[0])
    if X.dim() != 2 or X.shape[1] != 3:
        raise ValueError("X must have shape (n, 3)")
    ok_dt = (torch.int32,) + ((torch.uint32,) if hasattr(torch, "uint32") else ())
    if perm_out.dtype not in ok_dt or perm_out.numel() < n:
        raise ValueError("perm_out must hold at least n 32-bit integers")
    cur = torch.cuda.current_device()
    if not (X.is_cuda and perm_out.is_cuda and X.device.index == cur and perm_out.device.index == cur):
        raise ValueError("X and perm_out must be on the current CUDA device")
    _check(lib().ffm_morton_order_noalloc(_ptr(X), _dtype_code(X), int(X.shape[0]), _ptr(perm_out),
                                          _stream_of(X, stream=stream)))
    return perm_out


class Plan:
    """ffm_plan / ffm_apply / ffm_destroy.

    X: (nx, 3), Y: (ny, 3) float32/float64; kernel LAPLACE or HELMHOLTZ; eps in (0, 1);
    weights: (ny,) float32/float64 or None.
    """

    def __init__(self, X, Y, kernel, k=0.0, eps=1e-3, weights=None, stream=None, n_leaf=0, l_cap=0,
                 kappa_switch=0.0, r1_override=0, precision=PREC_AUTO, autotune_cache=None,
                 lagrange_transfer=0, normals=None, pw_transform=PW_AUTO, aca_eps=0.0, wait_tries=0):
        """normals: (ny, 3) source normals, required for LAPLACE_DL (double layer).
        pw_transform: PW_AUTO, PW_DIRECT, PW_NUFFT or PW_DIRECT_TC for the plane-wave levels'
        F steps (PW_DIRECT_TC: direct sums, on the tensor cores from 2 right-hand sides).
        aca_eps: LAPLACE only; > 0 replaces each transfer matrix by its adaptive cross
        approximation to that Frobenius tolerance (eq. 11).
        wait_tries: attempts per bounded device-side wait (0: the default; -1: none, so the
        failure path runs and info() raises FFM_ETIMEOUT)."""
        self._h = None
        self._keep = (X, Y, weights, normals)
        o = Opts(n_leaf, l_cap, float(kappa_switch), r1_override, int(precision), None, F64,
                 autotune_cache.encode() if autotune_cache else None, int(lagrange_transfer), None, F64,
                 int(pw_transform), float(aca_eps), int(wait_tries))
        if normals is not None:
            o.normals = _ptr(normals)
            o.normals_dtype = _dtype_code(normals)
        if weights is not None:
            o.weights = _ptr(weights)
            o.weights_dtype = _dtype_code(weights)
        self.stream = _stream_of(X, Y, stream=stream)
        self.nx, self.ny = int(X.shape[0]), int(Y.shape[0])
        self.kernel = kernel
        h = C.c_void_p()
        _check(lib().ffm_plan(_ptr(X), _dtype_code(X), self.nx, _ptr(Y), _dtype_code(Y), self.ny, kernel, float(k),
                              float(eps), C.byref(o), self.stream, C.byref(h)))
        self._h = h
        self._keep = None

    def close(self):
        if self._h:
            lib().ffm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def apply(self, u, out=None, stream=None):
        """v = G W u.  u: (ny,) or (nrhs, ny); returns (nx,) or (nrhs, nx) of u's dtype,
        on u's device (torch) or as a numpy array (numpy input).  LAPLACE_GRAD returns
        (3, nx) or (nrhs, 3, nx): the three components of the gradient."""
        one = u.ndim == 1
        nrhs = 1 if one else int(u.shape[0])
        shape = (self.nx,) if one else (nrhs, self.nx)
        if self.kernel == LAPLACE_GRAD:
            shape = (3, self.nx) if one else (nrhs, 3, self.nx)
        if out is None:
            if torch is not None and isinstance(u, torch.Tensor):
                out = torch.empty(shape, dtype=u.dtype, device=u.device)
            else:
                out = np.empty(shape, dtype=u.dtype)
        s = _stream_of(u, out, stream=stream)
        _check(lib().ffm_apply(self._h, _ptr(u), _dtype_code(u), nrhs, _ptr(out), s))
        return out

    def autotune(self, nrhs=1, cache_path=None, stream=None):
        """Time kernel variants on this plan and keep the fastest (ffm_autotune)."""
        s = _stream_of(stream=stream) if stream is not None else (
            torch.cuda.current_stream().cuda_stream if torch is not None and torch.cuda.is_available() else 0)
        _check(lib().ffm_autotune(self._h, int(nrhs), cache_path.encode() if cache_path else None, s))
        return self.info()

    def graph(self, u, out):
        """Capture apply(u, out) into a CUDA graph (device tensors only); Graph.launch()
        recomputes `out` from the current contents of `u`."""
        return Graph(self, u, out)

    def info(self):
        inf = Info()
        _check(lib().ffm_plan_info(self._h, C.byref(inf)))
        return inf.as_dict()

    def bytes(self):
        b = C.c_size_t()
        _check(lib().ffm_plan_bytes(self._h, C.byref(b)))
        return int(b.value)

    def perm(self, which):
        what = EXPORT_PERM_X if which == "X" else EXPORT_PERM_Y
        n = C.c_int64()
        _check(lib().ffm_plan_export(self._h, what, 0, None, C.byref(n)))
        out = np.zeros(n.value, np.int64)
        _check(lib().ffm_plan_export(self._h, what, 0, out.ctypes.data, C.byref(n)))
        return out

    def pairs(self, level, which):
        """(n, 2) uint64 Morton box ids (X box, Y box): which='adm' at `level`, 'near' at the stop level."""
        what = EXPORT_ADM if which == "adm" else EXPORT_NEAR
        n = C.c_int64()
        _check(lib().ffm_plan_export(self._h, what, level, None, C.byref(n)))
        out = np.zeros((n.value, 2), np.uint64)
        if n.value:
            _check(lib().ffm_plan_export(self._h, what, level, out.ctypes.data, C.byref(n)))
        return out


class Bem:
    """Boundary-element operator S = (Lambda*)^T (G W) Lambda + C of the Laplace single layer on
    P1 functions over a triangle mesh (ffm_bem_create / ffm_bem_apply / ffm_bem_solve /
    ffm_bem_destroy).  vertices (nv, 3) float64, triangles (nt, 3) int32; vectors are float64
    (nv,) arrays or tensors."""

    def __init__(self, vertices, triangles, eps=1e-3, stream=None):
        self._h = None
        self.nv = int(vertices.shape[0])
        self.stream = _stream_of(vertices, triangles, stream=stream)
        h = C.c_void_p()
        _check(lib().ffm_bem_create(_ptr(vertices), self.nv, _ptr(triangles), int(triangles.shape[0]), LAPLACE, 0.0,
                                    float(eps), None, self.stream, C.byref(h)))
        self._h = h

    def apply(self, u, out=None):
        if out is None:
            out = torch.empty_like(u) if torch is not None and isinstance(u, torch.Tensor) else np.empty_like(u)
        _check(lib().ffm_bem_apply(self._h, _ptr(u), _ptr(out), self.stream))
        return out

    def solve(self, rhs, tol=1e-8, restart=30, maxit=300, out=None):
        """GMRES for S x = rhs: returns (x, iterations, relative residual)."""
        if out is None:
            out = torch.empty_like(rhs) if torch is not None and isinstance(rhs, torch.Tensor) else np.empty_like(rhs)
        it = C.c_int()
        rr = C.c_double()
        _check(lib().ffm_bem_solve(self._h, _ptr(rhs), _ptr(out), float(tol), int(restart), int(maxit), C.byref(it),
                                   C.byref(rr), self.stream))
        return out, it.value, rr.value

    def products(self):
        n = C.c_int64()
        _check(lib().ffm_bem_products(self._h, C.byref(n)))
        return n.value

    def close(self):
        if self._h:
            lib().ffm_bem_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
