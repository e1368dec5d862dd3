"""Python access to the FP64 CPU oracle (test infrastructure only).

Thin ctypes marshalling around oracle/libffm_oracle.so: the direct sum of eq. 3 (O1),
the plain CPU FFM of Sec. 2 (O2) and the component functions the pins exercise.  Only
tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import this module.
It imports nothing from the CUDA package.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

LAPLACE, HELMHOLTZ, POLY, LAPLACE_DL, LAPLACE_GRAD = 0, 1, 2, 3, 4
MODE_NONE, MODE_LAGRANGE, MODE_PLANEWAVE = 0, 1, 2
LMAX = 21

_lib = None

_dp = C.POINTER(C.c_double)
_i64p = C.POINTER(C.c_int64)
_u64p = C.POINTER(C.c_uint64)


class Opts(C.Structure):
    _fields_ = [("n_leaf", C.c_int), ("l_cap", C.c_int), ("kappa_switch", C.c_double),
                ("r1_override", C.c_int), ("mode_override", C.c_int), ("pw_transform", C.c_int),
                ("aca_eps", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("l_stop", C.c_int), ("root_admissible", C.c_int), ("d0", C.c_double),
                ("oX", C.c_double * 3), ("oY", C.c_double * 3),
                ("nboxX", C.c_int64 * (LMAX + 1)), ("nboxY", C.c_int64 * (LMAX + 1)),
                ("n_adm", C.c_int64 * (LMAX + 1)), ("n_near", C.c_int64 * (LMAX + 1)),
                ("n_trans", C.c_int64 * (LMAX + 1)), ("mode", C.c_int * (LMAX + 1)),
                ("r1", C.c_int * (LMAX + 1)), ("L", C.c_int * (LMAX + 1)), ("nQ", C.c_int * (LMAX + 1)),
                ("aca_rank", C.c_int * (LMAX + 1))]

    def as_dict(self):
        out = {"l_stop": self.l_stop, "root_admissible": self.root_admissible, "d0": self.d0,
               "oX": list(self.oX), "oY": list(self.oY)}
        for name in ("nboxX", "nboxY", "n_adm", "n_near", "n_trans", "mode", "r1", "L", "nQ", "aca_rank"):
            out[name] = list(getattr(self, name))
        return out


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_direct.argtypes = [_dp, C.c_int64, _dp, C.c_int64, _dp, _dp, _dp, C.c_int, C.c_int, C.c_double,
                                 _i64p, C.c_int64, _dp, _dp]
        L.orc_direct.restype = C.c_int
        L.orc_plan_create.argtypes = [_dp, C.c_int64, _dp, C.c_int64, C.c_int, C.c_double, C.c_double,
                                      C.POINTER(Opts)]
        L.orc_plan_create.restype = C.c_void_p
        L.orc_plan_destroy.argtypes = [C.c_void_p]
        L.orc_plan_stats.argtypes = [C.c_void_p, C.POINTER(Stats)]
        L.orc_plan_pairs.argtypes = [C.c_void_p, C.c_int, C.c_int, _u64p, _u64p]
        L.orc_plan_pairs.restype = C.c_int64
        L.orc_plan_perm.argtypes = [C.c_void_p, C.c_int, _i64p]
        L.orc_apply.argtypes = [C.c_void_p, _dp, _dp, _dp, C.c_int, _dp, _dp]
        L.orc_apply.restype = C.c_int
        L.orc_default_opts.argtypes = [C.POINTER(Opts)]
        L.orc_admissible.argtypes = [_dp, C.c_int, _i64p]
        L.orc_admissible.restype = C.c_int
        L.orc_morton.argtypes = [C.c_uint64] * 3
        L.orc_morton.restype = C.c_uint64
        L.orc_aca.argtypes = [_dp, C.c_int, C.c_int, C.c_double, C.c_int, _dp, _dp]
        L.orc_aca.restype = C.c_int
        L.orc_r1_rule.argtypes = [C.c_int, C.c_double]
        L.orc_r1_rule.restype = C.c_int
        L.orc_r1_table.argtypes = [C.c_int, _dp]
        L.orc_lagrange_block_err.argtypes = [C.c_int, C.c_double, C.c_int, C.c_double]
        L.orc_lagrange_block_err.restype = C.c_double
        L.orc_gauss_legendre.argtypes = [C.c_int, _dp, _dp]
        L.orc_pw_rank.argtypes = [C.c_double, C.c_double, C.c_double]
        L.orc_pw_rank.restype = C.c_int
        L.orc_sphere_quad.argtypes = [C.c_int, _dp, _dp]
        L.orc_hankel.argtypes = [C.c_int, C.c_double, _dp, _dp]
        L.orc_gegenbauer.argtypes = [C.c_double, _dp, C.c_int, _dp, _dp, _dp]
        L.orc_nu_params.argtypes = [C.c_double, C.c_double, C.c_double, C.POINTER(C.c_int), _dp,
                                    C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.orc_nu_init.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, _dp, C.c_int]
        L.orc_nu_init.restype = C.c_int
        L.orc_nu_free.argtypes = [C.c_void_p]
        L.orc_nu_forward.argtypes = [C.c_void_p, _dp, C.c_int64, _dp, _dp, _dp, _dp]
        L.orc_nu_adjoint.argtypes = [C.c_void_p, _dp, C.c_int64, _dp, _dp, _dp, _dp]
        L.orc_es_kernel.argtypes = [C.c_double, C.c_double]
        L.orc_es_kernel.restype = C.c_double
        L.orc_es_hat.argtypes = [C.c_double, C.c_double]
        L.orc_es_hat.restype = C.c_double
        L.orc_dft3.argtypes = [C.c_int, _dp, _dp, C.c_int]
        L.orc_pw_pair.argtypes = [C.c_double, C.c_int, _dp, _dp, _dp, _dp, _dp, _dp]
        L.orc_kernel_eval.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, _dp, _dp]
        L.orc_direct_dl.argtypes = [_dp, C.c_int64, _dp, C.c_int64, _dp, _dp, _dp, C.c_int, _i64p, C.c_int64, _dp]
        L.orc_direct_dl.restype = C.c_int
        L.orc_apply_dl.argtypes = [C.c_void_p, _dp, _dp, _dp, C.c_int, _dp]
        L.orc_apply_dl.restype = C.c_int
        L.orc_direct_grad.argtypes = [_dp, C.c_int64, _dp, C.c_int64, _dp, _dp, C.c_int, _i64p, C.c_int64, _dp]
        L.orc_direct_grad.restype = C.c_int
        L.orc_apply_grad.argtypes = [C.c_void_p, _dp, _dp, C.c_int, _dp]
        L.orc_apply_grad.restype = C.c_int
        L.orc_nthreads.restype = C.c_int
        L.orc_set_threads.argtypes = [C.c_int]
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _split_u(u):
    """u as (ny, nrhs) or (ny,) real/complex -> Fortran-ordered re, im (or None), nrhs."""
    u = np.asarray(u)
    if u.ndim == 1:
        u = u[:, None]
    nrhs = u.shape[1]
    re = np.asfortranarray(u.real, dtype=np.float64)
    im = np.asfortranarray(u.imag, dtype=np.float64) if np.iscomplexobj(u) else None
    return re, im, nrhs


def nthreads():
    return lib().orc_nthreads()


def set_threads(n):
    lib().orc_set_threads(int(n))


def direct(X, Y, u, kind, k=0.0, w=None, targets=None):
    """O1: v_i = sum_j w_j G(x_i - y_j) u_j in FP64 (complex128 result, shape (n, nrhs))."""
    X = _c64(X).reshape(-1, 3)
    Y = _c64(Y).reshape(-1, 3)
    re, im, nrhs = _split_u(u)
    w = None if w is None else _c64(w)
    if targets is None:
        tsel, nt = None, X.shape[0]
    else:
        tsel = np.ascontiguousarray(targets, dtype=np.int64)
        nt = tsel.shape[0]
    vr = np.zeros((nt, nrhs), order="F")
    vi = np.zeros((nt, nrhs), order="F")
    rc = lib().orc_direct(_d(X), X.shape[0], _d(Y), Y.shape[0], _d(w), _d(re), _d(im), nrhs, kind, float(k),
                          tsel.ctypes.data_as(_i64p) if tsel is not None else None, nt, _d(vr), _d(vi))
    if rc:
        raise ValueError("orc_direct failed: %d" % rc)
    return vr + 1j * vi


def default_opts(**kw):
    o = Opts()
    lib().orc_default_opts(C.byref(o))
    for k_, v_ in kw.items():
        setattr(o, k_, v_)
    return o


class Plan:
    """O2: the plain CPU FFM plan (trees and pair lists) and its apply."""

    def __init__(self, X, Y, kind, k=0.0, eps=1e-3, **opts):
        self.X = _c64(X).reshape(-1, 3)
        self.Y = _c64(Y).reshape(-1, 3)
        self.nx, self.ny = self.X.shape[0], self.Y.shape[0]
        o = default_opts(**opts)
        self._h = lib().orc_plan_create(_d(self.X), self.nx, _d(self.Y), self.ny, kind, float(k), float(eps),
                                        C.byref(o))
        if not self._h:
            raise ValueError("orc_plan_create rejected its arguments")

    def close(self):
        if getattr(self, "_h", None):
            lib().orc_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def stats(self):
        s = Stats()
        lib().orc_plan_stats(self._h, C.byref(s))
        return s.as_dict()

    def pairs(self, level, which):
        """which 'adm' (admissible pairs at level) or 'near' (near pairs at the stop level):
        (n, 2) uint64 array of (X box id, Y box id), Morton ids at that level."""
        w = 0 if which == "adm" else 1
        n = lib().orc_plan_pairs(self._h, level, w, None, None)
        a = np.zeros(n, np.uint64)
        b = np.zeros(n, np.uint64)
        if n:
            lib().orc_plan_pairs(self._h, level, w, a.ctypes.data_as(_u64p), b.ctypes.data_as(_u64p))
        return np.stack([a, b], 1)

    def perm(self, which):
        n = self.nx if which == "X" else self.ny
        out = np.zeros(n, np.int64)
        lib().orc_plan_perm(self._h, 0 if which == "X" else 1, out.ctypes.data_as(_i64p))
        return out

    def apply_dl(self, u, nrm, w=None):
        """Double-layer product (plan built with kind LAPLACE_DL): real u, source normals nrm."""
        re, _, nrhs = _split_u(u)
        nrm = _c64(nrm).reshape(-1, 3)
        w = None if w is None else _c64(w)
        v = np.zeros((self.nx, nrhs), order="F")
        rc = lib().orc_apply_dl(self._h, _d(nrm), _d(w), _d(re), nrhs, _d(v))
        if rc:
            raise ValueError("orc_apply_dl failed: %d" % rc)
        return v

    def apply_grad(self, u, w=None):
        """Gradient product (plan built with kind LAPLACE_GRAD): real u; returns (nx, nrhs, 3)."""
        re, _, nrhs = _split_u(u)
        w = None if w is None else _c64(w)
        v = np.zeros((self.nx, 3 * nrhs), order="F")
        rc = lib().orc_apply_grad(self._h, _d(w), _d(re), nrhs, _d(v))
        if rc:
            raise ValueError("orc_apply_grad failed: %d" % rc)
        return v.reshape(self.nx, nrhs, 3)

    def apply(self, u, w=None):
        re, im, nrhs = _split_u(u)
        w = None if w is None else _c64(w)
        vr = np.zeros((self.nx, nrhs), order="F")
        vi = np.zeros((self.nx, nrhs), order="F")
        rc = lib().orc_apply(self._h, _d(w), _d(re), _d(im), nrhs, _d(vr), _d(vi))
        if rc:
            raise ValueError("orc_apply failed: %d" % rc)
        return vr + 1j * vi


def direct_dl(X, Y, nrm, u, w=None, targets=None):
    """O1 for the double layer: v_i = sum_j w_j u_j n_j.(x_i - y_j) / (4 pi |x_i - y_j|^3),
    real, shape (n, nrhs)."""
    X = _c64(X).reshape(-1, 3)
    Y = _c64(Y).reshape(-1, 3)
    nrm = _c64(nrm).reshape(-1, 3)
    re, _, nrhs = _split_u(u)
    w = None if w is None else _c64(w)
    if targets is None:
        tsel, nt = None, X.shape[0]
    else:
        tsel = np.ascontiguousarray(targets, dtype=np.int64)
        nt = tsel.shape[0]
    v = np.zeros((nt, nrhs), order="F")
    rc = lib().orc_direct_dl(_d(X), X.shape[0], _d(Y), Y.shape[0], _d(nrm), _d(w), _d(re), nrhs,
                             tsel.ctypes.data_as(_i64p) if tsel is not None else None, nt, _d(v))
    if rc:
        raise ValueError("orc_direct_dl failed: %d" % rc)
    return v


def ffm_dl(X, Y, nrm, u, eps=1e-3, w=None, **opts):
    p = Plan(X, Y, LAPLACE_DL, 0.0, eps, **opts)
    try:
        return p.apply_dl(u, nrm, w)
    finally:
        p.close()


def ffm(X, Y, u, kind, k=0.0, eps=1e-3, w=None, **opts):
    p = Plan(X, Y, kind, k, eps, **opts)
    try:
        return p.apply(u, w)
    finally:
        p.close()


def admissible(sigma, level, m):
    s = _c64(sigma)
    mm = np.ascontiguousarray(m, dtype=np.int64)
    return bool(lib().orc_admissible(_d(s), int(level), mm.ctypes.data_as(_i64p)))


def morton(gx, gy, gz):
    return int(lib().orc_morton(gx, gy, gz))


def r1_rule(kind, eps):
    return int(lib().orc_r1_rule(kind, float(eps)))


def aca(M, tol, kmax=None):
    """ACA with partial pivoting of a real matrix M (eq. 11): (A, B) with M ~ A @ B.T,
    A: nr x k, B: nc x k."""
    M = np.ascontiguousarray(M, dtype=np.float64)
    nr, nc = M.shape
    kmax = min(nr, nc) if kmax is None else int(kmax)
    A = np.zeros((kmax, nr))
    B = np.zeros((kmax, nc))
    k = int(lib().orc_aca(_d(M), nr, nc, float(tol), kmax, _d(A), _d(B)))
    return A[:k].T.copy(), B[:k].T.copy()


def r1_table(kind):
    out = np.zeros(11)
    lib().orc_r1_table(kind, _d(out))
    return out


def lagrange_block_err(kind, k, r1, d=1.0):
    return float(lib().orc_lagrange_block_err(kind, float(k), int(r1), float(d)))


def gauss_legendre(n):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().orc_gauss_legendre(n, _d(x), _d(w))
    return x, w


def pw_rank(k, dl, eps):
    return int(lib().orc_pw_rank(float(k), float(dl), float(eps)))


def sphere_quad(L):
    nq = 2 * L * (L + 1)
    s = np.zeros((nq, 3))
    w = np.zeros(nq)
    lib().orc_sphere_quad(L, _d(s), _d(w))
    return s, w


def hankel(L, z):
    hr = np.zeros(L + 1)
    hi = np.zeros(L + 1)
    lib().orc_hankel(L, float(z), _d(hr), _d(hi))
    return hr + 1j * hi


def gegenbauer(k, r0, L, s):
    r0 = _c64(r0)
    s = _c64(s)
    tr = C.c_double()
    ti = C.c_double()
    lib().orc_gegenbauer(float(k), _d(r0), int(L), _d(s), C.byref(tr), C.byref(ti))
    return tr.value + 1j * ti.value


def pw_pair(k, L, x, y, x0, y0):
    gr = C.c_double()
    gi = C.c_double()
    lib().orc_pw_pair(float(k), int(L), _d(_c64(x)), _d(_c64(y)), _d(_c64(x0)), _d(_c64(y0)), C.byref(gr),
                      C.byref(gi))
    return gr.value + 1j * gi.value


def kernel(kind, k, d):
    gr = C.c_double()
    gi = C.c_double()
    lib().orc_kernel_eval(kind, float(k), float(d[0]), float(d[1]), float(d[2]), C.byref(gr), C.byref(gi))
    return gr.value + 1j * gi.value


def rel_l2(v, ref):
    v = np.asarray(v)
    ref = np.asarray(ref)
    return float(np.linalg.norm((v - ref).ravel()) / np.linalg.norm(ref.ravel()))


if os.environ.get("FFM_ORACLE_THREADS"):
    set_threads(int(os.environ["FFM_ORACLE_THREADS"]))


# ---------------------------------------------------------------- type-3 NUFFT (Sec. 2.2.3)

class _Nu(C.Structure):
    _fields_ = [("w", C.c_int), ("beta", C.c_double), ("M", C.c_int), ("h", C.c_double), ("n1", C.c_int),
                ("n2", C.c_int), ("nq", C.c_int), ("s", _dp), ("corr", _dp), ("cinv", _dp)]


def nufft_params(d, k, eps):
    """(w, beta, M, n1, n2) of the NUFFT reading for a box of edge d at wavenumber k."""
    w, M, n1, n2 = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    beta = C.c_double()
    lib().orc_nu_params(float(d), float(k), float(eps), C.byref(w), C.byref(beta), C.byref(M), C.byref(n1),
                        C.byref(n2))
    return w.value, beta.value, M.value, n1.value, n2.value


class Nufft:
    """Type-3 NUFFT of one box: forward F_q = sum_j c_j e^{-i s_q.x_j} and its adjoint
    v_j = sum_q z_q e^{+i s_q.x_j}; x box-centred in [-d/2, d/2]^3, s = k shat."""

    def __init__(self, d, k, eps, s):
        self.s = _c64(s).reshape(-1, 3)
        self._nu = _Nu()
        if lib().orc_nu_init(C.byref(self._nu), float(d), float(k), float(eps), _d(self.s), self.s.shape[0]):
            raise MemoryError("orc_nu_init")

    def close(self):
        if getattr(self, "_nu", None) is not None:
            lib().orc_nu_free(C.byref(self._nu))
            self._nu = None

    def __del__(self):
        self.close()

    @property
    def params(self):
        return dict(w=self._nu.w, beta=self._nu.beta, M=self._nu.M, h=self._nu.h, n1=self._nu.n1, n2=self._nu.n2)

    def forward(self, x, c):
        x = _c64(x).reshape(-1, 3)
        c = np.asarray(c, np.complex128)
        cr, ci = _c64(c.real), _c64(c.imag)
        nq = self.s.shape[0]
        Fr, Fi = np.zeros(nq), np.zeros(nq)
        lib().orc_nu_forward(C.byref(self._nu), _d(x), x.shape[0], _d(cr), _d(ci), _d(Fr), _d(Fi))
        return Fr + 1j * Fi

    def adjoint(self, x, z):
        x = _c64(x).reshape(-1, 3)
        z = np.asarray(z, np.complex128)
        zr, zi = _c64(z.real), _c64(z.imag)
        vr, vi = np.zeros(x.shape[0]), np.zeros(x.shape[0])
        lib().orc_nu_adjoint(C.byref(self._nu), _d(x), x.shape[0], _d(zr), _d(zi), _d(vr), _d(vi))
        return vr + 1j * vi


def es_kernel(z, beta):
    return lib().orc_es_kernel(float(z), float(beta))


def es_hat(xi, beta):
    return lib().orc_es_hat(float(xi), float(beta))


def dft3(a, sign):
    """The oracle's 3-D DFT of an n^3 complex array, sum_j a_j e^{sign 2 pi i j.k / n}."""
    a = np.asarray(a, np.complex128)
    n = a.shape[0]
    re, im = _c64(a.real.ravel()), _c64(a.imag.ravel())
    lib().orc_dft3(n, _d(re), _d(im), int(sign))
    return (re + 1j * im).reshape(a.shape)


def ffm_nufft(X, Y, u, kind, k, eps, w=None, **opts):
    """O2 with the plane-wave steps computed by the type-3 NUFFT."""
    with_p = Plan(X, Y, kind, k, eps, pw_transform=1, **opts)
    try:
        return with_p.apply(u, w=w)
    finally:
        with_p.close()


def direct_grad(X, Y, u, w=None, targets=None):
    """O1 for the gradient of the single layer in the target variable:
    v_i = sum_j w_j u_j grad_x G(x_i - y_j), shape (n, nrhs, 3)."""
    X = _c64(X).reshape(-1, 3)
    Y = _c64(Y).reshape(-1, 3)
    re, _, nrhs = _split_u(u)
    w = None if w is None else _c64(w)
    if targets is None:
        tsel, nt = None, X.shape[0]
    else:
        tsel = np.ascontiguousarray(targets, dtype=np.int64)
        nt = tsel.shape[0]
    v = np.zeros((nt, 3 * nrhs), order="F")
    rc = lib().orc_direct_grad(_d(X), X.shape[0], _d(Y), Y.shape[0], _d(w), _d(re), nrhs,
                               tsel.ctypes.data_as(_i64p) if tsel is not None else None, nt, _d(v))
    if rc:
        raise ValueError("orc_direct_grad failed: %d" % rc)
    return v.reshape(nt, nrhs, 3)


def ffm_grad(X, Y, u, eps=1e-3, w=None, **opts):
    """O2 for the gradient: Lagrange levels with the three component kernels dG/dx_d."""
    p = Plan(X, Y, LAPLACE_GRAD, 0.0, eps, **opts)
    try:
        return p.apply_grad(u, w=w)
    finally:
        p.close()
