"""FP64 CPU oracle of the boundary-element wrapper (test infrastructure only).

Sec. 4.2 writes the Galerkin matrix of a boundary integral operator as
S = (Lambda*)^T (G Lambda): Lambda carries the basis functions to the quadrature nodes,
(Lambda*)^T brings the weighted node values back to the test functions, and G is the dense
kernel matrix between quadrature nodes, which the FFM applies.  The singular integrals
that the node quadrature misses are handled by an extra sparse matrix.  This module is the
plain version for P1 (piecewise-linear nodal) functions on flat triangles and the Laplace
single layer G = 1/(4 pi |x - y|):
  - 3-point quadrature per triangle, nodes at barycentric (2/3, 1/6, 1/6) and permutations,
    weights area / 3; pairs of coincident nodes are skipped (as in the FFM);
  - the correction of each triangle's self-interaction: its exact element matrix
    A_ab = int_T phi_a(x) int_T phi_b(y) G(x, y) dy dx (inner integral in closed form, the
    potential of a linear density on a flat triangle at a point of its plane; outer by a
    collapsed Gauss rule) minus what the node quadrature gives for it.
Nothing here is shared with the CUDA path; only tests may import it.
"""
import numpy as np

from . import oracle as O

BARY = np.array([[2.0 / 3, 1.0 / 6, 1.0 / 6], [1.0 / 6, 2.0 / 3, 1.0 / 6], [1.0 / 6, 1.0 / 6, 2.0 / 3]])


def quadrature(V, F):
    """Quadrature nodes (3 nt, 3), weights (3 nt,), and Lambda as a dense (3 nt, nv) matrix."""
    P = V[F]
    area = 0.5 * np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1)
    X = np.einsum('qk,tkd->tqd', BARY, P).reshape(-1, 3)
    w = np.repeat(area / 3.0, 3)
    L = np.zeros((3 * len(F), len(V)))
    for q in range(3):
        for k in range(3):
            np.add.at(L, (np.arange(len(F)) * 3 + q, F[:, k]), BARY[q, k])
    return X, w, L


def _gauss01(n):
    t, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (t + 1.0), 0.5 * w


def plane_integrals(P, x):
    """For points x (..., 3) inside flat triangles P (..., 3, 3): V0 = int_T dA / |y - x| and
    the vector Vv = int_T (y - x) / |y - x| dA, edge by edge in polar coordinates about x: an
    edge at distance d with end-point coordinates s-, s+ along it (distances R-, R+)
    contributes d ln((s+ + R+) / (s- + R-)) to V0 and d [n (atan(s+/d) - atan(s-/d)) +
    t ln(R+/R-)] to Vv, with n the unit normal towards the edge and t the edge direction."""
    V0 = 0.0
    Vv = 0.0
    for i in range(3):
        a, b = P[..., i, :], P[..., (i + 1) % 3, :]
        t = (b - a) / np.linalg.norm(b - a, axis=-1, keepdims=True)
        foot = a + np.sum((x - a) * t, axis=-1, keepdims=True) * t
        n = foot - x
        d = np.linalg.norm(n, axis=-1, keepdims=True)
        n = n / d
        sa = np.sum((a - foot) * t, axis=-1, keepdims=True)
        sb = np.sum((b - foot) * t, axis=-1, keepdims=True)
        ra = np.linalg.norm(x - a, axis=-1, keepdims=True)
        rb = np.linalg.norm(x - b, axis=-1, keepdims=True)
        V0 = V0 + (d * np.log((sb + rb) / (sa + ra)))[..., 0]
        Vv = Vv + d * (n * (np.arctan(sb / d) - np.arctan(sa / d)) + t * np.log(rb / ra))
    return V0, Vv


def self_element(P, n_outer=32):
    """Exact element matrices (nt, 3, 3) of the single layer on each triangle of P (nt, 3, 3):
    A_ab = int_T phi_a(x) int_T phi_b(y) / (4 pi |x - y|) dy dx, the inner integral in closed
    form (phi_b(y) = phi_b(x) + grad phi_b . (y - x)), the outer one by a collapsed Gauss rule
    x = p0 + u (p1 - p0) + u v (p2 - p1), dx = 2 area u du dv."""
    ot, ow = _gauss01(n_outer)
    U, Vv = np.meshgrid(ot, ot, indexing='ij')
    WU = np.outer(ow, ow)
    U, Vv, WU = U.ravel(), Vv.ravel(), WU.ravel()
    lam = np.stack([1 - U, U * (1 - Vv), U * Vv], 1)  # (no, 3)
    out = np.zeros((P.shape[0], 3, 3))
    for c0 in range(0, P.shape[0], 256):
        T = P[c0:c0 + 256]
        e1, e2 = T[:, 1] - T[:, 0], T[:, 2] - T[:, 0]
        nrm = np.cross(e1, e2)
        area2 = np.linalg.norm(nrm, axis=1)
        # gradients of the barycentric coordinates, constant on each triangle
        grads = np.stack([np.cross(nrm, T[:, 2] - T[:, 1]), np.cross(nrm, T[:, 0] - T[:, 2]),
                          np.cross(nrm, T[:, 1] - T[:, 0])], 1) / (area2 ** 2)[:, None, None]
        X = np.einsum('ok,tkd->tod', lam, T)
        V0, Vvec = plane_integrals(T[:, None], X)  # (nt, no), (nt, no, 3)
        inner = (lam[None] * V0[..., None] + np.einsum('tbd,tod->tob', grads, Vvec)) / (4 * np.pi)
        out[c0:c0 + 256] = np.einsum('o,ok,tob->tkb', WU * U, lam, inner) * area2[:, None, None]
    return out


def node_element(P):
    """What the node quadrature gives for each triangle's self-interaction (nt, 3, 3)."""
    area = 0.5 * np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1)
    Xq = np.einsum('qk,tkd->tqd', BARY, P)
    d = np.linalg.norm(Xq[:, :, None, :] - Xq[:, None, :, :], axis=3)
    G = np.where(d > 0, 1.0 / (4 * np.pi * np.where(d > 0, d, 1.0)), 0.0)
    w = (area / 3.0)[:, None]
    return np.einsum('qa,tqr,rb->tab', BARY, G * w[:, :, None] * w[:, None, :], BARY)


def correction(V, F):
    """Sparse correction as a dense (nv, nv) matrix: sum over triangles of (exact - node)."""
    P = V[F]
    Cl = self_element(P) - node_element(P)
    C = np.zeros((len(V), len(V)))
    for a in range(3):
        for b in range(3):
            np.add.at(C, (F[:, a], F[:, b]), Cl[:, a, b])
    return C


def dense_matrix(V, F):
    """S = (Lambda*)^T G W Lambda + C with the dense kernel matrix (small meshes)."""
    X, w, L = quadrature(V, F)
    r = np.linalg.norm(X[:, None, :] - X[None, :, :], axis=2)
    np.fill_diagonal(r, np.inf)
    G = 1.0 / (4 * np.pi * r)
    return L.T @ (w[:, None] * G * w[None, :]) @ L + correction(V, F)


def apply_ffm(V, F, u, eps, C=None):
    """S u with the oracle's plain CPU FFM (O2) in the middle."""
    X, w, L = quadrature(V, F)
    if C is None:
        C = correction(V, F)
    g = O.ffm(X, X, L @ u, O.LAPLACE, 0.0, eps, w=w)[:, 0].real
    return L.T @ (w * g) + C @ u
