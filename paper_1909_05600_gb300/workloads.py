"""Seeded synthetic inputs shaped like the paper's workloads (numpy only).

This module holds no part of the method's arithmetic: it only draws point clouds,
weights and densities.  Both the CUDA path's tests/bench and the CPU oracle take their
inputs from here.  Seeds follow one convention: X from `seed`, Y from `seed + 1000`,
u from `seed + 2000`.

Shapes:
  * random points on the unit sphere (Sec. 4.1, the paper's scalability runs), drawn as
    normalised standard normal vectors;
  * uniform points on the surface of the unit cube [0,1]^3;
  * uniform points in the unit cube;
  * a mixture of 8 isotropic Gaussians (sigma = 0.05, centres uniform in [0,1]^3).
"""
from dataclasses import dataclass, field
import math

import numpy as np

LAPLACE, HELMHOLTZ, LAPLACE_DL, LAPLACE_GRAD = 0, 1, 2, 3


def sphere_surface(n, seed):
    p = np.random.default_rng(seed).standard_normal((n, 3))
    return p / np.linalg.norm(p, axis=1, keepdims=True)


def cube_surface(n, seed):
    rng = np.random.default_rng(seed)
    face = rng.integers(0, 6, n)
    a = rng.random((n, 2))
    p = np.empty((n, 3))
    axis = face % 3
    side = (face // 3).astype(np.float64)
    for d in range(3):
        on = axis == d
        others = [e for e in range(3) if e != d]
        p[on, d] = side[on]
        p[on, others[0]] = a[on, 0]
        p[on, others[1]] = a[on, 1]
    return p


def cube_volume(n, seed):
    return np.random.default_rng(seed).random((n, 3))


def gaussian_mixture(n, seed, centres_seed=7, ncomp=8, sigma=0.05):
    centres = np.random.default_rng(centres_seed).random((ncomp, 3))
    rng = np.random.default_rng(seed)
    comp = rng.integers(0, ncomp, n)
    return centres[comp] + sigma * rng.standard_normal((n, 3))


GEOMETRIES = {"sphere": sphere_surface, "cube_surface": cube_surface, "cube_volume": cube_volume}
AREA = {"sphere": 4.0 * math.pi, "cube_surface": 6.0, "cube_volume": 1.0}


def wavenumber_ppw(n, geometry, ppw=10.0):
    """k giving `ppw` points per wavelength: dx = sqrt(area/n) on a surface,
    (volume/n)^(1/3) in a volume, k = 2 pi / (ppw dx)."""
    if geometry == "cube_volume":
        dx = (1.0 / n) ** (1.0 / 3.0)
    else:
        dx = math.sqrt(AREA[geometry] / n)
    return 2.0 * math.pi / (ppw * dx)


@dataclass
class Problem:
    name: str
    X: np.ndarray
    Y: np.ndarray
    u: np.ndarray          # (ny,) or (ny, nrhs); float64/float32/complex64
    w: np.ndarray          # (ny,) quadrature weights
    kind: int
    k: float
    eps: float
    meta: dict = field(default_factory=dict)

    @property
    def n(self):
        return max(self.X.shape[0], self.Y.shape[0])


def laplace_sphere(n=20000, seed=1, eps=1e-3):
    """Laplace 1/(4 pi r), X and Y independent uniform draws on the unit sphere,
    w = 4 pi / n, u ~ N(0, 1) float64."""
    X = sphere_surface(n, seed)
    Y = sphere_surface(n, seed + 1000)
    u = np.random.default_rng(seed + 2000).standard_normal(n)
    w = np.full(n, 4.0 * math.pi / n)
    return Problem("laplace_sphere_%d" % n, X, Y, u, w, LAPLACE, 0.0, eps)


def laplace_double_layer_sphere(n=20000, seed=1, eps=1e-3):
    """Laplace double layer dG/dn_y on the unit sphere: X and Y independent uniform draws,
    outward normals n_y = y (kept in meta['normals']), w = 4 pi / n, u ~ N(0, 1)."""
    X = sphere_surface(n, seed)
    Y = sphere_surface(n, seed + 1000)
    u = np.random.default_rng(seed + 2000).standard_normal(n)
    w = np.full(n, 4.0 * math.pi / n)
    return Problem("laplace_dl_sphere_%d" % n, X, Y, u, w, LAPLACE_DL, 0.0, eps, meta={"normals": Y.copy()})


def laplace_gradient_sphere(n=20000, seed=1, eps=1e-3):
    """Gradient of the Laplace single layer (the MFIE kernel) on the unit sphere: X and Y
    independent uniform draws, w = 4 pi / n, u ~ N(0, 1); three outputs per target."""
    X = sphere_surface(n, seed)
    Y = sphere_surface(n, seed + 1000)
    u = np.random.default_rng(seed + 2000).standard_normal(n)
    w = np.full(n, 4.0 * math.pi / n)
    return Problem("laplace_grad_sphere_%d" % n, X, Y, u, w, LAPLACE_GRAD, 0.0, eps)


def helmholtz_sphere(n=1_000_000, seed=1, eps=1e-3, ppw=10.0):
    """Helmholtz e^{ikr}/(4 pi r), X and Y independent on the unit sphere, k at `ppw`
    points per wavelength, u complex64 with N(0,1) parts, w = 4 pi / n."""
    X = sphere_surface(n, seed)
    Y = sphere_surface(n, seed + 1000)
    rng = np.random.default_rng(seed + 2000)
    u = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    w = np.full(n, 4.0 * math.pi / n)
    k = wavenumber_ppw(n, "sphere", ppw)
    return Problem("helmholtz_sphere_%d" % n, X, Y, u, w, HELMHOLTZ, k, eps)


def helmholtz_cube_multirhs(n=200_000, nrhs=64, seed=1, eps=1e-4, ppw=10.0):
    """Helmholtz on the unit-cube surface with X = Y, nrhs plane-wave densities
    u_m(y) = e^{ik d_m . y} with directions d_m uniform on the sphere, complex64."""
    X = cube_surface(n, seed)
    k = wavenumber_ppw(n, "cube_surface", ppw)
    d = sphere_surface(nrhs, seed + 2000)
    u = np.exp(1j * k * (X @ d.T)).astype(np.complex64)
    w = np.full(n, 6.0 / n)
    return Problem("helmholtz_cube_%dx%d" % (n, nrhs), X, X.copy(), u, w, HELMHOLTZ, k, eps)


def laplace_clustered(n=100_000_000, seed=1, eps=1e-3):
    """Laplace on a mixture of 8 Gaussians (sigma 0.05, shared centres), X and Y
    independent float32 point sets, u ~ U(-1, 1) float32, w = 1/n (float32)."""
    X = gaussian_mixture(n, seed).astype(np.float32)
    Y = gaussian_mixture(n, seed + 1000).astype(np.float32)
    u = np.random.default_rng(seed + 2000).uniform(-1.0, 1.0, n).astype(np.float32)
    w = np.full(n, 1.0 / n, dtype=np.float32)
    return Problem("laplace_clustered_%d" % n, X, Y, u, w, LAPLACE, 0.0, eps)


def serving_stream(nreq=500, seed=7, nmin=10_000, nmax=2_000_000, rate_hz=10.0, scenes=0):
    """Request descriptors for the serving stream: Poisson arrivals, N log-uniform in
    [nmin, nmax], kernel 50/50, geometry uniform over three shapes, eps in {1e-3, 1e-4}.

    scenes = 0: every request has its own point sets.  scenes = S > 0: S scenes (point sets,
    kernel, k, eps) are drawn from the same distributions, and each request picks one of
    them uniformly with a density of its own, as when clients apply one operator to many
    right-hand sides; requests of one scene share a plan."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, nreq))
    nd = scenes if scenes > 0 else nreq
    ns = np.exp(rng.uniform(math.log(nmin), math.log(nmax), nd)).astype(np.int64)
    kinds = rng.integers(0, 2, nd)
    geos = rng.integers(0, 3, nd)
    epss = np.where(rng.integers(0, 2, nd) == 0, 1e-3, 1e-4)
    pick = rng.integers(0, nd, nreq) if scenes > 0 else np.arange(nreq)
    names = list(GEOMETRIES)
    out = []
    for i in range(nreq):
        c = int(pick[i])
        out.append({"id": i, "t_arrival": float(t[i]), "n": int(ns[c]), "kind": int(kinds[c]),
                    "geometry": names[geos[c]], "eps": float(epss[c]), "seed": int(seed * 100000 + c),
                    "scene": c, "useed": int(seed * 100000 + 50000 + i) if scenes > 0 else None})
    return out


def serving_points(req):
    """The point sets of a request's scene: X and Y drawn independently."""
    g = req["geometry"]
    return GEOMETRIES[g](req["n"], req["seed"]), GEOMETRIES[g](req["n"], req["seed"] + 1000)


def serving_problem(req, points=None):
    """Materialise one serving request (points: its scene's (X, Y) if already drawn)."""
    g = req["geometry"]
    n = req["n"]
    X, Y = points if points is not None else serving_points(req)
    rng = np.random.default_rng(req["useed"] if req.get("useed") is not None else req["seed"] + 2000)
    w = np.full(n, AREA[g] / n)
    if req["kind"] == LAPLACE:
        u = rng.standard_normal(n).astype(np.float32)
        return Problem("req%d" % req["id"], X, Y, u, w, LAPLACE, 0.0, req["eps"])
    u = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    k = wavenumber_ppw(n, g)
    return Problem("req%d" % req["id"], X, Y, u, w, HELMHOLTZ, k, req["eps"])


def sample_targets(nx, count=4096, seed=12345):
    """Seeded random subset of target indices for error measurement at large N."""
    if nx <= count:
        return np.arange(nx, dtype=np.int64)
    return np.sort(np.random.default_rng(seed).choice(nx, count, replace=False)).astype(np.int64)


def icosphere(level):
    """Triangle mesh of the unit sphere: the icosahedron with each face split into four
    `level` times, new vertices pushed to the sphere.  Returns vertices (nv, 3) FP64 and
    triangles (nt, 3) int32 (outward orientation)."""
    t = (1.0 + 5.0 ** 0.5) / 2.0
    V = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    F = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2),
         (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11),
         (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    V = [np.array(v, float) / np.linalg.norm(v) for v in V]
    for _ in range(level):
        mid = {}

        def m(a, b):
            key = (min(a, b), max(a, b))
            if key not in mid:
                p = V[a] + V[b]
                V.append(p / np.linalg.norm(p))
                mid[key] = len(V) - 1
            return mid[key]

        F2 = []
        for a, b, c in F:
            ab, bc, ca = m(a, b), m(b, c), m(c, a)
            F2 += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        F = F2
    return np.array(V), np.array(F, np.int32)
