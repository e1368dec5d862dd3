"""Recompute the Lagrange rank table (plan constant): for each r1 the relative error of
the tensor Chebyshev-Lagrange approximation of the kernel block between the closest
admissible box pair (centre offset 2 d along one axis), for the Laplace kernel, for
the Helmholtz kernel at k d = 2 (the oscillation switch) and for the Laplace double
layer (its component kernels dG/dy_d interpolated on their own, weighted by fixed unit
normals).  The plan picks the smallest r1 whose tabulated error is <= eps.  Calls only
the oracle.

Usage: python -m oracle.calibrate_r1
"""
import math

from . import oracle as O


def calibrate():
    rows = {}
    for name, kind, k in (("laplace", O.LAPLACE, 0.0), ("helmholtz_kd2", O.HELMHOLTZ, 2.0),
                          ("laplace_double_layer", O.LAPLACE_DL, 0.0)):
        rows[name] = [O.lagrange_block_err(kind, k, r1, 1.0) for r1 in range(2, 11)]
    return rows


def round_up(x, digits=2):
    e = math.floor(math.log10(x))
    m = x / 10 ** e
    return math.ceil(m * 10 ** (digits - 1) - 1e-9) / 10 ** (digits - 1) * 10 ** e


if __name__ == "__main__":
    for name, errs in calibrate().items():
        print(name, ", ".join("%.1e" % round_up(e) for e in errs))
