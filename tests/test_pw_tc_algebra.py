"""The real-GEMM forms that the tensor-core plane-wave transforms compute (k_pw_forward_tc,
k_pw_backward_tc), checked on the CPU against the complex sums they replace.

Forward (source box): u~(h) = sum_j e_hj w_j and u~(h + nQ/2) = sum_j conj(e_hj) w_j, with
e_hj = F(h) e^{-i ph_hj}.  The kernel forms P = sum_j Re(e_hj) w_j and Q = sum_j Im(e_hj) w_j
as real GEMMs over (re, im) columns and returns P + iQ and P - iQ.

Backward (target box): v_x = sum_h g_xh a_h + conj(g_xh) b_h, g_xh = e^{i ph_xh} conj(F(h)),
a = v~(h), b = v~(h + nQ/2).  The kernel's K index runs over (h, Re g | Im g) and its B operand
holds S = a + b and D = a - b as rows (Re S, Im S) and (-Im D, Re D)."""
import numpy as np


def _rng():
    return np.random.default_rng(11)


def test_forward_pair_form_matches_the_complex_sums():
    rng = _rng()
    nh, nj, nrhs = 7, 13, 5
    ph = rng.uniform(-20, 20, (nh, nj))
    F = np.exp(1j * rng.uniform(0, 2 * np.pi, nh))
    w = rng.normal(size=(nj, nrhs)) + 1j * rng.normal(size=(nj, nrhs))
    e = F[:, None] * np.exp(-1j * ph)
    u_h = e @ w
    u_b = np.conj(e) @ w
    # real GEMMs: columns (re, im) of each right-hand side
    W = np.stack([w.real, w.imag], axis=2).reshape(nj, 2 * nrhs)
    P = (e.real @ W).reshape(nh, nrhs, 2)
    Q = (e.imag @ W).reshape(nh, nrhs, 2)
    Pc = P[..., 0] + 1j * P[..., 1]
    Qc = Q[..., 0] + 1j * Q[..., 1]
    # the kernel's epilogue: (P.re - Q.im, P.im + Q.re) and (P.re + Q.im, P.im - Q.re)
    v = (Pc.real - Qc.imag) + 1j * (Pc.imag + Qc.real)
    vb = (Pc.real + Qc.imag) + 1j * (Pc.imag - Qc.real)
    assert np.allclose(v, u_h, rtol=0, atol=1e-12 * np.abs(u_h).max())
    assert np.allclose(vb, u_b, rtol=0, atol=1e-12 * np.abs(u_b).max())


def test_backward_image_rows_give_the_complex_sums():
    rng = _rng()
    nx, nh, nrhs = 9, 11, 4
    ph = rng.uniform(-20, 20, (nx, nh))
    F = np.exp(1j * rng.uniform(0, 2 * np.pi, nh))
    a = rng.normal(size=(nh, nrhs)) + 1j * rng.normal(size=(nh, nrhs))
    b = rng.normal(size=(nh, nrhs)) + 1j * rng.normal(size=(nh, nrhs))
    g = np.exp(1j * ph) * np.conj(F)[None, :]
    v = g @ a + np.conj(g) @ b
    # A[x, 2h + part]: part 0 = Re g, 1 = Im g.  B[2h + part, 2m + comp] as k_pw_vt_image writes it.
    A = np.stack([g.real, g.imag], axis=2).reshape(nx, 2 * nh)
    S, D = a + b, a - b
    B = np.zeros((2 * nh, 2 * nrhs))
    B[0::2, 0::2] = S.real
    B[0::2, 1::2] = S.imag
    B[1::2, 0::2] = -D.imag
    B[1::2, 1::2] = D.real
    out = (A @ B).reshape(nx, nrhs, 2)
    vk = out[..., 0] + 1j * out[..., 1]
    assert np.allclose(vk, v, rtol=0, atol=1e-12 * np.abs(v).max())


def test_tf32_three_product_split_error():
    # hi = x rounded to 10 stored mantissa bits, lo = x - hi rounded likewise (what the tensor core
    # reads): hi*hi + hi*lo + lo*hi is off by at most about 2^-21 of |x y| (2^-24.8 typically)
    rng = _rng()

    def tf32(v):
        m, e = np.frexp(v)
        return np.ldexp(np.round(m * 2.0 ** 11) / 2.0 ** 11, e)

    x = rng.normal(size=20000).astype(np.float32).astype(np.float64)
    y = rng.normal(size=20000).astype(np.float32).astype(np.float64)
    xh, yh = tf32(x), tf32(y)
    xl, yl = tf32(x - xh), tf32(y - yh)
    approx = xh * yh + xh * yl + xl * yh
    rel = np.abs(approx - x * y) / np.abs(x * y)
    assert rel.max() < 2.0 ** -20.5
    assert np.median(rel) < 2.0 ** -24
