"""CPU checks of the arithmetic the mixed-precision pressure solve relies on
(no GPU; numpy restatements of the schemes, not of the kernels' code):

* the even/odd form of the Hartley transform of a row, with the tile
  pipeline's block pairing (stage j holds K blocks j and n/16 - 1 - j, the
  mirror of a block's first value carried from the previous stage, x[n/2]
  and the alternating sum kept per row), against the direct product x H;
* the double-single (FP32 pair) evaluation of the Poisson residual
  r = D - L_h phi, emulated in float32 with Knuth's TwoSum and the exact
  FMA product, against the FP64 evaluation rounded to FP32: identical where
  1/h^2 is a power of two, within one unit in the last place otherwise, on
  fields whose residual is 1e-6 of the stencil's terms;
* the refinement with a bfloat16 correction: an FP32 predictor solve, the
  residual in FP64 (which the double-single evaluation matches to an ulp),
  the correction solve with every transform operand and pass output rounded
  to bfloat16 (FP32 accumulation), summed: the predictor's error shrinks by
  the correction's relative error (about 2^-7 here), far below FP32
  rounding of the result.
"""
import numpy as np
import pytest

F32 = np.float32


def _hartley(n):
    k = np.arange(n)
    a = 2 * np.pi * np.outer(k, k) / n
    return np.cos(a) + np.sin(a)


def _even_odd_rows(X):
    """Row transforms of X (rows x n) by the stage pairing of the even/odd
    tensor-core form."""
    rows, n = X.shape
    m, NB, NS = n // 2, n // 16, n // 32
    kk = np.arange(m)
    Bc = np.cos(2 * np.pi * np.outer(kk, kk) / n)
    Bs = np.sin(2 * np.pi * np.outer(kk, kk) / n)
    C = np.zeros((rows, m))
    S = np.zeros((rows, m))
    carry = np.zeros(rows)
    alt = np.zeros(rows)
    xm = None
    for j in range(NS):
        a = X[:, 16 * j:16 * j + 16]
        b = X[:, 16 * (NB - 1 - j):16 * (NB - j)]
        e = np.empty((rows, 16))
        o = np.empty((rows, 16))
        e[:, 0] = a[:, 0] if j == 0 else a[:, 0] + carry
        o[:, 0] = 0.0 if j == 0 else a[:, 0] - carry
        for q in range(1, 16):
            e[:, q] = a[:, q] + b[:, 16 - q]
            o[:, q] = a[:, q] - b[:, 16 - q]
        carry = b[:, 0].copy()
        alt += ((a + b) * (-1.0) ** np.arange(16)).sum(axis=1)
        if j == NS - 1:
            xm = b[:, 0].copy()
        C += e @ Bc[16 * j:16 * j + 16]
        S += o @ Bs[16 * j:16 * j + 16]
    y = np.empty((rows, n))
    sgn = (-1.0) ** np.arange(m)
    y[:, :m] = C + S + xm[:, None] * sgn
    y[:, n - np.arange(1, m)] = (C - S + xm[:, None] * sgn)[:, 1:]
    y[:, m] = alt
    return y


@pytest.mark.parametrize("n", [32, 64, 128, 256])
def test_even_odd_form_equals_the_hartley_product(n):
    X = np.random.default_rng(n).standard_normal((128, n))
    ref = X @ _hartley(n)
    assert np.max(np.abs(_even_odd_rows(X) - ref)) < 1e-11 * np.max(np.abs(ref))


def _two_sum(a, b):
    s = (a + b).astype(F32)
    bb = (s - a).astype(F32)
    e = ((a - (s - bb).astype(F32)).astype(F32) + (b - bb).astype(F32)).astype(F32)
    return s, e


def _fma32(a, b, c):
    # float32 operands: the product is exact in float64 and the sum of two
    # float64 values is rounded once more to float32 (double rounding can
    # differ from a fused operation only at ties, absent in these data)
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(F32)


def _residual_ds(phi, D, ih2):
    hi = F32(ih2)
    lo = F32(ih2 - float(hi))
    pad = np.concatenate([phi[:1], phi, phi[-1:]], 0)   # Neumann ends in x
    pxm, pxp = pad[:-2], pad[2:]
    pym, pyp = np.roll(phi, 1, 1), np.roll(phi, -1, 1)
    pzm, pzp = np.roll(phi, 1, 2), np.roll(phi, -1, 2)
    s1, s2, s3 = _two_sum(pxm, pxp), _two_sum(pym, pyp), _two_sum(pzm, pzp)
    s4 = _two_sum(s1[0], s2[0])
    s5 = _two_sum(s4[0], s3[0])
    p6 = (F32(6) * phi).astype(F32)
    q6 = _fma32(np.full_like(phi, 6), phi, -p6)
    s6 = _two_sum(s5[0], -p6)
    low = ((((s1[1] + s2[1]).astype(F32) + (s3[1] + s4[1]).astype(F32)).astype(F32)
            + (s5[1] + s6[1]).astype(F32)).astype(F32) - q6).astype(F32)
    Sh, Sl = _two_sum(s6[0], low)
    ph = (Sh * hi).astype(F32)
    pe = (_fma32(Sh, np.full_like(phi, hi), -ph)
          + ((Sh * lo).astype(F32) + (Sl * hi).astype(F32)).astype(F32)).astype(F32)
    lap_h, lap_l = _two_sum(ph, pe)
    t_h, t_l = _two_sum(D, -lap_h)
    return (t_h + (t_l - lap_l).astype(F32)).astype(F32)


@pytest.mark.parametrize("h,exact", [(1 / 64, True), (0.0371, False)])
def test_double_single_residual_matches_fp64(h, exact):
    rng = np.random.default_rng(3)
    phi = (rng.standard_normal((6, 8, 16)) * 3 + 50).astype(F32)
    ih2 = 1.0 / (h * h)
    pad = np.concatenate([phi[:1], phi, phi[-1:]], 0).astype(np.float64)
    p64 = phi.astype(np.float64)
    lap64 = (pad[:-2] + pad[2:] + np.roll(p64, 1, 1) + np.roll(p64, -1, 1) + np.roll(p64, 1, 2)
             + np.roll(p64, -1, 2) - 6.0 * p64) * ih2
    # D close to L phi: the residual is 1e-6 of the terms (the refinement's case)
    D = (lap64 * (1 + 1e-6 * rng.standard_normal(lap64.shape))).astype(F32)
    ref = (D.astype(np.float64) - lap64).astype(F32)
    r = _residual_ds(phi, D, ih2)
    ulps = np.abs(r.astype(np.float64) - ref) / np.spacing(np.abs(ref)).astype(np.float64)
    if exact:
        assert np.array_equal(r, ref)
    else:
        assert np.max(ulps) <= 1.0
    # a plain FP32 evaluation loses the residual entirely at this cancellation
    r32 = (D - ((pad[:-2] + pad[2:]).astype(F32) + np.roll(phi, 1, 1) + np.roll(phi, -1, 1)
                + np.roll(phi, 1, 2) + np.roll(phi, -1, 2) - F32(6) * phi) * F32(ih2)).astype(F32)
    assert np.max(np.abs(r32.astype(np.float64) - ref)) > 100 * np.max(np.abs(r.astype(np.float64) - ref))


def _bf16(a):
    """Round to bfloat16 (nearest, ties to even), returned as float32."""
    b = np.asarray(a, dtype=F32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(F32)


def _x_solve(Dh, h):
    """Per transverse mode the Neumann x solve of the Hartley-transformed
    Poisson equation (mode (0, 0) pinned and its mean removed), in FP64."""
    nx, ny, nz = Dh.shape
    out = np.empty(Dh.shape)
    for j in range(ny):
        for k in range(nz):
            lam = -4 * np.sin(np.pi * j / ny) ** 2 - 4 * np.sin(np.pi * k / nz) ** 2
            A = np.diag(np.full(nx, -2.0 + lam)) + np.diag(np.ones(nx - 1), 1) + np.diag(np.ones(nx - 1), -1)
            A[0, 0] += 1.0
            A[-1, -1] += 1.0
            b = h * h * Dh[:, j, k].astype(np.float64) / (ny * nz)
            if j == 0 and k == 0:
                A[0, :] = 0.0
                A[0, 0] = 1.0
                b[0] = 0.0
                x = np.linalg.solve(A, b)
                out[:, j, k] = x - x.mean()
            else:
                out[:, j, k] = np.linalg.solve(A, b)
    return out


def _transform2d(X, dtype, rnd=None):
    n = X.shape[1]
    r = rnd or (lambda a: a.astype(dtype))
    H = r(_hartley(n))
    T = r(np.einsum("iyz,zk->iyk", r(X), H, dtype=dtype))
    return r(np.einsum("yj,ijk->iyk", H, T, dtype=dtype))


def _laplacian(p, h):
    pad = np.concatenate([p[:1], p, p[-1:]], 0)
    return (pad[:-2] + pad[2:] + np.roll(p, 1, 1) + np.roll(p, -1, 1) + np.roll(p, 1, 2) + np.roll(p, -1, 2)
            - 6.0 * p) / (h * h)


def test_bfloat16_correction_refines_the_fp32_predictor():
    rng = np.random.default_rng(0)
    nx, n, h = 24, 16, 1.0 / 16
    D = rng.standard_normal((nx, n, n))
    D -= D.mean()
    exact = _transform2d(_x_solve(_transform2d(D, np.float64), h), np.float64)
    x0 = _transform2d(_x_solve(_transform2d(D.astype(F32), F32), h).astype(F32), F32).astype(np.float64)
    r1 = D - _laplacian(x0, h)
    t1 = _transform2d(_x_solve(_transform2d(_bf16(r1), F32, _bf16), h).astype(F32), F32, _bf16)
    p = x0 + _bf16(t1).astype(np.float64)
    scale = np.abs(exact).max()
    e0 = np.abs(x0 - exact).max() / scale
    e1 = np.abs(p - exact).max() / scale
    assert 1e-8 < e0 < 1e-5          # an FP32 solve
    assert e1 < e0 / 30 and e1 < 1e-8
