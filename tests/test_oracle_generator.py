"""Pins of the inflow-generator oracle (CPU only).

* the periodic convolution against a brute-force loop with explicit modulo
  indices;
* its input adjoint and weight gradient through the identities
  <conv(W, X), G> = <X, conv_T(W, G)> = <W, dW(G, X)>;
* the whole network's gradient against central finite differences;
* bfloat16 rounding against hand-worked ties and torch's own conversion;
* Adam against its closed forms (first step, constant gradient);
* the rollout renormalisation (zero mean, target rms).
"""
import numpy as np
import pytest

from oracle import generator as gen
from paper_2103_08246_gb300 import inputs


def _brute_conv(W, X):
    ny, nz, C = X.shape
    O = W.shape[2]
    out = np.zeros((ny, nz, O))
    for y in range(ny):
        for z in range(nz):
            for o in range(O):
                s = 0.0
                for dy in (-1, 0, 1):
                    for dz in (-1, 0, 1):
                        for c in range(C):
                            s += W[dy + 1, dz + 1, o, c] * X[(y + dy) % ny, (z + dz) % nz, c]
                out[y, z, o] = s
    return out


def test_conv_matches_brute_force():
    rng = np.random.default_rng(1)
    W = rng.standard_normal((3, 3, 3, 2))
    X = rng.standard_normal((4, 5, 2))
    assert np.allclose(gen.conv(W, X), _brute_conv(W, X), rtol=0, atol=1e-13)


def test_adjoints():
    rng = np.random.default_rng(2)
    W = rng.standard_normal((3, 3, 4, 3))
    X = rng.standard_normal((5, 6, 3))
    G = rng.standard_normal((5, 6, 4))
    lhs = np.sum(gen.conv(W, X) * G)
    assert abs(lhs - np.sum(X * gen.conv_transpose(W, G))) < 1e-12 * abs(lhs) + 1e-12
    assert abs(lhs - np.sum(W * gen.conv_weight_grad(G, X))) < 1e-12 * abs(lhs) + 1e-12


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    width, blocks, c0 = 4, 2, 8
    p = gen.unflatten(inputs.generator_params(3, width, blocks, c0, block_scale=0.5, out_scale=1.0,
                                              bias_std=0.1), width, blocks, c0)
    xs = [rng.standard_normal((5, 6, c0)) for _ in range(2)]
    ts = [rng.standard_normal((5, 6, 3)) for _ in range(2)]
    _, g = gen.loss_and_grads(p, xs, ts)
    v = gen.flatten(p)
    gv = gen.flatten({"W_in": g["W_in"], "b_in": g["b_in"], "W": g["W"], "b": g["b"],
                      "W_out": g["W_out"], "b_out": g["b_out"]})
    idx = rng.choice(v.size, 40, replace=False)
    eps = 1e-6
    for i in idx:
        vp, vm = v.copy(), v.copy()
        vp[i] += eps
        vm[i] -= eps
        lp, _ = gen.loss_and_grads(gen.unflatten(vp, width, blocks, c0), xs, ts)
        lm, _ = gen.loss_and_grads(gen.unflatten(vm, width, blocks, c0), xs, ts)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - gv[i]) < 1e-6 * max(abs(fd), 1e-3), (i, fd, gv[i])


def test_flat_order_round_trips():
    v = inputs.generator_params(4, 4, 3, 8)
    assert v.size == 9 * 4 * 8 + 4 + 3 * (9 * 16 + 4) + 9 * 3 * 4 + 3
    assert v.size == inputs.generator_param_count(4, 3, 8)
    p = gen.unflatten(v, 4, 3, 8)
    assert p["W_in"].shape == (3, 3, 4, 8) and p["W_out"].shape == (3, 3, 3, 4)
    assert np.array_equal(gen.flatten(p), v)


def test_advected_planes_are_shifted_copies():
    pl = inputs.advected_planes(4, 6, 16, seed=1, shift=1)
    assert np.allclose(pl[1], np.roll(pl[0], 1, axis=-1), atol=1e-12)
    assert np.allclose(pl[3], np.roll(pl[0], 3, axis=-1), atol=1e-12)


def test_bf16_rounding():
    one = 1.0
    assert gen.bf16_round(one) == one
    assert gen.bf16_round(1 + 2.0 ** -8) == 1.0                     # tie -> even (1.0)
    assert gen.bf16_round(1 + 3 * 2.0 ** -8) == 1 + 2.0 ** -6       # tie -> even (1 + 2^-6)
    assert gen.bf16_round(1 + 2.0 ** -8 + 2.0 ** -20) == 1 + 2.0 ** -7
    assert gen.bf16_round(-(1 + 2.0 ** -7)) == -(1 + 2.0 ** -7)
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(5).standard_normal(10000) * 10.0 ** np.random.default_rng(6).integers(-8, 8, 10000)
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(gen.bf16_round(x), ref)


def test_adam_closed_forms():
    rng = np.random.default_rng(7)
    w0 = rng.standard_normal(50)
    g = rng.standard_normal(50)
    m = np.zeros(50)
    v = np.zeros(50)
    lr, eps = 1e-3, 1e-8
    w, m, v = gen.adam_step(w0, g, m, v, 1, lr, eps=eps)
    assert np.allclose(w, w0 - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    # a constant gradient keeps the bias-corrected moments at g and g^2
    for t in range(2, 6):
        w_prev = w
        w, m, v = gen.adam_step(w, g, m, v, t, lr, eps=eps)
        assert np.allclose(w - w_prev, -lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-16)


def test_renormalise():
    rng = np.random.default_rng(8)
    q = rng.standard_normal((8, 6, 3)) * np.array([2.0, 0.5, 1.0]) + np.array([1.0, -3.0, 0.2])
    out = gen.renormalise(q, [0.3, 0.2, 0.1])
    assert np.allclose(out.mean(axis=(0, 1)), 0.0, atol=1e-15)
    assert np.allclose(np.sqrt((out ** 2).mean(axis=(0, 1))), [0.3, 0.2, 0.1], rtol=1e-14)
    # a rescaling of the input does not change the result
    assert np.allclose(gen.renormalise(3.0 * q, [0.3, 0.2, 0.1]), out, atol=1e-14)


def test_splitmix64_published_outputs():
    # the reference generator seeded with 0 starts 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F
    r = gen.splitmix64(0, np.arange(3))
    assert [int(x) for x in r] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_box_muller_normals():
    z = gen.normal_from(gen.splitmix64(12345, np.arange(400000)))
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01
    from scipy import stats
    assert stats.kstest(z, "norm").pvalue > 1e-3


def test_noisy_inputs_shift_by_the_drawn_noise():
    rng = np.random.default_rng(9)
    qt, qp = rng.standard_normal((2, 3, 4, 3))
    a, b = gen.noisy_inputs(qt, qp, 1, 0.0, 7)
    assert np.array_equal(a, qt) and np.array_equal(b, qp)
    a, b = gen.noisy_inputs(qt, qp, 1, 0.5, 7)
    eps = gen.normal_from(gen.splitmix64(7, (12 + 0) * 6 + 4))     # sample 1, pixel 0, q_{t-1} channel 1
    assert abs((b[0, 0, 1] - qp[0, 0, 1]) - 0.5 * eps) < 1e-15


def test_rollout_step_relaxation():
    rng = np.random.default_rng(10)
    qt, d, qr = rng.standard_normal((3, 6, 5, 3))
    rms = [1.0, 2.0, 0.5]
    assert np.allclose(gen.rollout_step(qt, d, rms), gen.renormalise(qt + d, rms), atol=1e-15)
    # lambda = 1 replaces q_t by the reference: the step starts from q_ref
    assert np.allclose(gen.rollout_step(qt, d, rms, qr, 1.0), gen.renormalise(qr + d, rms), atol=1e-14)


def test_spectral_relaxation_pins():
    """lam = 0 leaves the plane; lam = 1 with unclamped factors gives exactly
    the target power at every wavenumber with the phases kept (checked
    against a direct DFT sum on a small plane); clamped factors move the
    power by at most 4x; the result stays real."""
    from oracle import generator as gen
    rng = np.random.default_rng(5)
    ny, nz = 6, 8
    q = rng.standard_normal((ny, nz, 3))
    qr = 0.1 * rng.standard_normal((ny, nz, 3))
    f = q - qr
    # direct DFT, independent of numpy's FFT
    y = np.arange(ny)[:, None, None, None]
    z = np.arange(nz)[None, :, None, None]
    ky = np.arange(ny)[None, None, :, None]
    kz = np.arange(nz)[None, None, None, :]
    E = np.exp(-2j * np.pi * (y * ky / ny + z * kz / nz))
    F = np.einsum("yzc,yzab->cab", f, E)
    P0 = np.abs(F) ** 2
    assert np.allclose(gen.spectral_relax(q, qr, P0 * 3.0, 0.0), q, atol=1e-14)
    target = P0 * rng.uniform(0.3, 3.0, size=P0.shape)
    target = 0.5 * (target + target[:, (-np.arange(ny)) % ny][:, :, (-np.arange(nz)) % nz])   # real plane: S(k) = S(-k)
    out = gen.spectral_relax(q, qr, target, 1.0, lo=0.0, hi=np.inf)
    F1 = np.einsum("yzc,yzab->cab", out - qr, E)
    assert np.allclose(np.abs(F1) ** 2, target, rtol=1e-10, atol=1e-12)
    ph = np.abs(F) > 1e-9
    assert np.allclose(F1[ph] / np.abs(F1[ph]), F[ph] / np.abs(F[ph]), atol=1e-10)
    clamped = gen.spectral_relax(q, qr, P0 * 100.0, 1.0)
    F2 = np.einsum("yzc,yzab->cab", clamped - qr, E)
    assert np.allclose(np.abs(F2) ** 2, 4.0 * P0, rtol=1e-10, atol=1e-12)
