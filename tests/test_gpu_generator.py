"""Learned inflow generator through the C ABI (GPU) against the FP64 oracle.

The oracle runs with the GPU's operand precision (every convolution operand
rounded to bfloat16 the same way), so the two differ only by FP32 against
FP64 accumulation and by the rare operand whose rounding that difference
flips (one bfloat16 ulp, 2^-8 relative). Bounds:
* network output: max error <= 2e-3 max |delta| (a flipped operand moves an
  output by ~2^-8 |w a| of one of 9 * 128 terms), mean error <= 1e-4 of it;
* loss: 1e-4 relative; every gradient tensor: 5e-3 in the 2-norm;
* Adam: where the gradient is not tiny the first step is -lr sign(g) to
  1e-3 lr; everywhere its size is at most lr (1 + 1e-6) plus the rounding
  of the FP32 master weight.
Shapes span several tiles per image row (nz = 256, two 128-pixel tiles),
the periodic wrap in y (ny = 3) and z, a batch of two samples, weight-
gradient CTAs without work (fewer pixel blocks than CTAs), the 6-channel
input layer and the 3-channel output layer.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NY, NZ, BLOCKS, CIN, BATCH = 3, 256, 2, 6, 2


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_08246_gb300 import binding, build
    build.build()
    return binding.load()


def _params(seed=11):
    from paper_2103_08246_gb300 import inputs
    return inputs.generator_params(seed, 128, BLOCKS, CIN, block_scale=0.5, out_scale=1.0, bias_std=0.1)


def _qs(seed):
    rng = np.random.default_rng(seed)
    shape = (BATCH, NY, NZ, 3)
    return [rng.standard_normal(shape).astype(np.float32).astype(np.float64) for _ in range(3)]


def _oracle_grads(p, qt, qp, tg):
    from oracle import generator as og
    xs = [og.make_input(qt[b], qp[b], CIN) for b in range(BATCH)]
    loss, g = og.loss_and_grads(p, xs, [tg[b] for b in range(BATCH)], bf16=True)
    return loss, og.flatten({"W_in": g["W_in"], "b_in": g["b_in"], "W": g["W"], "b": g["b"],
                             "W_out": g["W_out"], "b_out": g["b_out"]})


def test_forward_matches_oracle(lib):
    from oracle import generator as og
    from paper_2103_08246_gb300 import binding
    gen = binding.Generator(NY, NZ, blocks=BLOCKS, in_channels=CIN, batch=BATCH)
    w = _params()
    gen.set_params(w)
    w32 = w.astype(np.float32).astype(np.float64)
    p = og.unflatten(w32, 128, BLOCKS, CIN)
    qt, qp, _ = _qs(1)
    d = gen.forward(qt, qp)
    for b in range(BATCH):
        ref, _ = og.forward(p, og.make_input(qt[b], qp[b], CIN), bf16=True)
        err = np.abs(d[b] - ref)
        scale = np.abs(ref).max()
        assert scale > 0.1
        assert err.max() <= 2e-3 * scale, (err.max(), scale)
        assert err.mean() <= 1e-4 * scale, (err.mean(), scale)
    gen.close()


def test_gradients_and_adam_match_oracle(lib):
    from oracle import generator as og
    from paper_2103_08246_gb300 import binding, inputs
    gen = binding.Generator(NY, NZ, blocks=BLOCKS, in_channels=CIN, batch=BATCH, lr=1e-3)
    w = _params(12)
    gen.set_params(w)
    w32 = w.astype(np.float32).astype(np.float64)
    p = og.unflatten(w32, 128, BLOCKS, CIN)
    qt, qp, tg = _qs(2)
    loss = gen.grad(qt, qp, tg)
    g = gen.grads()
    loss_ref, g_ref = _oracle_grads(p, qt, qp, tg)
    assert abs(loss - loss_ref) <= 1e-4 * loss_ref
    # per tensor, in the flat order
    off = 0
    sizes = [9 * 128 * CIN, 128] + [9 * 128 * 128, 128] * BLOCKS + [9 * 3 * 128, 3]
    assert sum(sizes) == inputs.generator_param_count(128, BLOCKS, CIN) == g.size
    for n in sizes:
        a, r = g[off:off + n], g_ref[off:off + n]
        assert np.linalg.norm(a - r) <= 5e-3 * np.linalg.norm(r), (off, n)
        off += n
    # one Adam step from zero moments
    gen.adam_step()
    w1 = gen.params()
    w_ref, _, _ = og.adam_step(w32, g_ref, np.zeros_like(w32), np.zeros_like(w32), 1, 1e-3)
    step, step_ref = w1 - w32, w_ref - w32
    big = np.abs(g_ref) > 1e-2 * np.sqrt(np.mean(g_ref ** 2))
    assert big.mean() > 0.5
    assert np.abs(step - step_ref)[big].max() <= 1e-3 * 1e-3
    # the FP32 master weights round the sum w + step (an ulp of w)
    assert np.all(np.abs(step) <= 1e-3 * (1 + 1e-6) + 2.0 ** -23 * np.abs(w32) * 2)
    gen.close()


def test_training_on_planes(lib):
    """Raw-plane path: the first step's loss is the oracle's loss of the
    normalised batch; 60 steps on planes carried one cell per step in z (a
    shift the network can represent) cut the loss of a fixed batch."""
    from oracle import generator as og
    from paper_2103_08246_gb300 import binding, inputs
    planes = inputs.advected_planes(12, NY, NZ, seed=3, shift=1)
    mean = planes.mean(axis=(0, 2, 3))
    std = planes.std(axis=(0, 2, 3))
    gen = binding.Generator(NY, NZ, blocks=BLOCKS, in_channels=CIN, batch=BATCH, lr=1e-3)
    w = _params(13)
    gen.set_params(w)
    gen.set_norm(mean, std, [1.0, 1.0, 1.0])
    dev = torch.as_tensor(planes.astype(np.float32)).cuda()
    torch.cuda.synchronize()
    idx = [4, 7]
    pl32 = planes.astype(np.float32).astype(np.float64)
    m32, s32 = mean.astype(np.float32), std.astype(np.float32)
    inv = (np.float32(1.0) / s32).astype(np.float64)

    def q(t):
        return np.moveaxis((pl32[t] - m32.astype(np.float64)[:, None, None]) * inv[:, None, None], 0, -1)
    p = og.unflatten(w.astype(np.float32).astype(np.float64), 128, BLOCKS, CIN)
    xs = [og.make_input(q(t), q(t - 1), CIN) for t in idx]
    ts = [q(t + 1) - q(t) for t in idx]
    loss_ref, _ = og.loss_and_grads(p, xs, ts, bf16=True)
    first = gen.train_step(dev, idx)
    assert abs(first - loss_ref) <= 1e-3 * loss_ref, (first, loss_ref)
    rng = np.random.default_rng(0)
    for _ in range(60):
        gen.train_step(dev, rng.integers(1, 11, size=BATCH), with_loss=False)
    gen.set_norm(mean, std, [1.0, 1.0, 1.0])
    after = gen.train_step(dev, idx)
    assert after < 0.5 * first, (first, after)
    gen.close()


def test_pushforward_step_matches_oracle(lib):
    """The pushforward step's loss is the oracle's loss of the inputs
    (q^_t, q_{t-1}) with target q_{t+1} - q^_t, q^_t = q_{t-1} + delta the
    network's own prediction from (q_{t-1}, q_{t-2}) (taken from the GPU's
    forward pass, rounded as the kernel rounds it); the update follows (the
    parameters move)."""
    from oracle import generator as og
    from paper_2103_08246_gb300 import binding, inputs
    planes = inputs.advected_planes(12, NY, NZ, seed=5, shift=1)
    mean = planes.mean(axis=(0, 2, 3))
    std = planes.std(axis=(0, 2, 3))
    gen = binding.Generator(NY, NZ, blocks=BLOCKS, in_channels=CIN, batch=BATCH, lr=1e-3)
    w = _params(14)
    gen.set_params(w)
    gen.set_norm(mean, std, [1.0, 1.0, 1.0])
    dev = torch.as_tensor(planes.astype(np.float32)).cuda()
    torch.cuda.synchronize()
    idx = [4, 8]
    pl32 = planes.astype(np.float32).astype(np.float64)
    m32 = mean.astype(np.float32).astype(np.float64)
    inv = (np.float32(1.0) / std.astype(np.float32)).astype(np.float64)

    def q(t):
        return np.moveaxis((pl32[t] - m32[:, None, None]) * inv[:, None, None], 0, -1)
    qprev = np.stack([q(t - 1) for t in idx])
    delta = gen.forward(qprev, np.stack([q(t - 2) for t in idx]))
    qhat = (qprev.astype(np.float32) + delta.astype(np.float32)).astype(np.float64)
    p = og.unflatten(w.astype(np.float32).astype(np.float64), 128, BLOCKS, CIN)
    xs = [og.make_input(qhat[b], qprev[b], CIN) for b in range(BATCH)]
    ts = [q(t + 1) - qhat[b] for b, t in enumerate(idx)]
    loss_ref, _ = og.loss_and_grads(p, xs, ts, bf16=True)
    loss = gen.train_step_pushforward(dev, idx)
    assert abs(loss - loss_ref) <= 1e-3 * loss_ref, (loss, loss_ref)
    assert np.abs(gen.params() - w.astype(np.float32)).max() > 0
    with pytest.raises(binding.IBMError):
        gen.train_step_pushforward(dev, [1, 4])   # needs t >= 2 stride
    gen.close()


def test_training_noise_matches_oracle(lib):
    """With input noise the first step's loss is the oracle's loss of the
    same SplitMix64 / Box-Muller draws (key = seed + Adam steps done)."""
    from oracle import generator as og
    from paper_2103_08246_gb300 import binding, inputs
    planes = inputs.advected_planes(12, NY, NZ, seed=4, shift=1)
    mean = planes.mean(axis=(0, 2, 3))
    std = planes.std(axis=(0, 2, 3))
    gen = binding.Generator(NY, NZ, blocks=BLOCKS, in_channels=CIN, batch=BATCH, lr=1e-3)
    w = _params(15)
    gen.set_params(w)
    gen.set_norm(mean, std, [1.0, 1.0, 1.0])
    gen.set_noise(0.05, seed=99)
    dev = torch.as_tensor(planes.astype(np.float32)).cuda()
    torch.cuda.synchronize()
    idx = [3, 8]
    pl32 = planes.astype(np.float32).astype(np.float64)
    m32 = mean.astype(np.float32).astype(np.float64)
    inv = (np.float32(1.0) / std.astype(np.float32)).astype(np.float64)

    def q(t):
        return np.moveaxis((pl32[t] - m32[:, None, None]) * inv[:, None, None], 0, -1)
    p = og.unflatten(w.astype(np.float32).astype(np.float64), 128, BLOCKS, CIN)
    xs, ts = [], []
    for b, t in enumerate(idx):
        qt, qp = og.noisy_inputs(q(t), q(t - 1), b, 0.05, 99)
        xs.append(og.make_input(qt, qp, CIN))
        ts.append(q(t + 1) - qt)
    loss_ref, _ = og.loss_and_grads(p, xs, ts, bf16=True)
    first = gen.train_step(dev, idx)
    assert abs(first - loss_ref) <= 1e-3 * loss_ref, (first, loss_ref)
    gen.close()


def test_rollout_matches_oracle(lib):
    """One rollout step: q = q_t + delta, renormalised to the target rms,
    emitted as mean + std q into FP64 and FP32 planes; the history advances."""
    from oracle import generator as og
    from paper_2103_08246_gb300 import binding, inputs
    gen = binding.Generator(NY, NZ, blocks=BLOCKS, in_channels=CIN, batch=BATCH)
    w = _params(14)
    gen.set_params(w)
    planes = inputs.advected_planes(2, NY, NZ, seed=5)
    mean = np.array([1.0, 0.02, -0.01])
    std = np.array([0.1, 0.05, 0.06])
    rms = np.array([0.9, 1.1, 1.0])
    gen.set_norm(mean, std, rms)
    gen.rollout_init(planes[0], planes[1])
    m32 = mean.astype(np.float32).astype(np.float64)
    inv = (np.float32(1.0) / std.astype(np.float32)).astype(np.float64)

    def q(pl):
        return np.moveaxis((pl.astype(np.float32).astype(np.float64) - m32[:, None, None]) * inv[:, None, None], 0, -1)
    qt, qp = q(planes[1]), q(planes[0])
    p = og.unflatten(w.astype(np.float32).astype(np.float64), 128, BLOCKS, CIN)
    delta, _ = og.forward(p, og.make_input(qt, qp, CIN), bf16=True)
    q_new = og.renormalise(qt + delta, rms)
    emit = m32 + std.astype(np.float32).astype(np.float64) * q_new
    out = [torch.zeros((NY, NZ), dtype=torch.float64, device="cuda") for _ in range(3)]
    torch.cuda.synchronize()
    gen.rollout(*[o.data_ptr() for o in out], precision=binding.IBM_FP64)
    gen.sync()
    h_t, h_prev = gen.history()
    tol = 2e-3 * np.abs(q_new).max()
    assert np.abs(h_t - q_new).max() <= tol
    assert np.abs(h_prev - qt).max() <= 1e-6
    for c in range(3):
        got = out[c].cpu().numpy()
        assert np.abs(got - emit[..., c]).max() <= tol * std[c] * 1.01
        assert abs(got.mean() - mean[c]) <= 1e-6 * max(1.0, abs(mean[c]))
        assert abs(got.std() - std[c] * rms[c]) <= 1e-4 * std[c]
    # FP32 planes, second step from the advanced history
    out32 = [torch.zeros((NY, NZ), dtype=torch.float32, device="cuda") for _ in range(3)]
    torch.cuda.synchronize()
    gen.rollout(*[o.data_ptr() for o in out32], precision=binding.IBM_FP32)
    gen.sync()
    assert all(np.isfinite(o.cpu().numpy()).all() for o in out32)
    gen.close()


def test_keyframe_stride_and_interpolated_planes(lib):
    """Stride s: the first training loss is the oracle's on (t - s, t, t + s);
    rollout keyframes and the planes emitted between them are
    mean + std ((1 - w) q_prev + w q_t)."""
    from oracle import generator as og
    from paper_2103_08246_gb300 import binding, inputs
    s = 3
    planes = inputs.advected_planes(16, NY, NZ, seed=6, shift=1)
    mean = planes.mean(axis=(0, 2, 3))
    std = planes.std(axis=(0, 2, 3))
    gen = binding.Generator(NY, NZ, blocks=BLOCKS, in_channels=CIN, batch=BATCH, stride=s)
    w = _params(16)
    gen.set_params(w)
    gen.set_norm(mean, std, [1.0, 1.0, 1.0])
    dev = torch.as_tensor(planes.astype(np.float32)).cuda()
    torch.cuda.synchronize()
    idx = [3, 12]
    pl32 = planes.astype(np.float32).astype(np.float64)
    m32 = mean.astype(np.float32).astype(np.float64)
    inv = (np.float32(1.0) / std.astype(np.float32)).astype(np.float64)

    def q(t):
        return np.moveaxis((pl32[t] - m32[:, None, None]) * inv[:, None, None], 0, -1)
    p = og.unflatten(w.astype(np.float32).astype(np.float64), 128, BLOCKS, CIN)
    xs = [og.make_input(q(t), q(t - s), CIN) for t in idx]
    ts = [q(t + s) - q(t) for t in idx]
    loss_ref, _ = og.loss_and_grads(p, xs, ts, bf16=True)
    assert abs(gen.eval(dev, idx) - loss_ref) <= 1e-3 * loss_ref
    with pytest.raises(binding.IBMError):
        gen.eval(dev, [2, 5])            # t - s < 0
    gen.rollout_init(planes[0], planes[3])
    gen.rollout(None, None, None, precision=binding.IBM_FP32)
    q_t, q_prev = gen.history()
    out = [torch.zeros((NY, NZ), dtype=torch.float64, device="cuda") for _ in range(3)]
    torch.cuda.synchronize()
    gen.emit(0.25, *[o.data_ptr() for o in out], precision=binding.IBM_FP64)
    gen.sync()
    for c in range(3):
        ref = m32[c] + std.astype(np.float32)[c] * (0.75 * q_prev[..., c] + 0.25 * q_t[..., c])
        assert np.abs(out[c].cpu().numpy() - ref).max() <= 1e-5 * std[c]
    gen.close()


def test_rollout_relaxation_matches_oracle(lib):
    """With relaxation towards a reference plane the keyframe is
    renormalise(q_t + delta - lambda (q_t - q_ref))."""
    from oracle import generator as og
    from paper_2103_08246_gb300 import binding, inputs
    gen = binding.Generator(NY, NZ, blocks=BLOCKS, in_channels=CIN, batch=BATCH)
    w = _params(17)
    gen.set_params(w)
    planes = inputs.advected_planes(3, NY, NZ, seed=7)
    mean = np.array([1.0, 0.01, -0.02])
    std = np.array([0.1, 0.05, 0.06])
    rms = np.array([1.0, 0.9, 1.1])
    gen.set_norm(mean, std, rms)
    ref_plane = planes.mean(axis=0)
    gen.set_relax(ref_plane, 0.2)
    gen.rollout_init(planes[0], planes[1])
    gen.rollout(None, None, None, precision=binding.IBM_FP32)
    gen.sync()
    h_t, _ = gen.history()
    m32 = mean.astype(np.float32).astype(np.float64)
    inv = (np.float32(1.0) / std.astype(np.float32)).astype(np.float64)

    def q(pl):
        return np.moveaxis((pl.astype(np.float32).astype(np.float64) - m32[:, None, None]) * inv[:, None, None], 0, -1)
    qt, qp = q(planes[1]), q(planes[0])
    q_ref = np.moveaxis((ref_plane - mean[:, None, None]) / std[:, None, None], 0, -1)
    p = og.unflatten(w.astype(np.float32).astype(np.float64), 128, BLOCKS, CIN)
    delta, _ = og.forward(p, og.make_input(qt, qp, CIN), bf16=True)
    ref = og.rollout_step(qt, delta, rms, q_ref, 0.2)
    assert np.abs(h_t - ref).max() <= 2e-3 * np.abs(ref).max()
    gen.close()


def test_checkpoint_restores_training(lib, tmp_path):
    """save after two Adam steps, load into a fresh generator: the next step
    gives the same loss and parameters as the uninterrupted run; a file of
    another configuration or a truncated file is refused."""
    from paper_2103_08246_gb300 import binding, inputs
    planes = inputs.advected_planes(12, NY, NZ, seed=8, shift=1)
    mean, std = planes.mean(axis=(0, 2, 3)), planes.std(axis=(0, 2, 3))
    dev = torch.as_tensor(planes.astype(np.float32)).cuda()
    torch.cuda.synchronize()
    a = binding.Generator(NY, NZ, blocks=BLOCKS, in_channels=CIN, batch=BATCH)
    a.set_params(_params(18))
    a.set_norm(mean, std, [1.0, 1.0, 1.0])
    a.train_step(dev, [2, 5])
    a.train_step(dev, [3, 9])
    path = str(tmp_path / "gen.ckpt")
    a.save(path)
    la = a.train_step(dev, [4, 7])
    b = binding.Generator(NY, NZ, blocks=BLOCKS, in_channels=CIN, batch=BATCH)
    b.load(path)
    lb = b.train_step(dev, [4, 7])
    assert lb == la
    assert np.array_equal(a.params(), b.params())
    other = binding.Generator(NY, NZ, blocks=BLOCKS + 1, in_channels=CIN, batch=BATCH)
    with pytest.raises(binding.IBMError) as e:
        other.load(path)
    assert e.value.code == binding.IBM_EINVAL
    blob = open(path, "rb").read()
    short = str(tmp_path / "short.ckpt")
    open(short, "wb").write(blob[: len(blob) // 2])
    before = b.params()
    with pytest.raises(binding.IBMError) as e:
        b.load(short)
    assert e.value.code == binding.IBM_EIO
    assert np.array_equal(b.params(), before)
    for g in (a, b, other):
        g.close()


def test_bad_configurations_are_refused(lib):
    from paper_2103_08246_gb300 import binding
    for kw in ({"nz": 100}, {"nz": 64}, {"blocks": -1}, {"in_channels": 7}, {"batch": 0}, {"batch": 65}):
        args = {"ny": 4, "nz": 128, "blocks": 1, "in_channels": 6, "batch": 1}
        args.update(kw)
        with pytest.raises(binding.IBMError) as e:
            binding.Generator(args["ny"], args["nz"], blocks=args["blocks"],
                              in_channels=args["in_channels"], batch=args["batch"])
        assert e.value.code == binding.IBM_EINVAL


def test_rollout_spectral_relaxation_matches_oracle(lib):
    """At 256 x 256 planes the keyframe's fluctuation about the reference
    plane is moved towards a target power spectrum (the FP32 radix-16
    transform on the GPU against numpy's FFT in the oracle): the same
    generator state without the spectral step gives the input, the oracle's
    spectral_relax the expected keyframe."""
    from oracle import generator as og
    from paper_2103_08246_gb300 import binding, inputs
    ny = nz = 256
    w = _params(23)
    planes = inputs.advected_planes(3, ny, nz, seed=9)
    mean = np.array([1.0, 0.01, -0.02])
    std = np.array([0.1, 0.05, 0.06])
    rms = np.array([1.0, 0.9, 1.1])
    ref_plane = planes.mean(axis=0)
    q_ref = np.moveaxis((ref_plane - mean[:, None, None]) / std[:, None, None], 0, -1)

    def keyframe(power=None, lam=0.0):
        gen = binding.Generator(ny, nz, blocks=BLOCKS, in_channels=CIN, batch=1)
        gen.set_params(w)
        gen.set_norm(mean, std, rms)
        gen.set_relax(ref_plane, 0.2)
        if power is not None:
            gen.set_spectrum(power, lam)
        gen.rollout_init(planes[0], planes[1])
        gen.rollout(None, None, None, precision=binding.IBM_FP32)
        gen.sync()
        h_t, _ = gen.history()
        gen.close()
        return h_t
    h_off = keyframe()
    rng = np.random.default_rng(4)
    P0 = np.abs(np.fft.fft2(np.moveaxis(h_off - q_ref, -1, 0), axes=(1, 2))) ** 2
    power = P0 * np.exp(rng.uniform(np.log(0.2), np.log(5.0), size=P0.shape))
    power = 0.5 * (power + power[:, (-np.arange(ny)) % ny][:, :, (-np.arange(nz)) % nz])
    h_on = keyframe(power, 0.5)
    ref = og.spectral_relax(h_off, q_ref, power, 0.5)
    assert np.abs(h_on - ref).max() <= 1e-4 * np.abs(ref).max()
    assert np.abs(h_on - h_off).max() > 1e-2 * np.abs(ref).max()   # the step did something
