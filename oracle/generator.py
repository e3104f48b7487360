"""Learned inflow generator: plain FP64 oracle of the network, its gradients
and its optimiser.

TEST INFRASTRUCTURE ONLY (see the package header): nothing on the product
path imports this module.

The paper closes (Sec. V) by proposing that the costly grid-resolved inflow
turbulence be replaced by a generated one. The generator here is a stated
reading of that proposal: an autoregressive convolutional network that
predicts the next keyframe of the inflow plane of velocity fluctuations
from the two latest ones (keyframes s recorded planes apart), on the
periodic y-z plane of the domain (Sec. II.A: periodic in y and z).

Feature maps are channels-last arrays [ny, nz, C]. Definitions:

* periodic 3x3 cross-correlation
      conv(W, X)[y, z, o] = sum_{dy, dz in {-1, 0, 1}} sum_c
                            W[dy + 1, dz + 1, o, c] X[(y + dy) mod ny, (z + dz) mod nz, c]
* activation  phi(s) = s (s > 0), s / 8 (s <= 0);  phi'(s) = 1 (s > 0), 1 / 8 (s <= 0)
* network (L residual blocks of width C, input x with C0 channels):
      h_1     = conv(W_in, x) + b_in
      h_{l+1} = h_l + conv(W_l, phi(h_l)) + b_l        l = 1 .. L
      delta   = conv(W_out, phi(h_{L+1})) + b_out      (3 channels)
* loss  = mean over batch, pixels and the 3 channels of (delta - target)^2
* Adam (Kingma & Ba): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
  w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

The input x holds the normalised planes q_t (channels 0-2) and q_{t-s}
(channels 3-5); the remaining input channels are zero.

``bf16=True`` rounds every convolution operand (weights, activations,
back-propagated gradients) to bfloat16 (round to nearest, ties to even)
before the FP64 arithmetic: the operand precision of the GPU path, for
comparisons whose rounding decisions must match. The default is plain FP64.

Parameters are kept in a dict of arrays:
  W_in [3, 3, C, C0], b_in [C], W[l] [3, 3, C, C], b[l] [C], W_out [3, 3, 3, C], b_out [3].
The flat order used by the C interface is: W_in, b_in, then for each block
W_l, b_l, then W_out, b_out, every W in [dy][dz][o][c] order.
"""
from __future__ import annotations

import numpy as np


def bf16_round(a):
    """Round FP64 values to the nearest bfloat16 (ties to even), returned as FP64."""
    f = np.asarray(a, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def phi(s):
    """Activation of the generator (a stated reading of the synthetic-inflow
    perspective of Sec. V): s for s > 0, s / 8 otherwise."""
    return np.where(s > 0, s, s / 8.0)


def dphi(s):
    """Derivative of ``phi``: 1 for s > 0, 1 / 8 otherwise (1 / 8 at 0)."""
    return np.where(s > 0, 1.0, 1.0 / 8.0)


def conv(W, X):
    """Periodic 3x3 cross-correlation, W [3, 3, O, C], X [ny, nz, C] -> [ny, nz, O]."""
    out = np.zeros(X.shape[:2] + (W.shape[2],))
    for dy in (-1, 0, 1):
        for dz in (-1, 0, 1):
            # shifted[y, z] = X[(y + dy) mod ny, (z + dz) mod nz]
            shifted = np.roll(X, shift=(-dy, -dz), axis=(0, 1))
            out += np.einsum("yzc,oc->yzo", shifted, W[dy + 1, dz + 1])
    return out


def conv_transpose(W, G):
    """Adjoint of ``conv`` in its input: [ny, nz, O] -> [ny, nz, C],
    out[p, c] = sum_tap sum_o W[tap, o, c] G[p - tap, o]."""
    out = np.zeros(G.shape[:2] + (W.shape[3],))
    for dy in (-1, 0, 1):
        for dz in (-1, 0, 1):
            shifted = np.roll(G, shift=(dy, dz), axis=(0, 1))   # G[p - tap]
            out += np.einsum("yzo,oc->yzc", shifted, W[dy + 1, dz + 1])
    return out


def conv_weight_grad(G, X):
    """Gradient of sum(G * conv(W, X)) in W: [3, 3, O, C],
    dW[tap, o, c] = sum_p G[p, o] X[p + tap, c]."""
    dW = np.zeros((3, 3, G.shape[2], X.shape[2]))
    for dy in (-1, 0, 1):
        for dz in (-1, 0, 1):
            shifted = np.roll(X, shift=(-dy, -dz), axis=(0, 1))
            dW[dy + 1, dz + 1] = np.einsum("yzo,yzc->oc", G, shifted)
    return dW


def flatten(p):
    """Parameter dict -> flat vector in the interface order W_in, b_in,
    (W_l, b_l) per block, W_out, b_out, every W in [dy][dz][o][c] order."""
    parts = [p["W_in"].ravel(), p["b_in"]]
    for W, b in zip(p["W"], p["b"]):
        parts += [W.ravel(), b]
    parts += [p["W_out"].ravel(), p["b_out"]]
    return np.concatenate(parts)


def unflatten(v, width, blocks, in_channels):
    """Flat vector in the interface order -> parameter dict (inverse of
    ``flatten``)."""
    v = np.asarray(v, dtype=np.float64)
    o = 0

    def take(shape):
        nonlocal o
        n = int(np.prod(shape))
        a = v[o:o + n].reshape(shape)
        o += n
        return a.copy()
    p = {"W_in": take((3, 3, width, in_channels)), "b_in": take((width,)), "W": [], "b": []}
    for _ in range(blocks):
        p["W"].append(take((3, 3, width, width)))
        p["b"].append(take((width,)))
    p["W_out"] = take((3, 3, 3, width))
    p["b_out"] = take((3,))
    assert o == v.size
    return p


def forward(p, x, bf16=False):
    """Network output delta [ny, nz, 3] and the residual stream h_1 .. h_{L+1}."""
    r = bf16_round if bf16 else (lambda a: a)
    hs = [conv(r(p["W_in"]), r(x)) + p["b_in"]]
    for W, b in zip(p["W"], p["b"]):
        hs.append(hs[-1] + conv(r(W), r(phi(hs[-1]))) + b)
    delta = conv(r(p["W_out"]), r(phi(hs[-1]))) + p["b_out"]
    return delta, hs


def loss_and_grads(p, xs, targets, bf16=False):
    """Mean-square loss over a batch (lists of x and target) and its gradient
    in every parameter, by the chain rule through the definitions above."""
    r = bf16_round if bf16 else (lambda a: a)
    count = sum(t.size for t in targets)
    g = {"W_in": 0.0, "b_in": 0.0, "W": [0.0] * len(p["W"]), "b": [0.0] * len(p["b"]),
         "W_out": 0.0, "b_out": 0.0}
    loss = 0.0
    for x, t in zip(xs, targets):
        delta, hs = forward(p, x, bf16)
        err = delta - t
        loss += float(np.sum(err * err))
        gd = 2.0 * err / count
        top = hs[-1]
        g["W_out"] = g["W_out"] + conv_weight_grad(r(gd), r(phi(top)))
        g["b_out"] = g["b_out"] + gd.sum(axis=(0, 1))
        gh = dphi(top) * conv_transpose(r(p["W_out"]), r(gd))
        for l in range(len(p["W"]) - 1, -1, -1):
            h = hs[l]
            g["W"][l] = g["W"][l] + conv_weight_grad(r(gh), r(phi(h)))
            g["b"][l] = g["b"][l] + gh.sum(axis=(0, 1))
            gh = gh + dphi(h) * conv_transpose(r(p["W"][l]), r(gh))
        g["W_in"] = g["W_in"] + conv_weight_grad(r(gh), r(x))
        g["b_in"] = g["b_in"] + gh.sum(axis=(0, 1))
    return loss / count, g


def adam_step(w, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update of flat FP64 arrays (t counts from 1); returns new (w, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def make_input(q_t, q_prev, in_channels):
    """x = the first in_channels of [q_t, q_{t-1}], then zeros: planes
    [ny, nz, 3] -> [ny, nz, in_channels]."""
    full = np.concatenate([q_t, q_prev], axis=-1)
    x = np.zeros(q_t.shape[:2] + (in_channels,))
    k = min(6, in_channels)
    x[..., :k] = full[..., :k]
    return x


def splitmix64(key, counter):
    """SplitMix64 (Steele, Lea and Flood, 2014): the state key + (counter + 1)
    times the golden gamma 0x9E3779B97F4A7C15, then the finaliser
    z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27; z *= 0x94D049BB133111EB;
    z ^= z >> 31 (arithmetic modulo 2^64). Arrays of counters."""
    with np.errstate(over="ignore"):
        z = np.uint64(key) + (np.asarray(counter, dtype=np.uint64) + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def normal_from(r):
    """Box-Muller of the two 32-bit halves: u1 = (hi + 1) / 2^32 in (0, 1],
    u2 = lo / 2^32, N = sqrt(-2 ln u1) cos(2 pi u2)."""
    hi = (r >> np.uint64(32)).astype(np.float64)
    lo = (r & np.uint64(0xFFFFFFFF)).astype(np.float64)
    u1 = (hi + 1.0) / 2.0 ** 32
    u2 = lo / 2.0 ** 32
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def noisy_inputs(q_t, q_prev, b, noise_std, key):
    """Training-input noise of sample b: q_t + std N, q_{t-1} + std N with the
    counters (b P + p) 6 + channel (channels 0-2 for q_t, 3-5 for q_{t-1})."""
    P = q_t.shape[0] * q_t.shape[1]
    base = (np.uint64(b) * np.uint64(P) + np.arange(P, dtype=np.uint64)) * np.uint64(6)
    eps = np.stack([normal_from(splitmix64(key, base + np.uint64(c))) for c in range(6)], axis=-1)
    eps = eps.reshape(q_t.shape[:2] + (6,))
    return q_t + noise_std * eps[..., :3], q_prev + noise_std * eps[..., 3:]


def rollout_step(q_t, delta, rms_target, q_ref=None, lam=0.0):
    """One rollout keyframe: q_t + delta, relaxed towards q_ref at rate lam
    (a stated reading: nudging towards the data's time-mean plane), then
    renormalised."""
    q = q_t + delta
    if lam > 0.0:
        q = q - lam * (q_t - q_ref)
    return renormalise(q, rms_target)


def spectral_relax(q, q_ref, power, lam, lo=0.5, hi=2.0):
    """Spectral relaxation of a keyframe (a stated reading, the rollout's
    second closure): the fluctuation f = q - q_ref of every component is
    taken to Fourier space (2-D, periodic y and z), the amplitude of each
    wavenumber k multiplied by clip((S(k) / |F(k)|^2)^(lam / 2), lo, hi) with
    S = power[c] the target power (unnormalised FFT), the phases kept, and
    the plane transformed back. q, q_ref: [ny, nz, 3]; power: [3, ny, nz]."""
    out = np.array(q, dtype=np.float64)
    for c in range(3):
        F = np.fft.fft2(out[:, :, c] - q_ref[:, :, c])
        P = np.abs(F) ** 2
        S = np.asarray(power[c], dtype=np.float64)
        fac = np.ones_like(P)
        ok = (P > 0) & (S > 0)
        fac[ok] = np.clip((S[ok] / P[ok]) ** (0.5 * lam), lo, hi)
        out[:, :, c] = q_ref[:, :, c] + np.real(np.fft.ifft2(F * fac))
    return out


def renormalise(q, rms_target):
    """Rollout closure (a stated reading): each component of a generated plane
    has its plane mean removed and is rescaled to the target rms, so that the
    emitted inflow keeps the flux (mean) and the turbulence intensity of the
    training data."""
    out = q - q.mean(axis=(0, 1))
    rms = np.sqrt((out * out).mean(axis=(0, 1)))
    return out * (np.asarray(rms_target) / np.where(rms > 0, rms, 1.0))
