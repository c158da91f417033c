"""FP64 CPU oracle of the learned interface guess (the network behind dd_cnn_*).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` use it;
it shares no code with the CUDA library.

The paper starts every step from the previous converged interface vector (Sec. 5); the
network below is an addition with no counterpart in the paper.  Definition (the one the
library documents):
* features of the last three converged vectors g1 (most recent), g2, g3, each an image of
  2(N-1) traces by ny+1 nodes: x = (g1/s0, (g1-g2)/s1, (g2-g3)/s1) split into real and
  imaginary parts (6 channels), s0 = rms(g1), s1 = rms(g1 - g2);
* four 3x3 convolutions with zero padding, 6 -> 32 -> 32 -> 32 -> 2 channels, ReLU between;
* guess g0 = 2 g1 - g2 + s1 (out_re + i out_im); training target for a converged gt:
  (gt - 2 g1 + g2)/s1; loss = mean squared error over the 2 output channels.
Parameters are packed per layer as weights [Cout][Cin][3][3] then biases [Cout].
"""
import numpy as np

LAYERS = ((6, 32), (32, 32), (32, 32), (32, 2))


def unpack(params):
    out, off = [], 0
    for ci, co in LAYERS:
        w = params[off:off + co * ci * 9].reshape(co, ci, 3, 3)
        off += co * ci * 9
        b = params[off:off + co]
        off += co
        out.append((np.asarray(w, np.float64), np.asarray(b, np.float64)))
    return out


def pack(layers):
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in layers])


def conv3x3(x, w, b):
    """y[o,h,w] = b[o] + sum_{c,kh,kw} w[o,c,kh,kw] x[c, h+kh-1, w+kw-1] (zero outside)."""
    C, H, W = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1)))
    y = np.zeros((w.shape[0], H, W))
    for kh in range(3):
        for kw in range(3):
            y += np.einsum("oc,chw->ohw", w[:, :, kh, kw], xp[:, kh:kh + H, kw:kw + W])
    return y + b[:, None, None]


def forward(params, x):
    """Returns (output, list of (input, pre-activation) per layer)."""
    layers = unpack(params)
    cache = []
    a = x
    for i, (w, b) in enumerate(layers):
        z = conv3x3(a, w, b)
        cache.append((a, z))
        a = z if i == len(layers) - 1 else np.maximum(z, 0.0)
    return a, cache


def loss_grad(params, x, tgt):
    """Mean squared error and its gradient with respect to the packed parameters."""
    out, cache = forward(params, x)
    n = out.size
    d = 2.0 * (out - tgt) / n
    loss = float(np.mean((out - tgt) ** 2))
    layers = unpack(params)
    grads = [None] * len(layers)
    for i in reversed(range(len(layers))):
        a, z = cache[i]
        if i != len(layers) - 1:
            d = d * (z > 0)
        w, b = layers[i]
        C, H, W = a.shape
        ap = np.pad(a, ((0, 0), (1, 1), (1, 1)))
        gw = np.zeros_like(w)
        for kh in range(3):
            for kw in range(3):
                gw[:, :, kh, kw] = np.einsum("ohw,chw->oc", d, ap[:, kh:kh + H, kw:kw + W])
        grads[i] = (gw, d.sum(axis=(1, 2)))
        # input gradient: da[c,h,w] = sum_{o,kh,kw} w[o,c,kh,kw] d[o, h-kh+1, w-kw+1]
        dp = np.pad(d, ((0, 0), (1, 1), (1, 1)))
        da = np.zeros_like(a)
        for kh in range(3):
            for kw in range(3):
                da += np.einsum("oc,ohw->chw", w[:, :, kh, kw], dp[:, 2 - kh:2 - kh + H, 2 - kw:2 - kw + W])
        d = da
    return loss, pack(grads)


def features(g1, g2, g3, gt=None):
    """(x, target or None, s0, s1) for complex interface images g of shape (2(N-1), ny+1)."""
    s0 = np.sqrt(np.mean(np.abs(g1) ** 2)) + 1e-300
    s1 = np.sqrt(np.mean(np.abs(g1 - g2) ** 2)) + 1e-300
    parts = [g1 / s0, (g1 - g2) / s1, (g2 - g3) / s1]
    x = np.stack([f for p in parts for f in (p.real, p.imag)])
    tgt = None
    if gt is not None:
        t = (gt - 2 * g1 + g2) / s1
        tgt = np.stack([t.real, t.imag])
    return x, tgt, s0, s1


def guess(params, g1, g2, g3):
    x, _, _, s1 = features(g1, g2, g3)
    out, _ = forward(params, x)
    return 2 * g1 - g2 + s1 * (out[0] + 1j * out[1])
