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

Arithmetic: FP64 throughout, or (``bf16=True``) with the operands of every convolution rounded
to BF16 where the definition puts them -- the features, the weights, the ReLU activations and
the back-propagated output gradients -- and everything else (accumulation, biases, the loss) in
FP64.  ``adam_step`` is the Adam update (Kingma & Ba) with bias-corrected moments.
"""
import numpy as np

LAYERS = ((6, 32), (32, 32), (32, 32), (32, 2))


def bf16(a):
    """Nearest BF16 value (ties to even) of the FP32 rounding of a, returned as float64."""
    u = np.asarray(a, np.float64).astype(np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _ident(a):
    return a


def adam_step(w, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update at step t (1-based): returns (w, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


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


def forward(params, x, bf16_ops=False):
    """Returns (output, list of (input, pre-activation) per layer)."""
    R = bf16 if bf16_ops else _ident
    layers = unpack(params)
    cache = []
    a = R(x)
    for i, (w, b) in enumerate(layers):
        z = conv3x3(a, R(w), b)
        cache.append((a, z))
        a = z if i == len(layers) - 1 else R(np.maximum(z, 0.0))
    return a, cache


def loss_grad(params, x, tgt, bf16_ops=False):
    """Mean squared error and its gradient with respect to the packed parameters."""
    R = bf16 if bf16_ops else _ident
    out, cache = forward(params, x, bf16_ops)
    n = out.size
    d = R(2.0 * (out - tgt) / n)
    loss = float(np.mean((out - tgt) ** 2))
    layers = unpack(params)
    grads = [None] * len(layers)
    for i in reversed(range(len(layers))):
        a, z = cache[i]
        if i != len(layers) - 1:
            d = R(d * (z > 0))
        w, b = layers[i]
        w = R(w)
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


def features(g1, g2, g3, gt=None, e=1.0):
    """(x, target or None, s0, s1) for complex interface images g of shape (2(N-1), ny+1); the
    target is the correction to the base guess g1 + e (g1 - g2) (e = 1 linear extrapolation,
    e = 0 the previous-step vector), in units of s1."""
    s0 = np.sqrt(np.mean(np.abs(g1) ** 2)) + 1e-300
    s1 = np.sqrt(np.mean(np.abs(g1 - g2) ** 2)) + 1e-300
    parts = [g1 / s0, (g1 - g2) / s1, (g2 - g3) / s1]
    x = np.stack([f for p in parts for f in (p.real, p.imag)])
    tgt = None
    if gt is not None:
        t = (gt - g1 - e * (g1 - g2)) / s1
        tgt = np.stack([t.real, t.imag])
    return x, tgt, s0, s1


def guess(params, g1, g2, g3, bf16_ops=False, e=1.0):
    x, _, _, s1 = features(g1, g2, g3, e=e)
    out, _ = forward(params, x, bf16_ops)
    return g1 + e * (g1 - g2) + s1 * (out[0] + 1j * out[1])
