"""Plain FP64 CPU restatement of the small convolutional network of the learned warm start
(a 4-layer, 32-channel, 3x3 CNN with GELU that maps the forcing sampled on the
streamfunction control grid and log10(sigma/nu) to a streamfunction and a pressure).

TEST INFRASTRUCTURE ONLY (the oracle): only tests/ may import it.  It shares no code with
the CUDA kernels.  Forward, loss and backward are written from their definitions:
  conv (3x3, zero padding, cross-correlation):
      y[b,o,i,j] = bias[o] + sum_{c,di,dj} w[o,c,di+1,dj+1] x[b,c,i+di,j+dj]
  GELU: g(z) = z Phi(z), Phi the standard normal CDF
  loss: per output channel, mean over its mask of (output - target)^2, summed
  Adam (Kingma & Ba) with bias correction.
"""
import math

import numpy as np

SQRT2 = math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)
_erf = np.vectorize(math.erf)


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / SQRT2))


def gelu_grad(z):
    return 0.5 * (1.0 + _erf(z / SQRT2)) + z * INV_SQRT_2PI * np.exp(-0.5 * z * z)


def conv3x3(x, w, b, d=1):
    """x (B,C,H,W), w (O,C,3,3), b (O,) -> (B,O,H,W); taps at offsets -d, 0, d."""
    B, C, H, W = x.shape
    xp = np.zeros((B, C, H + 2 * d, W + 2 * d))
    xp[:, :, d:d + H, d:d + W] = x
    y = np.zeros((B, w.shape[0], H, W)) + b[None, :, None, None]
    for di in range(3):
        for dj in range(3):
            patch = xp[:, :, d * di:d * di + H, d * dj:d * dj + W]   # x[b,c,i+d(di-1),j+d(dj-1)]
            y += np.einsum("oc,bcij->boij", w[:, :, di, dj], patch)
    return y


def conv3x3_backward(x, w, dy, d=1):
    """Gradients of sum(dy * conv3x3(x, w, b, d)) with respect to x, w, b."""
    B, C, H, W = x.shape
    xp = np.zeros((B, C, H + 2 * d, W + 2 * d))
    xp[:, :, d:d + H, d:d + W] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for di in range(3):
        for dj in range(3):
            patch = xp[:, :, d * di:d * di + H, d * dj:d * dj + W]
            dw[:, :, di, dj] = np.einsum("boij,bcij->oc", dy, patch)
            dxp[:, :, d * di:d * di + H, d * dj:d * dj + W] += np.einsum("oc,boij->bcij", w[:, :, di, dj], dy)
    return dxp[:, :, d:d + H, d:d + W], dw, dy.sum(axis=(0, 2, 3))


class CNN:
    """Layers: 3x3 convs cin -> 32 -> 32 -> 32 -> cout with GELU after the first three;
    layer l uses dilation dil[l].  masks: one (H, W) 0/1 mask per output channel."""

    def __init__(self, params, dil=(1, 1, 1, 1)):
        self.params = [np.asarray(p, dtype=np.float64) for p in params]   # w1,b1,...,w4,b4
        self.dil = tuple(dil)

    def forward(self, x, mask):
        acts, pre = [x], []
        a = x
        for layer in range(4):
            w, b = self.params[2 * layer], self.params[2 * layer + 1]
            z = conv3x3(a, w, b, self.dil[layer])
            pre.append(z)
            a = gelu(z) if layer < 3 else z
            acts.append(a)
        self._cache = (acts, pre)
        return acts[-1] * mask[None]

    def loss_and_grads(self, x, mask, target):
        """mask (C, H, W), target (B, C, H, W)."""
        out = self.forward(x, mask)
        m = mask.reshape(mask.shape[0], -1).sum(axis=1) * x.shape[0]      # points per channel
        diff = (out - target) * mask[None]
        loss = float(sum((diff[:, c] ** 2).sum() / m[c] for c in range(mask.shape[0])))
        acts, pre = self._cache
        d = 2.0 * diff / m[None, :, None, None]                            # d loss / d z4
        grads = [None] * 8
        for layer in range(3, -1, -1):
            w = self.params[2 * layer]
            dx, dw, db = conv3x3_backward(acts[layer], w, d, self.dil[layer])
            grads[2 * layer], grads[2 * layer + 1] = dw, db
            if layer > 0:
                d = dx * gelu_grad(pre[layer - 1])
        return loss, grads


def adam_step(params, grads, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in place; t is the 1-based step count."""
    for i in range(len(params)):
        m[i] = beta1 * m[i] + (1.0 - beta1) * grads[i]
        v[i] = beta2 * v[i] + (1.0 - beta2) * grads[i] ** 2
        mh = m[i] / (1.0 - beta1 ** t)
        vh = v[i] / (1.0 - beta2 ** t)
        params[i] = params[i] - lr * mh / (np.sqrt(vh) + eps)
    return params, m, v
