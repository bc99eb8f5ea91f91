"""ORACLE -- test infrastructure, not the product.

Plain float64 numpy definition of the planner network that the learned
sizing step consults: 264 sketch features -> 64 -> 64 -> 4, ReLU hidden
layers; output 0 estimates log2 of the number of groups, outputs 1..3 are
logits over the three group-by variants (per-CTA tables, one global table,
partitioned).  The paper has no planner; the network, its loss and its
optimiser are fixed by the library's interface, and this module pins them to
mathematics instead of to the paper:

* ``bf16_round``     -- round-to-nearest-even to bfloat16 (checked against
                        torch's conversion);
* ``forward``        -- the layers as written above (checked on a network
                        built by hand whose output has a closed form);
* ``loss``/``backward`` -- squared error on output 0 plus softmax cross-
                        entropy on outputs 1..3, batch mean; the gradient is
                        written out by the chain rule (checked by central
                        finite differences in float64);
* ``adamw``          -- AdamW (Loshchilov & Hutter, 2019), decoupled weight
                        decay on weights only (checked by the closed form of a
                        constant-gradient run).

With ``quant=True`` the operands are rounded as the GPU kernels round them:
weights and inputs to BF16, hidden activations to BF16 after the ReLU,
biases kept in FP32; products and sums are exact float64 here.  The rounding
is treated as the identity in the backward pass (the kernels do the same).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT = 264, 64, 4
OFF_W1 = 0
OFF_B1 = OFF_W1 + N_H * N_IN
OFF_W2 = OFF_B1 + N_H
OFF_B2 = OFF_W2 + N_H * N_H
OFF_W3 = OFF_B2 + N_H
OFF_B3 = OFF_W3 + N_OUT * N_H
N_PARAMS = OFF_B3 + N_OUT  # 21380


def bf16_round(x) -> np.ndarray:
    """Round float32 values to the nearest bfloat16, ties to even; float64 out.

    A bfloat16 is the top 16 bits of a float32, so rounding adds half an
    ulp of the kept part (0x7FFF, plus the kept part's lowest bit for ties)
    and clears the low 16 bits.  Finite inputs only."""
    b = np.ascontiguousarray(np.asarray(x, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params):
    """W1[64,264], b1[64], W2[64,64], b2[64], W3[4,64], b3[4] views (float64)."""
    p = np.asarray(params, dtype=np.float64)
    assert p.shape == (N_PARAMS,)
    W1 = p[OFF_W1:OFF_B1].reshape(N_H, N_IN)
    b1 = p[OFF_B1:OFF_W2]
    W2 = p[OFF_W2:OFF_B2].reshape(N_H, N_H)
    b2 = p[OFF_B2:OFF_W3]
    W3 = p[OFF_W3:OFF_B3].reshape(N_OUT, N_H)
    b3 = p[OFF_B3:]
    return W1, b1, W2, b2, W3, b3


def _operands(params, quant: bool):
    W1, b1, W2, b2, W3, b3 = unpack(params)
    if quant:
        W1, W2, W3 = bf16_round(W1), bf16_round(W2), bf16_round(W3)
        f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
        b1, b2, b3 = f32(b1), f32(b2), f32(b3)
    return W1, b1, W2, b2, W3, b3


def _act(z, quant: bool):
    h = np.maximum(z, 0.0)
    return bf16_round(h) if quant else h


def forward(params, x, quant: bool = True):
    """Returns (y[B,4], z1[B,64], z2[B,64]) -- z are pre-activations."""
    W1, b1, W2, b2, W3, b3 = _operands(params, quant)
    x = np.asarray(x, dtype=np.float64)
    xi = bf16_round(x) if quant else x
    z1 = xi @ W1.T + b1
    z2 = _act(z1, quant) @ W2.T + b2
    y = _act(z2, quant) @ W3.T + b3
    return y, z1, z2


def layer2(params, z1, quant: bool = True):
    """z2 from given layer-1 pre-activations (to test one layer in isolation)."""
    _, _, W2, b2, _, _ = _operands(params, quant)
    return _act(np.asarray(z1, np.float64), quant) @ W2.T + b2


def layer3(params, z2, quant: bool = True):
    _, _, _, _, W3, b3 = _operands(params, quant)
    return _act(np.asarray(z2, np.float64), quant) @ W3.T + b3


def loss(y, t_ndv, t_var) -> float:
    """Batch mean of (y0 - t_ndv)^2 + cross-entropy(softmax(y1..y3), t_var)."""
    y = np.asarray(y, np.float64)
    t_var = np.asarray(t_var)
    logits = y[:, 1:]
    m = logits.max(axis=1, keepdims=True)
    lse = np.log(np.exp(logits - m).sum(axis=1)) + m[:, 0]
    ce = lse - logits[np.arange(len(y)), t_var]
    se = (y[:, 0] - np.asarray(t_ndv, np.float64)) ** 2
    return float(np.mean(se + ce))


def dloss_dy(y, t_ndv, t_var) -> np.ndarray:
    """d loss / d y, [B, 4]."""
    y = np.asarray(y, np.float64)
    B = len(y)
    g = np.zeros_like(y)
    g[:, 0] = 2.0 * (y[:, 0] - np.asarray(t_ndv, np.float64)) / B
    logits = y[:, 1:]
    e = np.exp(logits - logits.max(axis=1, keepdims=True))
    p = e / e.sum(axis=1, keepdims=True)
    p[np.arange(B), np.asarray(t_var)] -= 1.0
    g[:, 1:] = p / B
    return g


def backward(params, x, t_ndv, t_var, quant: bool = True, z1=None, z2=None, y=None):
    """(gradient[21380], loss).  z1, z2, y may be supplied (e.g. the GPU's own)
    to check the backward pass in isolation from the forward rounding."""
    W1, b1, W2, b2, W3, b3 = _operands(params, quant)
    x = np.asarray(x, dtype=np.float64)
    xi = bf16_round(x) if quant else x
    if z1 is None or z2 is None or y is None:
        y, z1, z2 = forward(params, x, quant)
    z1, z2, y = (np.asarray(a, np.float64) for a in (z1, z2, y))
    h1, h2 = _act(z1, quant), _act(z2, quant)
    dy = dloss_dy(y, t_ndv, t_var)            # [B, 4]
    dz2 = (dy @ W3) * (z2 > 0)                # [B, 64]
    dz1 = (dz2 @ W2) * (z1 > 0)               # [B, 64]
    g = np.empty(N_PARAMS, dtype=np.float64)
    g[OFF_W1:OFF_B1] = (dz1.T @ xi).ravel()
    g[OFF_B1:OFF_W2] = dz1.sum(axis=0)
    g[OFF_W2:OFF_B2] = (dz2.T @ h1).ravel()
    g[OFF_B2:OFF_W3] = dz2.sum(axis=0)
    g[OFF_W3:OFF_B3] = (dy.T @ h2).ravel()
    g[OFF_B3:] = dy.sum(axis=0)
    return g, loss(y, t_ndv, t_var)


def grad_abs_bound(params, x, z1, z2, y, t_ndv, t_var, quant: bool = True) -> np.ndarray:
    """Per-parameter sum over the batch of |each sample's term| -- the scale
    against which a float32 sum of those terms is compared."""
    W1, b1, W2, b2, W3, b3 = _operands(params, quant)
    x = np.asarray(x, dtype=np.float64)
    xi = bf16_round(x) if quant else x
    z1, z2, y = (np.asarray(a, np.float64) for a in (z1, z2, y))
    h1, h2 = _act(z1, quant), _act(z2, quant)
    dy = np.abs(dloss_dy(y, t_ndv, t_var))
    dz2 = (dy @ np.abs(W3)) * (z2 > 0)
    dz1 = (dz2 @ np.abs(W2)) * (z1 > 0)
    a = np.empty(N_PARAMS, dtype=np.float64)
    a[OFF_W1:OFF_B1] = (dz1.T @ np.abs(xi)).ravel()
    a[OFF_B1:OFF_W2] = dz1.sum(axis=0)
    a[OFF_W2:OFF_B2] = (dz2.T @ np.abs(h1)).ravel()
    a[OFF_B2:OFF_W3] = dz2.sum(axis=0)
    a[OFF_W3:OFF_B3] = (dy.T @ np.abs(h2)).ravel()
    a[OFF_B3:] = dy.sum(axis=0)
    return a


def is_weight() -> np.ndarray:
    """True for weight entries (decayed), False for biases."""
    w = np.zeros(N_PARAMS, dtype=bool)
    w[OFF_W1:OFF_B1] = True
    w[OFF_W2:OFF_B2] = True
    w[OFF_W3:OFF_B3] = True
    return w


def adamw(p, m, v, g, step: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, wd=1e-4):
    """One AdamW step; returns (p, m, v) in float64.

    Moments: m <- beta1 m + (1 - beta1) g, v <- beta2 v + (1 - beta2) g^2,
    bias-corrected by 1 - beta^step.  Decoupled weight decay multiplies the
    weights (not the biases) by 1 - lr * wd before the moment update."""
    p, m, v, g = (np.asarray(a, np.float64).copy() for a in (p, m, v, g))
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mhat = m / (1 - beta1 ** step)
    vhat = v / (1 - beta2 ** step)
    p = np.where(is_weight(), p - lr * wd * p, p)
    p = p - lr * mhat / (np.sqrt(vhat) + eps)
    return p, m, v

