"""Pins for the float64 planner-network oracle (oracle/mlp.py).

The paper has no planner; these pin the oracle to mathematics: torch's own
bfloat16 conversion, a hand-built network with a closed-form output, central
finite differences of the loss, the softmax/cross-entropy special cases and
the closed form of AdamW under a constant gradient."""
import numpy as np
import pytest
import torch

import synth
from oracle import mlp as M


def test_layout():
    assert M.N_PARAMS == 21380
    assert M.OFF_B3 + 4 == M.N_PARAMS
    assert M.is_weight().sum() == 64 * 264 + 64 * 64 + 4 * 64


def test_bf16_round_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([
        rng.standard_normal(20000).astype(np.float32) * 10.0 ** rng.integers(-30, 30, 20000),
        np.array([0.0, -0.0, 1.0, -1.0, 3.0, 1e-40, 3.4e38], np.float32),
    ]).astype(np.float32)
    # exact ties: low 16 bits 0x8000 with either parity of the kept part
    bits = rng.integers(0, 2**32, 5000, dtype=np.uint64).astype(np.uint32)
    bits = (bits & 0x7F7FFFFF & 0xFFFF0000) | 0x8000
    ties = bits.view(np.float32)
    for a in (x, ties):
        want = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
        np.testing.assert_array_equal(M.bf16_round(a), want)


def _hand_net():
    """W1 copies the 8 statistics (inputs 256..263) to hidden units 0..7,
    W2 is the identity on them, W3 row 0 sums them; biases zero except b3."""
    p = np.zeros(M.N_PARAMS)
    W1, b1, W2, b2, W3, b3 = M.unpack(p)
    for j in range(8):
        W1[j, 256 + j] = 1.0
        W2[j, j] = 1.0
        W3[0, j] = 1.0
    W3[1, 0] = 2.0   # logit 1 = 2 * relu(x256)
    W3[2, 1] = -1.0  # logit 2 = -relu(x257)
    b3[:] = [0.5, 0.0, 0.0, 0.25]
    return p


def test_forward_closed_form():
    p = _hand_net()
    rng = np.random.default_rng(1)
    x = rng.integers(-8, 9, size=(16, 264)).astype(np.float64)  # bf16-exact values
    y, z1, z2 = M.forward(p, x, quant=True)
    r = np.maximum(x[:, 256:264], 0)
    np.testing.assert_array_equal(y[:, 0], r.sum(axis=1) + 0.5)
    np.testing.assert_array_equal(y[:, 1], 2 * r[:, 0])
    np.testing.assert_array_equal(y[:, 2], -r[:, 1])
    np.testing.assert_array_equal(y[:, 3], 0.25)
    np.testing.assert_array_equal(z1[:, :8], x[:, 256:264])
    np.testing.assert_array_equal(z1[:, 8:], 0)


def test_forward_quant_rounds_operands():
    # one weight and one input that are not bf16 values: the product uses
    # their roundings; hidden activation rounding shows in the next layer
    p = np.zeros(M.N_PARAMS)
    W1, b1, W2, b2, W3, b3 = M.unpack(p)
    W1[0, 0] = 1.0 + 2.0**-10            # rounds to 1.0 in bf16
    W2[0, 0] = 1.0
    W3[0, 0] = 1.0
    b1[0] = 2.0**-12                     # FP32 bias, kept
    x = np.zeros((1, 264))
    x[0, 0] = 3.0 + 2.0**-9              # rounds to 3.0 in bf16
    y, z1, _ = M.forward(p, x, quant=True)
    assert z1[0, 0] == 3.0 + 2.0**-12
    assert y[0, 0] == 3.0                # bf16(3 + 2^-12) = 3
    y, z1, _ = M.forward(p, x, quant=False)
    assert z1[0, 0] == (1.0 + 2.0**-10) * (3.0 + 2.0**-9) + 2.0**-12


def test_loss_special_cases():
    y = np.array([[5.0, 0.3, 0.3, 0.3], [2.0, 0.0, 0.0, 0.0]])
    assert M.loss(y, [5.0, 2.0], [0, 2]) == pytest.approx(np.log(3.0), rel=1e-15)
    y = np.array([[1.0, 0.0, 0.0, 0.0]])
    assert M.loss(y, [4.0], [1]) == pytest.approx(9.0 + np.log(3.0), rel=1e-15)
    # a confident correct logit drives the cross-entropy to ~0
    y = np.array([[0.0, 0.0, 50.0, 0.0]])
    assert M.loss(y, [0.0], [1]) == pytest.approx(2 * np.exp(-50.0), rel=1e-6)
    g = M.dloss_dy(np.random.default_rng(2).standard_normal((7, 4)), np.zeros(7), np.arange(7) % 3)
    np.testing.assert_allclose(g[:, 1:].sum(axis=1), 0.0, atol=1e-16)


def _rand_case(seed, B=6):
    rng = np.random.default_rng(seed)
    p = synth.mlp_params(seed).astype(np.float64)
    p[M.OFF_B1:M.OFF_W2] = rng.uniform(-0.1, 0.1, 64)
    p[M.OFF_B2:M.OFF_W3] = rng.uniform(-0.1, 0.1, 64)
    p[M.OFF_B3:] = rng.uniform(-0.1, 0.1, 4)
    x = rng.uniform(0, 1, (B, 264))
    x[:, 256] = rng.uniform(20, 26, B)
    return p, x, rng.uniform(0, 20, B), rng.integers(0, 3, B)


def test_backward_matches_finite_differences():
    p, x, t, v = _rand_case(3)
    g, L0 = M.backward(p, x, t, v, quant=False)
    assert L0 == pytest.approx(M.loss(M.forward(p, x, quant=False)[0], t, v))
    rng = np.random.default_rng(4)
    idx = np.concatenate([rng.choice(np.arange(M.OFF_B1), 40, replace=False),
                          np.arange(M.OFF_B1, M.OFF_B1 + 8),
                          rng.choice(np.arange(M.OFF_W2, M.OFF_B2), 30, replace=False),
                          np.arange(M.OFF_B2, M.OFF_B2 + 8),
                          np.arange(M.OFF_W3, M.N_PARAMS)])
    h = 1e-4  # loss ~ 1e2: smaller steps drown in cancellation
    for q in idx:
        pp, pm = p.copy(), p.copy()
        pp[q] += h
        pm[q] -= h
        fd = (M.loss(M.forward(pp, x, quant=False)[0], t, v) -
              M.loss(M.forward(pm, x, quant=False)[0], t, v)) / (2 * h)
        assert g[q] == pytest.approx(fd, rel=1e-5, abs=1e-9), q


def test_backward_quant_equals_plain_on_exact_values():
    # small integer weights and inputs: every operand and every hidden value
    # is a bfloat16, so the rounded and the plain passes must agree exactly
    rng = np.random.default_rng(5)
    p = np.zeros(M.N_PARAMS)
    W1, b1, W2, b2, W3, b3 = M.unpack(p)
    W1[:, :] = rng.integers(-1, 2, W1.shape) * (rng.random(W1.shape) < 0.05)
    W2[:, :] = rng.integers(-1, 2, W2.shape) * (rng.random(W2.shape) < 0.1)
    W3[:, :] = rng.integers(-1, 2, W3.shape)
    x = rng.integers(0, 3, (5, 264)).astype(np.float64)
    t, v = rng.integers(0, 8, 5).astype(np.float64), rng.integers(0, 3, 5)
    y, z1, z2 = M.forward(p, x, quant=True)
    assert np.all(np.abs(z1) < 256) and np.all(np.abs(z2) < 256)
    gq, lq = M.backward(p, x, t, v, quant=True)
    gp, lp = M.backward(p, x, t, v, quant=False)
    np.testing.assert_array_equal(gq, gp)
    assert lq == lp


def test_adamw_constant_gradient_closed_form():
    # with a constant gradient the bias-corrected moments equal g and g^2
    # exactly, so every step moves by lr * g / (|g| + eps); weights also
    # shrink by (1 - lr * wd) per step, biases do not
    rng = np.random.default_rng(6)
    p0 = rng.standard_normal(M.N_PARAMS)
    g = rng.standard_normal(M.N_PARAMS)
    lr, wd, eps = 1e-3, 1e-2, 1e-8
    p, m, v = p0.copy(), np.zeros_like(p0), np.zeros_like(p0)
    K = 5
    for k in range(1, K + 1):
        p, m, v = M.adamw(p, m, v, g, k, lr=lr, wd=wd, eps=eps)
    step = lr * g / (np.abs(g) + eps)
    d = 1 - lr * wd
    w = M.is_weight()
    want = np.where(w, p0 * d**K - step * sum(d**j for j in range(K)), p0 - K * step)
    np.testing.assert_allclose(p, want, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(m, g * (1 - 0.9**K), rtol=1e-12)
    np.testing.assert_allclose(v, g * g * (1 - 0.999**K), rtol=1e-12)


def test_adamw_zero_gradient_only_decays():
    p0 = np.random.default_rng(7).standard_normal(M.N_PARAMS)
    z = np.zeros_like(p0)
    p, m, v = M.adamw(p0, z, z, z, 1, lr=0.1, wd=0.5)
    np.testing.assert_array_equal(p, np.where(M.is_weight(), p0 - 0.05 * p0, p0))
    assert not m.any() and not v.any()
