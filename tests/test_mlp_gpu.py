"""GPU parity of the planner network's kernels (rel_mlp_round / forward /
backward / adamw) against the float64 oracle (oracle/mlp.py).

Tolerances follow from the arithmetic.  BF16 x BF16 products are exact in
FP32, so a layer's only error is the FP32 rounding of its FMA chain: with n
roundings, |GPU - exact| <= gamma_n * sum |w_i x_i| (+ |b|), gamma_n =
n u / (1 - n u), u = 2^-24 (Higham, Accuracy and Stability of Numerical
Algorithms, 2nd ed., Sec. 3.1).  Each layer is compared with the oracle fed
the GPU's own previous layer, so the BF16 rounding of a hidden activation
cannot flip between the two sides.  BF16 copies are compared bit for bit."""
import ctypes

import numpy as np
import pytest
import torch

import synth
from oracle import mlp as M
from paper_2608_13696_gb300 import rel

pytestmark = pytest.mark.gpu

U = 2.0**-24


def gamma(n):
    return n * U / (1 - n * U)


def setup(seed, B):
    params = synth.mlp_params(seed)
    x = synth.mlp_features(B, seed + 100)
    p = torch.from_numpy(params).cuda()
    bf = torch.empty(M.N_PARAMS, dtype=torch.bfloat16, device="cuda")
    rel.mlp_round(p, bf)
    xc = torch.from_numpy(x).cuda().reshape(B, 264)
    return params, x, p, bf, xc


def test_round_bit_exact():
    params, _, p, bf, _ = setup(1, 1)
    extra = np.array([1.0 + 2.0**-8, 1.0 + 3 * 2.0**-8, -2.5, 0.0, 1e-30, 3e38], np.float32)
    params[:extra.size] = extra
    p = torch.from_numpy(params).cuda()
    rel.mlp_round(p, bf)
    got = bf.float().cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(got, M.bf16_round(params))


@pytest.mark.parametrize("B", [1, 3, 256, 1000])
def test_forward_layers(B):
    params, x, p, bf, xc = setup(2 + B, B)
    acts = torch.empty((B, 128), dtype=torch.float32, device="cuda")
    y = rel.mlp_forward(bf, p, xc, acts).cpu().numpy().astype(np.float64)
    a = acts.cpu().numpy().astype(np.float64)
    z1g, z2g = a[:, :64], a[:, 64:]
    W1, b1, W2, b2, W3, b3 = (np.abs(t) for t in M._operands(params, True))
    xb = M.bf16_round(x)
    # layer 1: 264 FMAs + the bias add
    _, z1, _ = M.forward(params, x)
    bound1 = gamma(265) * (np.abs(xb) @ W1.T + b1) + 1e-30
    assert np.all(np.abs(z1g - z1) <= bound1)
    # layer 2 from the GPU's layer 1
    z2 = M.layer2(params, z1g)
    h1 = M.bf16_round(np.maximum(z1g, 0))
    assert np.all(np.abs(z2g - z2) <= gamma(65) * (h1 @ W2.T + b2) + 1e-30)
    # outputs from the GPU's layer 2
    yr = M.layer3(params, z2g)
    h2 = M.bf16_round(np.maximum(z2g, 0))
    assert np.all(np.abs(y - yr) <= gamma(65) * (h2 @ W3.T + b3) + 1e-30)
    # end to end: close (a hidden BF16 rounding may flip on a near-tie)
    ye, _, _ = M.forward(params, x)
    np.testing.assert_allclose(y, ye, rtol=1e-2, atol=1e-2)


def test_forward_empty_batch():
    _, _, p, bf, _ = setup(5, 1)
    x = torch.empty((0, 264), dtype=torch.float32, device="cuda")
    assert rel.mlp_forward(bf, p, x).shape == (0, 4)


def run_backward(seed, B):
    params, x, p, bf, xc = setup(seed, B)
    rng = np.random.default_rng(seed)
    t = rng.uniform(0, 26, B).astype(np.float32)
    v = rng.integers(0, 3, B).astype(np.int32)
    acts = torch.empty((B, 128), dtype=torch.float32, device="cuda")
    out = rel.mlp_forward(bf, p, xc, acts)
    grad = torch.empty(M.N_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    rel.mlp_backward(bf, xc, acts, out, torch.from_numpy(t).cuda(), torch.from_numpy(v).cuda(),
                     grad, loss)
    return params, x, t, v, acts, out, grad, loss


@pytest.mark.parametrize("B", [1, 64, 300])
def test_backward_matches_oracle(B):
    params, x, t, v, acts, out, grad, loss = run_backward(10 + B, B)
    a = acts.cpu().numpy().astype(np.float64)
    y = out.cpu().numpy().astype(np.float64)
    g_ref, L_ref = M.backward(params, x, t, v, quant=True, z1=a[:, :64], z2=a[:, 64:], y=y)
    A = M.grad_abs_bound(params, x, a[:, :64], a[:, 64:], y, t, v)
    # per-sample terms: softmax/exp/log (a few ulp), 4- and 64-term sums,
    # then the B-term batch sum; doubled for safety
    tol = 2 * gamma(B + 100) * A + 1e-30
    g = grad.cpu().numpy().astype(np.float64)
    bad = np.abs(g - g_ref) > tol
    assert not bad.any(), (np.flatnonzero(bad)[:10], g[bad][:5], g_ref[bad][:5])
    assert float(loss.item()) == pytest.approx(L_ref, rel=1e-5)


def test_backward_empty_batch_zeroes_grad():
    _, _, p, bf, _ = setup(7, 1)
    grad = torch.full((M.N_PARAMS,), 5.0, device="cuda")
    loss = torch.full((1,), 5.0, device="cuda")
    z = torch.empty((0, 264), device="cuda")
    rel.mlp_backward(bf, z, torch.empty((0, 128), device="cuda"), torch.empty((0, 4), device="cuda"),
                     torch.empty(0, device="cuda"), torch.empty(0, dtype=torch.int32, device="cuda"),
                     grad, loss)
    assert not grad.any() and loss.item() == 0.0


def test_backward_workspace_too_small():
    L = rel.load()
    params, x, t, v, acts, out, grad, loss = run_backward(8, 16)
    xc = torch.from_numpy(x).cuda()
    ws = torch.empty(int(L.rel_mlp_ws_bytes(16)) - 4, dtype=torch.uint8, device="cuda")
    tc, vc = torch.from_numpy(t).cuda(), torch.from_numpy(v).cuda()
    bf = torch.empty(M.N_PARAMS, dtype=torch.bfloat16, device="cuda")
    r = L.rel_mlp_backward(bf.data_ptr(), xc.data_ptr(), acts.data_ptr(), out.data_ptr(),
                           tc.data_ptr(), vc.data_ptr(), 16, ws.data_ptr(), ws.numel(),
                           grad.data_ptr(), loss.data_ptr(), None)
    assert r == rel.REL_E_CAPACITY


@pytest.mark.parametrize("step", [1, 7])
def test_adamw_matches_oracle(step):
    rng = np.random.default_rng(20 + step)
    p0 = synth.mlp_params(30 + step)
    m0 = (rng.standard_normal(M.N_PARAMS) * 1e-3).astype(np.float32)
    v0 = (rng.uniform(0, 1e-5, M.N_PARAMS)).astype(np.float32)
    g = (rng.standard_normal(M.N_PARAMS) * 1e-2).astype(np.float32)
    if step == 1:
        m0[:] = 0
        v0[:] = 0
    hp = dict(lr=3e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=1e-2)
    p, m, v = (torch.from_numpy(a.copy()).cuda() for a in (p0, m0, v0))
    bf = torch.empty(M.N_PARAMS, dtype=torch.bfloat16, device="cuda")
    rel.mlp_adamw(p, bf, m, v, torch.from_numpy(g).cuda(), step, **hp)
    # the C interface takes FP32 hyper-parameters: the oracle gets those values
    f = {k: float(np.float32(x)) for k, x in hp.items()}
    pr, mr, vr = M.adamw(p0, m0, v0, g, step, lr=f["lr"], beta1=f["beta1"], beta2=f["beta2"],
                         eps=f["eps"], wd=f["weight_decay"])
    hp = f
    pg, mg, vg = (a.cpu().numpy().astype(np.float64) for a in (p, m, v))
    # m may cancel (beta1 m0 against (1 - beta1) g): bound by the terms' sizes
    m_abs = hp["beta1"] * np.abs(m0) + (1 - hp["beta1"]) * np.abs(g)
    assert np.all(np.abs(mg - mr) <= 4 * U * m_abs + 1e-30)
    np.testing.assert_allclose(vg, vr, rtol=8 * U, atol=1e-30)
    vhat = vr / (1 - hp["beta2"]**step)
    upd = hp["lr"] * m_abs / (1 - hp["beta1"]**step) / (np.sqrt(vhat) + hp["eps"])
    assert np.all(np.abs(pg - pr) <= 4 * U * np.abs(pr) + 32 * U * upd + 1e-30)
    np.testing.assert_array_equal(bf.float().cpu().numpy().astype(np.float64),
                                  M.bf16_round(pg.astype(np.float32)))


def test_adamw_rejects_bad_step():
    p = torch.zeros(M.N_PARAMS, device="cuda")
    bf = torch.empty(M.N_PARAMS, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(rel.RelError):
        rel.mlp_adamw(p, bf, p.clone(), p.clone(), p.clone(), 0)


def test_training_loop_fits_a_rule():
    # the kernels together: fit log2-size = feature 256 and variant = which of
    # features 257..259 is largest; the loss must fall by 20x
    B = 512
    x = torch.from_numpy(synth.mlp_features(B, 40)).cuda()
    t = x[:, 256].contiguous()
    v = torch.argmax(x[:, 257:260], dim=1).to(torch.int32).contiguous()
    p = torch.from_numpy(synth.mlp_params(41)).cuda()
    bf = torch.empty(M.N_PARAMS, dtype=torch.bfloat16, device="cuda")
    rel.mlp_round(p, bf)
    m, vv = torch.zeros_like(p), torch.zeros_like(p)
    acts = torch.empty((B, 128), device="cuda")
    grad = torch.empty_like(p)
    loss = torch.empty(1, device="cuda")
    first = None
    for step in range(1, 601):
        out = rel.mlp_forward(bf, p, x, acts)
        rel.mlp_backward(bf, x, acts, out, t, v, grad, loss)
        if first is None:
            first = loss.item()
        rel.mlp_adamw(p, bf, m, vv, grad, step, lr=3e-3)
    assert loss.item() < first / 20, (first, loss.item())
