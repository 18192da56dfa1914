"""Pins of the float64 MLP reference (oracle/mlp.py) against things other
than itself: central finite differences, torch's own bfloat16 conversion
and Adam optimiser, closed forms of SiLU and of Adam under a constant
gradient, a brute-force disc over all pixels, and a learnable toy target."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import mlp
from paper_2609_11181_b300 import synth


def _data(seed, n=48):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, mlp.F))
    t = rng.standard_normal(n)
    theta = synth.mlp_init_params(seed).double().numpy()
    return theta, X, t


@pytest.mark.parametrize("weights", ["fp32", "bf16"])
def test_gradient_matches_central_differences(weights):
    theta, X, t = _data(1)
    L, g = mlp.loss_and_grad(theta, X, t, weights=weights)
    rng = np.random.default_rng(2)
    # every bias and a sample of each weight block
    probe = np.concatenate([np.arange(mlp.OFF_B1, mlp.OFF_W2), np.arange(mlp.OFF_B2, mlp.NPARAMS),
                            rng.choice(np.arange(mlp.OFF_W1, mlp.OFF_B1), 40, replace=False),
                            rng.choice(np.arange(mlp.OFF_W2, mlp.OFF_B2), 200, replace=False)])
    # fp32 weights: differences on the parameters themselves; bf16 weights are
    # piecewise constant in the master value, so differentiate the rounded
    # network by perturbing in the fp32 mode at the rounded point
    base = theta.copy()
    if weights == "bf16":
        for off, size in mlp.WEIGHT_BLOCKS:
            base[off:off + size] = mlp.bf16_round(base[off:off + size])
    h = 1e-6
    num = np.empty(probe.size)
    for k, p in enumerate(probe):
        tp, tm = base.copy(), base.copy()
        tp[p] += h
        tm[p] -= h
        num[k] = (mlp.loss_and_grad(tp, X, t, weights="fp32")[0] - mlp.loss_and_grad(tm, X, t, weights="fp32")[0]) / (2 * h)
    np.testing.assert_allclose(g[probe], num, rtol=1e-6, atol=1e-9)


def test_bf16_rounding_ties_to_even_and_matches_torch():
    one = 1.0
    assert mlp.bf16_round(one) == 1.0
    assert mlp.bf16_round(1 + 2 ** -8) == 1.0                       # tie -> even (down)
    assert mlp.bf16_round(1 + 3 * 2 ** -8) == 1 + 2 ** -6            # tie -> even (up)
    assert mlp.bf16_round(1 + 2 ** -8 + 2 ** -20) == 1 + 2 ** -7     # above the tie
    x = np.random.default_rng(3).standard_normal(10000) * np.exp(np.random.default_rng(4).uniform(-20, 20, 10000))
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).double().numpy()
    np.testing.assert_array_equal(mlp.bf16_round(x), ref)


def test_silu_closed_forms():
    x = np.linspace(-8, 8, 101)
    np.testing.assert_allclose(mlp.silu(x) - mlp.silu(-x), x, rtol=0, atol=1e-14)
    assert mlp.silu(0.0) == 0.0 and mlp.dsilu(0.0) == 0.5
    h = 1e-6
    np.testing.assert_allclose(mlp.dsilu(x), (mlp.silu(x + h) - mlp.silu(x - h)) / (2 * h), rtol=1e-8, atol=1e-10)


def test_zero_second_layer_gives_constant_output_and_no_first_layer_gradient():
    theta, X, t = _data(5)
    theta[mlp.OFF_W2:mlp.OFF_B2] = 0.0
    y, c = mlp.forward(theta, X, weights="fp32")
    p = c["p"]
    np.testing.assert_allclose(y, p["w3"] @ mlp.silu(p["b2"]) + p["b3"], rtol=1e-14)
    L, g = mlp.loss_and_grad(theta, X, t, weights="fp32")
    assert np.all(g[mlp.OFF_W1:mlp.OFF_W2] == 0.0)
    # the output bias gradient is 2 mean(y - t)
    assert math.isclose(g[mlp.OFF_B3], 2 * np.mean(y - t), rel_tol=1e-12)


def test_adam_constant_gradient_closed_form():
    # with a constant gradient the bias-corrected moments are g and g^2 at every
    # step, so each step moves by -lr g / (|g| + eps)
    rng = np.random.default_rng(6)
    g = rng.standard_normal(20)
    theta = rng.standard_normal(20)
    m = np.zeros(20)
    v = np.zeros(20)
    th = theta.copy()
    for k in range(1, 6):
        th, m, v = mlp.adam_step(th, m, v, g, k, 1e-2)
    np.testing.assert_allclose(th, theta - 5 * 1e-2 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-14)


def test_adam_matches_torch_optimiser():
    rng = np.random.default_rng(7)
    theta0 = rng.standard_normal(50)
    grads = [rng.standard_normal(50) * 10 ** rng.uniform(-3, 1) for _ in range(7)]
    p = torch.nn.Parameter(torch.from_numpy(theta0.copy()))
    opt = torch.optim.Adam([p], lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    th, m, v = theta0.copy(), np.zeros(50), np.zeros(50)
    for k, g in enumerate(grads, start=1):
        p.grad = torch.from_numpy(g.copy())
        opt.step()
        th, m, v = mlp.adam_step(th, m, v, g, k, 3e-3)
    np.testing.assert_allclose(th, p.detach().numpy(), rtol=1e-13, atol=1e-15)


def test_disc_moments_match_brute_force_over_all_pixels():
    nside = 8
    npix = 12 * nside * nside
    n_p = np.random.default_rng(8).poisson(5.0, npix)
    allv = oracle.pix2vec(nside, np.arange(npix))
    centres = oracle.pix2vec(nside, np.array([0, 17, 300, 400, npix - 1]))
    theta = math.radians(20.0)
    T = oracle.chord2(theta)
    K, S1, S2 = mlp.disc_count_moments(nside, centres, n_p, theta)
    for k, r0 in enumerate(centres):
        d = allv - r0
        inside = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2] <= T
        assert K[k] == inside.sum()
        assert S1[k] == n_p[inside].sum()
        assert S2[k] == (n_p[inside] ** 2).sum()


def test_feature_variance_closed_forms():
    f = mlp.features(map_e=[0.1, 0.2, 0.0], sum_w=[3.0, 5.0, 0.0], count=[6, 10, 0], members=[3, 2, 0],
                     sum_n2=[14, 50, 0], z=[0.5, -0.5, 0.0])
    # counts {1, 2, 3}: variance 2/3; counts {5, 5}: variance 0; empty aperture: 0
    np.testing.assert_allclose(f[:, 2], [2.0 / 3.0, 0.0, 0.0], atol=1e-15)
    np.testing.assert_array_equal(f[:, 3], [0.5, -0.5, 0.0])


def test_training_learns_a_smooth_target():
    rng = np.random.default_rng(9)
    X = rng.standard_normal((2048, mlp.F))
    t = 0.6 * X[:, 0] - 0.4 * np.tanh(X[:, 3]) + 0.1
    theta = synth.mlp_init_params(9).double().numpy()
    batches = [rng.choice(2048, 256, replace=False) for _ in range(300)]
    _, _, _, losses = mlp.train(theta, X, t, batches, lr=3e-3, weights="bf16")
    assert np.mean(losses[-20:]) < 0.05 * np.mean(losses[:5])
