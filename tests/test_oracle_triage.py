"""Pins of the triage oracle (oracle/triage.py) against closed forms, hand
cases, finite differences and library routines -- nothing here re-types the
oracle's own formulas."""
import math

import numpy as np
import pytest

from oracle import triage as T


def test_parameter_count_and_layout():
    assert T.N_PARAMS == 128 * 256 + 256 + 256 * 256 + 256 + 256 + 1
    th = np.arange(T.N_PARAMS, dtype=np.float64)
    p = T.unpack(th)
    assert p["W1"][1, 0] == 256 and p["b1"][0] == 128 * 256
    assert p["b3"][0] == T.N_PARAMS - 1


def test_bf16_round_matches_torch_and_ties_to_even():
    torch = pytest.importorskip("torch")
    r = np.random.default_rng(5)
    x = np.concatenate([r.normal(size=2000) * 10.0 ** r.integers(-5, 5, 2000),
                        [0.0, -0.0, 1.0, 65504.0, 1e-40]]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(T.bf16_round(x), ref)
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7: ties to the even mantissa (1)
    assert T.bf16_round(np.float32(1 + 2 ** -8)) == 1.0
    assert T.bf16_round(np.float32(1 + 3 * 2 ** -8)) == 1 + 2 ** -6


def test_backward_matches_central_differences():
    r = np.random.default_rng(6)
    params = r.normal(scale=0.2, size=T.N_PARAMS)
    X = r.normal(size=(7, 128))
    lab = np.array([1, 0, 0, 1, 0, 1, 0], np.float64)

    def loss(pv):
        _, _, y = T.mlp_forward_raw(pv, X)
        return T.bce_with_logits(y, lab, pw=2.0)[0]

    H1, H2, y = T.mlp_forward_raw(params, X)
    _, dy = T.bce_with_logits(y, lab, pw=2.0)
    # mlp_backward differentiates at the rounded parameters: feed exact ones
    exact = T.rounded(params)
    H1, H2, y = T.mlp_forward_raw(exact, X)
    _, dy = T.bce_with_logits(y, lab, pw=2.0)
    g = T.mlp_backward(exact, X, H1, H2, dy)
    idx = np.concatenate([r.integers(0, T.N_PARAMS, 300), [T.N_PARAMS - 1, 128 * 256 + 3]])
    h = 1e-6
    for i in idx:
        e = np.zeros(T.N_PARAMS)
        e[i] = h
        fd = (loss(exact + e) - loss(exact - e)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_bce_closed_forms():
    loss, dy = T.bce_with_logits(np.zeros(4), np.array([0, 1, 0, 1.0]))
    assert math.isclose(loss, math.log(2.0), rel_tol=1e-15)
    np.testing.assert_allclose(dy, np.array([0.5, -0.5, 0.5, -0.5]) / 4, rtol=1e-15)
    loss, _ = T.bce_with_logits(np.array([50.0]), np.array([1.0]), pw=3.0)
    assert loss < 1e-20


def test_zero_network_output_is_bias():
    th = np.zeros(T.N_PARAMS)
    th[-1] = 0.75
    _, _, y = T.mlp_forward(th, np.random.default_rng(1).normal(size=(5, 128)))
    np.testing.assert_array_equal(y, np.full(5, 0.75))


def test_adam_first_step_is_signed_learning_rate():
    g = np.array([3.0, -0.5, 1e-3])
    th, m, v = T.adam_step(np.zeros(3), np.zeros(3), np.zeros(3), g, 1, lr=0.01, eps=0.0)
    np.testing.assert_allclose(th, -0.01 * np.sign(g), rtol=1e-12)


def test_histogram_hand_case():
    psi = np.array([[-np.inf, -100.0, 0.0, 0.999, 1.0, 7.99, 8.0, 1e9]])
    counts, feat = T.histogram_features(psi, lo=0.0, hi=8.0, n_bins=8)
    np.testing.assert_array_equal(counts[0], [4, 1, 0, 0, 0, 0, 0, 3])
    np.testing.assert_allclose(feat[0, 0], math.log(5.0))


def test_sky_order_and_patches():
    v = np.zeros((1, 5, 3))
    v[0, 2] = [1.0, 0.0, 0.0]     # middle segment of 5
    nhat = np.array([[0.3, 0.9539392, 0], [-1, 0, 0], [0.3, -0.9539392, 0], [0.9, 0.43588989, 0]])
    np.testing.assert_array_equal(T.sky_order(v, nhat), [1, 0, 2, 3])
    assert T.patches(10, 4) == [(0, 4, 1), (4, 4, 5), (8, 2, 8)]
