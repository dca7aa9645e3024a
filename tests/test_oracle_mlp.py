"""Pins of the float64 network reference (oracle.mlp), CPU only: central
finite differences of the loss, closed forms of special cases, and the
definition of bfloat16 rounding."""
import numpy as np
import pytest

from oracle import mlp as M


def data(seed, n=40):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 20, size=(n, M.D_IN))
    y = rng.uniform(0, 25, size=n)
    theta = M.init(seed) * 0.5
    return theta, X, y


@pytest.mark.parametrize("tau", [0.9, 0.5, 0.1])
def test_gradient_matches_finite_differences(tau):
    theta, X, y = data(1)
    _, g = M.gradient(theta, X, y, tau)
    rng = np.random.default_rng(2)
    idx = rng.choice(M.N_PARAMS, size=120, replace=False)
    idx = np.concatenate([idx, [M.N_PARAMS - 1, M.N_PARAMS - 2, 0]])  # b3, w3, W1
    eps = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        num = (M.pinball(M.forward(tp, X)[0], y, tau) - M.pinball(M.forward(tm, X)[0], y, tau)) / (2 * eps)
        assert abs(num - g[i]) <= 1e-6 + 1e-5 * abs(g[i]), (i, num, g[i])


def test_constant_model_gradient_closed_form():
    # all weights zero: the prediction is b3 for every sample, and
    # dL/db3 = (tau * #(y > b3) - (1 - tau) * #(y <= b3)) * (-1) / n
    theta = np.zeros(M.N_PARAMS)
    theta[-1] = 10.0
    y = np.array([1.0, 5.0, 12.0, 30.0, 10.0])
    tau = 0.9
    loss, g = M.gradient(theta, np.ones((5, M.D_IN)), y, tau)
    above = (y > 10).sum()
    assert g[-1] == pytest.approx((-tau * above + (1 - tau) * (5 - above)) / 5)
    assert loss == pytest.approx(np.mean(np.maximum(tau * (y - 10), (tau - 1) * (y - 10))))
    assert np.count_nonzero(g[:-1]) == 0


def test_pinball_half_is_half_mae():
    rng = np.random.default_rng(3)
    p, y = rng.normal(size=50), rng.normal(size=50)
    assert M.pinball(p, y, 0.5) == pytest.approx(0.5 * np.mean(np.abs(p - y)))


def test_adam_first_step_is_lr_times_sign():
    g = np.array([0.3, -2.0, 1e-3, -5e-4])
    th, _, _ = M.adam(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    assert np.allclose(th, -0.01 * np.sign(g), rtol=1e-4)


def test_bf16_rounding():
    vals = np.array([1.0, 1.00390625, 1.005859375, -3.14159265, 65504.0, 1e-20], dtype=np.float32)
    r = M.to_bf16(vals)
    # 1 + 2^-8 is exactly halfway between 1 and 1 + 2^-7: ties to even -> 1
    assert r[0] == 1.0 and r[1] == 1.0
    assert r[2] == pytest.approx(1.0078125)
    assert abs(r[3] + 3.140625) < 1e-12
    assert r[4] == 65536.0
    # 8 significant bits survive: relative error <= 2^-9
    assert np.all(np.abs(r - vals) <= np.abs(vals) * 2.0 ** -8)


def test_adam_constant_gradient_closed_form():
    # with a constant gradient g, m_t = g (1 - b1^t) and v_t = g^2 (1 - b2^t),
    # so the bias-corrected step is lr g / (|g| + eps) at every t
    g = np.array([0.3, -2.0, 1e-3, -5e-4, 7.0])
    th, m, v = np.ones(5), np.zeros(5), np.zeros(5)
    lr, eps, T = 0.01, 1e-8, 50
    for t in range(1, T + 1):
        th, m, v = M.adam(th, g, m, v, t, lr=lr, eps=eps)
    assert np.allclose(th, 1.0 - T * lr * g / (np.abs(g) + eps), rtol=0, atol=1e-12)
    assert np.allclose(m, g * (1 - 0.9 ** T)) and np.allclose(v, g * g * (1 - 0.999 ** T))


def test_forward_bf16_hand_computed():
    # unit 0: x0 -> 3 x0 -> h1 -> h2 -> out; unit 1 is cut by the ReLU.
    # x0 = 1.005859375 rounds to 1.0078125 (bf16 spacing 2^-7 in [1, 2));
    # 3 * 1.0078125 = 3.0234375 lies halfway between 3.015625 and 3.03125
    # (spacing 2^-6 in [2, 4)) and rounds to the even 3.03125;
    # b3 = 0.1f rounds to 0.10009765625.
    p = {k: np.zeros(s) for k, s in M.SIZES}
    p["W1"][0, 0], p["W1"][1, 0] = 3.0, -1.0
    p["W2"][0, 0], p["W2"][1, 1] = 1.0, 1.0
    p["w3"][0], p["w3"][1] = 1.0, 5.0
    p["b3"][0] = np.float32(0.1)
    x = np.zeros((1, M.D_IN), dtype=np.float32)
    x[0, 0] = 1.005859375
    got = M.forward_bf16(M.pack(p), x)[0]
    assert got == 3.03125 + 0.10009765625
    # neither rounding skipped: without the input's, 3 * 1.005859375 rounds
    # to 3.015625; without h1's the value would be 3.0234375
    assert abs(got - (3.015625 + 0.10009765625)) > 1e-3
    assert abs(got - (3.0234375 + 0.10009765625)) > 1e-3
    # the float64 forward keeps every digit
    assert M.forward(M.pack(p), x)[0][0] == pytest.approx(3 * 1.005859375 + float(np.float32(0.1)))
