"""Pins of the MLP oracle: backpropagation against central finite differences, and closed forms."""

import numpy as np

from oracle.mlp import N_PARAMS, forward, init_params, loss_and_grad, pack, unpack


def test_parameter_count():
    assert N_PARAMS == 64 * 8 + 64 + 64 * 64 + 64 + 64 + 1 == 4801


def test_gradient_against_central_differences():
    rng = np.random.default_rng(0)
    theta = init_params(3) + rng.normal(scale=0.05, size=N_PARAMS)
    X = rng.normal(size=(16, 8))
    t = rng.normal(size=16)
    L, g = loss_and_grad(theta, X, t)
    idx = rng.choice(N_PARAMS, size=60, replace=False)
    idx = np.concatenate([idx, [N_PARAMS - 1, 0, 512, 576, 4672]])  # b3, W1[0,0], b1[0], W2[0,0], W3[0]
    h = 1e-6
    for i in idx:
        e = np.zeros(N_PARAMS)
        e[i] = h
        fd = (loss_and_grad(theta + e, X, t)[0] - loss_and_grad(theta - e, X, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd)), (i, fd, g[i])


def test_closed_forms():
    theta = np.zeros(N_PARAMS)
    parts = unpack(theta)
    parts["b3"] = np.array([0.25])
    X = np.random.default_rng(1).normal(size=(5, 8))
    y, _ = forward(pack(parts), X)
    assert np.allclose(y, 0.25)           # zero weights: the output bias alone
    L, g = loss_and_grad(pack(parts), X, np.zeros(5))
    assert abs(L - 0.0625) < 1e-15
    gp = unpack(g)
    assert abs(gp["b3"][0] - 0.5) < 1e-15  # d/db3 mean((b3 - 0)^2) = 2 b3
    assert np.all(gp["W1"] == 0) and np.all(gp["W2"] == 0) and np.all(gp["W3"] == 0)
    # a single active path: y = w3 tanh(w2 tanh(w1 x0))
    parts = unpack(np.zeros(N_PARAMS))
    parts["W1"][0, 0], parts["W2"][0, 0], parts["W3"][0] = 0.7, -1.3, 2.0
    x = np.zeros((1, 8))
    x[0, 0] = 0.4
    y, _ = forward(pack(parts), x)
    assert abs(y[0] - 2.0 * np.tanh(-1.3 * np.tanh(0.7 * 0.4))) < 1e-15


# ---- Adam (Kingma & Ba 2015, Algorithm 1) ---------------------------------------------------------

def _run_adam(theta, grads, lr, step=None, **kw):
    from oracle.mlp import adam_step
    step = step or adam_step
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    for t, g in enumerate(grads, start=1):
        theta, m, v = step(theta, g, m, v, t, lr, **kw)
    return theta, m, v


def test_adam_constant_gradient_closed_form():
    """With a constant gradient g from zero moments, the raw moments are the geometric sums
    m_t = (1 - b1^t) g and v_t = (1 - b2^t) g^2, so the bias-corrected estimates are exactly g and g^2
    and every step is lr g / (|g| + eps): after T steps theta = theta_0 - T lr g / (|g| + eps)."""
    g = np.array([0.5, -2.0, 1e-3, 0.0, 7.0])
    theta0 = np.array([1.0, -1.0, 0.25, 3.0, 0.0])
    lr, T, eps = 0.01, 25, 1e-8
    theta, m, v = _run_adam(theta0, [g] * T, lr)
    assert np.allclose(theta, theta0 - T * lr * g / (np.abs(g) + eps), rtol=0, atol=1e-14)
    assert np.allclose(m, (1 - 0.9 ** T) * g, rtol=1e-14, atol=0)
    assert np.allclose(v, (1 - 0.999 ** T) * g * g, rtol=1e-12, atol=0)


def test_adam_two_steps_closed_form():
    """Two steps from zero moments with gradients g1, g2: m_2 = (1 - b1)(b1 g1 + g2) and
    1 - b1^2 = (1 - b1)(1 + b1), so m_hat = (b1 g1 + g2) / (1 + b1); likewise
    v_hat = (b2 g1^2 + g2^2) / (1 + b2).  The first step is lr sign(g1) (eps = 0)."""
    b1, b2, lr = 0.9, 0.999, 0.1
    g1, g2 = np.array([0.5, -3.0, 2.0]), np.array([-0.25, 1.0, 2.0])
    theta0 = np.array([1.0, 0.0, -1.0])
    th1, _, _ = _run_adam(theta0, [g1], lr, eps=0.0)
    assert np.allclose(th1, theta0 - lr * np.sign(g1), rtol=0, atol=1e-15)
    th2, _, _ = _run_adam(theta0, [g1, g2], lr, eps=0.0)
    m_hat = (b1 * g1 + g2) / (1 + b1)
    v_hat = (b2 * g1 * g1 + g2 * g2) / (1 + b2)
    assert np.allclose(th2, th1 - lr * m_hat / np.sqrt(v_hat), rtol=0, atol=1e-15)


def test_adam_is_invariant_to_gradient_scale():
    """With eps = 0 the update depends on the gradients only through their direction per coordinate
    history: scaling every gradient by c > 0 leaves the iterates unchanged."""
    rng = np.random.default_rng(5)
    grads = [rng.normal(size=7) for _ in range(6)]
    theta0 = rng.normal(size=7)
    a, _, _ = _run_adam(theta0, grads, 0.05, eps=0.0)
    b, _, _ = _run_adam(theta0, [1e4 * g for g in grads], 0.05, eps=0.0)
    assert np.allclose(a, b, rtol=0, atol=1e-13)


def test_adam_pins_catch_planted_mistakes():
    """Dropping the bias correction, or swapping the two decay rates, breaks the closed forms."""
    g = np.array([0.5, -2.0])
    theta0 = np.zeros(2)

    def no_bias_correction(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        m = beta1 * m + (1 - beta1) * grad
        v = beta2 * v + (1 - beta2) * grad * grad
        return theta - lr * m / (np.sqrt(v) + eps), m, v

    def swapped_rates(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        from oracle.mlp import adam_step
        return adam_step(theta, grad, m, v, t, lr, beta1=beta2, beta2=beta1, eps=eps)

    want = theta0 - 5 * 0.01 * g / (np.abs(g) + 1e-8)
    for bad in (no_bias_correction,):
        got, _, _ = _run_adam(theta0, [g] * 5, 0.01, step=bad)
        assert not np.allclose(got, want, rtol=0, atol=1e-6)
    g1, g2 = np.array([0.5, -3.0]), np.array([-0.25, 1.0])
    th1, _, _ = _run_adam(theta0, [g1], 0.1, eps=0.0)
    want2 = th1 - 0.1 * ((0.9 * g1 + g2) / 1.9) / np.sqrt((0.999 * g1 * g1 + g2 * g2) / 1.999)
    got2, _, _ = _run_adam(theta0, [g1, g2], 0.1, step=swapped_rates, eps=0.0)
    assert not np.allclose(got2, want2, rtol=0, atol=1e-6)
