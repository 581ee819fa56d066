"""Small MLP for the temperature initial guess: FP64 forward pass, backpropagation and Adam step.

Not in the paper (it appears only as a requirement of this build's learned form):
an 8 -> 64 -> 64 -> 1 perceptron with tanh hidden layers maps normalised
(e, Y_1..Y_7) to a normalised temperature, trained by mean-squared error.  The
GPU path trains it with its own kernels; this oracle is the reference for their
gradients.

Parameter vector (the library's flat layout, float):
    W1 [64][8], b1 [64], W2 [64][64], b2 [64], W3 [64], b3 [1]   (4801 values)
Model:  h1 = tanh(W1 x + b1),  h2 = tanh(W2 h1 + b2),  y = W3 . h2 + b3
Loss:   L = mean over the batch of (y - t)^2
Update: Adam (Kingma & Ba, "Adam: A Method for Stochastic Optimization", ICLR 2015, Algorithm 1).

Test infrastructure only: the tests, the smoke check and the benchmark's CPU baseline use it; the
library never does.
"""

from __future__ import annotations

import numpy as np

N_IN, N_HID = 8, 64
SHAPES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_HID,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def forward(theta, X):
    """X [B][8] -> (y [B], cache)."""
    p = unpack(theta)
    a1 = X @ p["W1"].T + p["b1"]
    h1 = np.tanh(a1)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.tanh(a2)
    y = h2 @ p["W3"] + p["b3"][0]
    return y, (X, h1, h2)


def loss_and_grad(theta, X, t):
    """Mean-squared error and its gradient with respect to the flat parameter vector."""
    p = unpack(theta)
    y, (X, h1, h2) = forward(theta, X)
    B = X.shape[0]
    r = y - t
    L = float(np.mean(r * r))
    dy = 2.0 * r / B                       # dL/dy
    g = {"W3": dy @ h2, "b3": np.array([dy.sum()])}
    d2 = np.outer(dy, p["W3"]) * (1.0 - h2 * h2)   # dL/da2
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ p["W2"]) * (1.0 - h1 * h1)          # dL/da1
    g["W1"] = d1.T @ X
    g["b1"] = d1.sum(axis=0)
    return L, pack(g)


def init_params(seed=0):
    """Glorot-uniform weights, zero biases (seeded)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = {}
    for name, shape in SHAPES:
        if name.startswith("W"):
            fan_in = shape[-1] if len(shape) == 2 else N_HID
            fan_out = shape[0] if len(shape) == 2 else 1
            lim = np.sqrt(6.0 / (fan_in + fan_out))
            parts[name] = rng.uniform(-lim, lim, size=shape)
        else:
            parts[name] = np.zeros(shape)
    return pack(parts)


def adam_step(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) at step number t >= 1, in FP64.

    First and second raw moment estimates m, v are exponential averages of the gradient and its
    square; dividing them by 1 - beta^t removes the bias of their zero initialisation; the step is
    lr * m_hat / (sqrt(v_hat) + eps).  Returns (theta', m', v').
    """
    g = np.asarray(grad, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    theta = np.asarray(theta, dtype=np.float64) - lr * m_hat / (np.sqrt(v_hat) + eps)
    return theta, m, v
