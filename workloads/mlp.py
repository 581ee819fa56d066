"""Seeded inputs for the learned temperature guess: initial MLP weights and training samples.

Only random draws live here (Glorot-uniform initial weights, uniform temperatures,
Dirichlet mass fractions); energies and Newton labels are computed by each
consumer with its own equation of state.
"""

import numpy as np

N_IN, N_HID = 8, 64
# (name, shape, fan_in, fan_out) in the flat order W1, b1, W2, b2, W3, b3; biases have no fan
LAYOUT = [("W1", (N_HID, N_IN), N_IN, N_HID), ("b1", (N_HID,), 0, 0), ("W2", (N_HID, N_HID), N_HID, N_HID),
          ("b2", (N_HID,), 0, 0), ("W3", (N_HID,), N_HID, 1), ("b3", (1,), 0, 0)]


def glorot_params(seed=0):
    """Flat float32 [4801]: Glorot-uniform weights U(+-sqrt(6 / (fan_in + fan_out))), zero biases."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for _, shape, fan_in, fan_out in LAYOUT:
        if fan_in:
            lim = np.sqrt(6.0 / (fan_in + fan_out))
            parts.append(rng.uniform(-lim, lim, size=shape).ravel())
        else:
            parts.append(np.zeros(int(np.prod(shape))))
    return np.concatenate(parts).astype(np.float32)


def temperature_samples(n, nspecies=7, seed=0, T_min=300.0, T_max=3000.0):
    """(T [n], Y [nspecies][n]): T ~ U(T_min, T_max), Y ~ Dirichlet(1, ..., 1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    T = rng.uniform(T_min, T_max, size=n)
    Y = rng.dirichlet(np.ones(nspecies), size=n).T.copy()
    return T, Y
