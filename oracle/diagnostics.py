"""Oracle of the two global reductions of a distributed run: the integrals of the conserved
variables (the conservation diagnostics) and the largest stability rate, from which the time
step follows as dt = CFL / rate.  Test infrastructure only: imported by tests/,
__graft_entry__.smoke() and bench.py's CPU legs, never by the library.

The paper reports its runs by time step (§5.4) and names neither a step-size rule nor a
diagnostic.  The readings here are:
* integral of q_v over the elements: sum_e J_e sum_i w_i q_v(e, i), with w_i the integral of
  the i-th nodal basis function over the reference tetrahedron (the row sums of its mass
  matrix), exact for the element's polynomial;
* stability rate of element e, the nodal-DG estimate of Hesthaven and Warburton (advective
  (N+1)^2 h^-1 and diffusive (N+1)^4 h^-2 scalings, with 1/h read as half the largest Fscale of
  the element's faces):
      lambda_e = max over the element's nodes of
                 (N+1)^2 / 2 * F_e * (|u| + c)  +  (N+1)^4 / 4 * F_e^2 * nu,
      F_e = max_f Fscale_{e,f},  nu = (mu / rho) max(4/3, gamma / Pr)  (0 without viscosity);
  the rate of a state is the largest lambda_e.
"""

from __future__ import annotations

import numpy as np


def mass_weights(ref):
    """w_i = integral of l_i over the reference element = (M 1)_i."""
    return ref.M @ np.ones(ref.Np)


def integrals(ref, geo, q):
    """[V]: sum over elements and nodes of J_e w_i q[v][e][i]."""
    w = mass_weights(ref)
    return np.einsum("vki,i,k->v", np.asarray(q, dtype=np.float64), w, geo.J)


def element_rates(ref, geo, q, gas, mu=0.0, Pr=0.71):
    """lambda_e [K] of a perfect-gas state q [5][K][Np]."""
    N = ref.N
    rho = q[0]
    u = q[1:4] / rho
    p, c = gas.pressure_sound_speed(q)
    speed = np.sqrt((u * u).sum(axis=0)) + c
    F = geo.Fscale.max(axis=1)[:, None]  # [K][1]
    nu = (mu / rho) * max(4.0 / 3.0, gas.gamma / Pr) if mu > 0 else np.zeros_like(rho)
    node = (N + 1) ** 2 / 2.0 * F * speed + (N + 1) ** 4 / 4.0 * F * F * nu
    return node.max(axis=1)


def max_rate(ref, geo, q, gas, mu=0.0, Pr=0.71):
    return float(element_rates(ref, geo, q, gas, mu, Pr).max())
