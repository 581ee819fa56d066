"""Time stepping: the low-storage (2N) five-stage fourth-order Runge-Kutta scheme.

The paper advances its DG semi-discretisation with "explicit 4th-order
Runge-Kutta" / "fixed step RK4" (§5.2, Fig. 13) and gives no tableau.  The
low-storage RK4 stage is read as the Carpenter-Kennedy five-stage, 2N-storage
scheme (M. H. Carpenter, C. A. Kennedy, "Fourth-order 2N-storage Runge-Kutta
schemes", NASA TM-109112, 1994; the scheme of Hesthaven & Warburton's codes):

    k  <- a_s k + dt rhs(q),     q <- q + b_s k,     s = 0..4,   a_0 = 0,

with the published rational coefficients below.  The stage times are not
needed (the right-hand sides are autonomous); ``butcher_tableau`` rewrites the
scheme in Butcher form, whose row sums give them.  Classical RK4 is included
for ODE cross-checks only.
"""

from __future__ import annotations

from fractions import Fraction as Fr

import numpy as np

RK4A_EXACT = (Fr(0), Fr(-567301805773, 1357537059087), Fr(-2404267990393, 2016746695238),
              Fr(-3550918686646, 2091501179385), Fr(-1275806237668, 842570457699))
RK4B_EXACT = (Fr(1432997174477, 9575080441755), Fr(5161836677717, 13612068292357),
              Fr(1720146321549, 2090206949498), Fr(3134564353537, 4481467310338),
              Fr(2277821191437, 14882151754819))
NSTAGES = 5
RK4A = tuple(float(x) for x in RK4A_EXACT)
RK4B = tuple(float(x) for x in RK4B_EXACT)


def butcher_tableau():
    """Exact Butcher matrix A[6][5] and weights of the 2N-storage scheme.

    With S_s = a_s S_(s-1) + dt f(Y_s) and Y_(s+1) = Y_s + b_s S_s, the state
    entering stage i is Y_0 + dt sum_(j<i) A_ij f(Y_j) with
    A_ij = sum_(s=j..i-1) b_s prod_(m=j+1..s) a_m; row 5 is the step's weights.
    """
    A = [[Fr(0)] * NSTAGES for _ in range(NSTAGES + 1)]
    for i in range(NSTAGES + 1):
        for j in range(i):
            total = Fr(0)
            for s in range(j, i):
                prod = Fr(1)
                for m in range(j + 1, s + 1):
                    prod *= RK4A_EXACT[m]
                total += RK4B_EXACT[s] * prod
            A[i][j] = total
    return A[:NSTAGES], A[NSTAGES]


def lsrk4_stage(q, k, s, dt, rhs_fn):
    """One stage s of the 2N-storage scheme; returns (q_new, k_new)."""
    k_new = RK4A[s] * k + dt * rhs_fn(q)
    return q + RK4B[s] * k_new, k_new


def lsrk4_step(q, dt, rhs_fn):
    """One full step (five stages) from q; returns the new state."""
    k = np.zeros_like(q)
    for s in range(NSTAGES):
        q, k = lsrk4_stage(q, k, s, dt, rhs_fn)
    return q


def rk4_classic_step(q, dt, rhs_fn):
    """Classical four-stage RK4 (ODE cross-checks only)."""
    k1 = rhs_fn(q)
    k2 = rhs_fn(q + 0.5 * dt * k1)
    k3 = rhs_fn(q + 0.5 * dt * k2)
    k4 = rhs_fn(q + dt * k3)
    return q + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
