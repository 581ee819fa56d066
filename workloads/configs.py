"""The five synthetic workloads (shapes of the paper's runs, on tetrahedra).

Each config fixes the mesh (periodic box of n^3 hexahedra x 6 tetrahedra),
the order N, the physics, the initial state recipe, the number of RK4 steps
and the time step.  DOFs are counted per scalar field, as the paper counts
them (§5.3): one DOF = one node of one element.

The time step is a fixed number derived from a closed-form bound of the
initial state's wave speed: dt = 0.3 h / ((N+1)^2 (|u|_max + c_max)), h the
hexahedron edge.  Both the oracle and the GPU path receive the same dt.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .gas import IdealGas, seeded_nasa7_mixture, mixture_primitive_state
from .hexmesh import gll_nodes, hex_box, hex_nodes
from .mesh import box_face_bc, box_mesh, equispaced_tet_nodes, physical_nodes, n_nodes
from .states import advected_wave, channel_flow, sod_fronts, isentropic_vortex, taylor_green, uniform_perturbation


@dataclass(frozen=True)
class Config:
    name: str
    n: int  # hexahedra per box side
    N: int  # polynomial order
    physics: str  # "euler", "ns" or "euler_mixture"
    state: str  # "vortex", "tgv" or "mixture"
    steps: int
    dt: float
    precision: str = "fp64"
    seed: int = 0
    gas: object = field(default=None)
    description: str = ""
    walls: tuple = ()  # ((axis, end, DG_BC_* code), ...): boundary faces instead of periodicity

    @property
    def hexahedral(self) -> bool:
        return self.physics.endswith("_hex")

    @property
    def K(self) -> int:
        return self.n ** 3 if self.hexahedral else 6 * self.n ** 3

    @property
    def Np(self) -> int:
        return (self.N + 1) ** 3 if self.hexahedral else n_nodes(self.N)

    @property
    def dofs(self) -> int:
        return self.K * self.Np


def _tgv_dt(n, N, gamma=1.4, mach=0.1, noise=0.01):
    V0 = mach
    umax = V0 * (1 + noise) * math.sqrt(2.0)
    p0 = 1.0 / gamma
    pmax = p0 + V0 * V0 / 16.0 * 2.0 * 3.0
    cmax = math.sqrt(gamma * pmax / 1.0)
    return 0.3 * (1.0 / n) / ((N + 1) ** 2 * (umax + cmax))


def _vortex_dt(n, N):
    """|u| <= 1 + beta/(2 pi) e^(1/2) ~ 2.31 and c <= sqrt(1.4) ~ 1.19 for the vortex of the workloads."""
    return 0.3 * (1.0 / n) / ((N + 1) ** 2 * (2.31 + 1.19))


def _mixture_dt(n, N):
    """Bound for the seeded 7-species mixture: R_mix <= R_u / W_min with W >= 2 kg/kmol,
    gamma <= 5/3 (cp/R > 2 keeps cv/R > 1.5), T <= 3000 K, |u| <= 10*sqrt(3) m/s."""
    cmax = math.sqrt(5.0 / 3.0 * 8314.462618 / 2.0 * 3000.0)
    return 0.3 * (1.0 / n) / ((N + 1) ** 2 * (cmax + 10.0 * math.sqrt(3.0)))


def _channel_dt(n, N, mach=0.3, noise=0.01):
    return 0.3 * (1.0 / n) / ((N + 1) ** 2 * (mach * (1 + noise) + 1.0))


def _sod_dt(n, N):
    """|u| + c <= 2.2 for the Sod states (c <= sqrt(1.4), |u| below the Sod contact speed 0.93)."""
    return 0.3 * (1.0 / n) / ((N + 1) ** 2 * 2.2)


ADVECTION_VELOCITY = (1.0, 0.5, 0.25)


def _advection_dt(n, N, velocity=ADVECTION_VELOCITY):
    return 0.3 * (1.0 / n) / ((N + 1) ** 2 * sum(abs(v) for v in velocity))


_NS_GAS = IdealGas(gamma=1.4, R=1.0, mu=1.0e-3, Pr=0.71)

CONFIGS = {
    "euler_small": Config(
        name="euler_small", n=4, N=2, physics="euler", state="vortex", steps=1, dt=1.0e-3,
        gas=IdealGas(gamma=1.4, R=1.0),
        description="single-species Euler, 4^3 hexes x 6 = 384 tets, N=2, isentropic vortex + U(+-1e-3), "
                    "one RK4 step, dt=1e-3"),
    "ns_viscous": Config(
        name="ns_viscous", n=24, N=3, physics="ns", state="tgv", steps=10, dt=_tgv_dt(24, 3),
        gas=_NS_GAS,
        description="Navier-Stokes with BR1, mu=1e-3, Pr=0.71, 24^3 hexes x 6 = 82,944 tets, N=3, "
                    "Taylor-Green Mach 0.1 + 1% noise, 10 RK4 steps"),
    "ns_precision": Config(
        name="ns_precision", n=32, N=4, physics="ns", state="tgv", steps=10, dt=_tgv_dt(32, 4),
        gas=_NS_GAS, precision="mixed",
        description="as ns_viscous at 32^3 hexes x 6 = 196,608 tets, N=4; split-product tensor-core D/LIFT"),
    "hex_vortex": Config(
        name="hex_vortex", n=32, N=4, physics="euler_hex", state="vortex", steps=10, dt=_vortex_dt(32, 4),
        gas=IdealGas(gamma=1.4, R=1.0),
        description="Euler on tensor-product hexahedra (the paper's element type), periodic box of 32^3 "
                    "hexahedra, N=4 (125 GLL nodes each, 4,096,000 DOFs), isentropic vortex + U(+-1e-3), "
                    "10 RK4 steps"),
    "ns_channel": Config(
        name="ns_channel", n=24, N=3, physics="ns", state="channel", steps=1, dt=_channel_dt(24, 3),
        gas=_NS_GAS, walls=((1, 0, 2), (1, 1, 2)),
        description="Navier-Stokes with BR1, mu=1e-3, Pr=0.71, 24^3 hexes x 6 = 82,944 tets, N=3, "
                    "no-slip adiabatic walls at y = 0 and y = 1, periodic in x and z; parabolic "
                    "Mach 0.3 channel profile with 1% noise; 1 RK4 step"),
    "euler_shock_av": Config(
        name="euler_shock_av", n=24, N=3, physics="euler", state="fronts", steps=1,
        dt=_sod_dt(24, 3),
        gas=IdealGas(gamma=1.4, R=1.0),
        description="Euler with artificial viscosity (eps0 = 5e-3, s0 = -4 log10 N, kappa = 1), "
                    "24^3 hexes x 6 = 82,944 tets, N=3, two smoothed Sod fronts (width 0.01) in a "
                    "periodic box; 1 RK4 step"),
    "hex_advection": Config(
        name="hex_advection", n=128, N=1, physics="advection_hex", state="wave", steps=10,
        dt=_advection_dt(128, 1),
        description="scalar advection on tensor-product hexahedra, p = 1 (the paper's GPU comparison "
                    "workload), periodic box of 128^3 hexahedra (8 GLL nodes each, 16,777,216 DOFs), "
                    "velocity (1, 0.5, 0.25), smooth wave + U(+-1e-3), 10 RK4 steps"),
    "mixture_learned": Config(
        name="mixture_learned", n=32, N=2, physics="euler_mixture", state="mixture", steps=1, dt=_mixture_dt(32, 2),
        description="7-species Euler mixture, seeded NASA-7, 32^3 hexes x 6 = 196,608 tets, N=2; "
                    "temperature Newton seeded by an MLP"),
}


def get_config(name: str) -> Config:
    return CONFIGS[name]


def build_case(cfg: Config, n=None, N=None):
    """Mesh and initial state of a config (optionally at another size/order).

    Returns dict(vertices, period, ref_nodes, xyz, q or mixture primitives).
    """
    n = cfg.n if n is None else n
    N = cfg.N if N is None else N
    verts, period = box_mesh(n, 1.0)
    rst = equispaced_tet_nodes(N)
    xyz = physical_nodes(verts, rst)
    out = dict(vertices=verts, period=period, ref_nodes=rst, xyz=xyz, N=N, n=n, face_bc=None)
    if cfg.walls:
        period = np.array(period, dtype=np.float64)
        for axis, _, _ in cfg.walls:
            period[axis] = 0.0
        out["period"] = period
        out["face_bc"] = box_face_bc(verts, 1.0, sides={(a, e): c for a, e, c in cfg.walls})
    if cfg.state == "vortex":
        q = isentropic_vortex(xyz, 0.0, gamma=cfg.gas.gamma, period=period)
        out["q"] = uniform_perturbation(q, 1.0e-3, seed=cfg.seed)
    elif cfg.state == "fronts":
        out["q"] = sod_fronts(xyz, gamma=cfg.gas.gamma, width=0.01)
    elif cfg.state == "channel":
        out["q"] = channel_flow(xyz, gamma=cfg.gas.gamma, mach=0.3, noise=0.01, seed=cfg.seed)
    elif cfg.state == "tgv":
        out["q"] = taylor_green(xyz, gamma=cfg.gas.gamma, mach=0.1, noise=0.01, seed=cfg.seed)
    elif cfg.state == "mixture":
        mix = seeded_nasa7_mixture(7, seed=cfg.seed)
        Y, T, vel, p0 = mixture_primitive_state(xyz, 7, seed=cfg.seed)
        out.update(mixture=mix, Y=Y, T=T, vel=vel, p0=p0)
    else:
        raise ValueError(cfg.state)
    return out


def build_hex_case(cfg: Config, n=None, N=None):
    """Mesh, node set and initial state of a hexahedral config: dict(box, nodes1d, xyz, q)."""
    n = cfg.n if n is None else n
    N = cfg.N if N is None else N
    box = hex_box(n, 1.0)
    x = gll_nodes(N)
    xyz = hex_nodes(box, x)
    q = isentropic_vortex(xyz, 0.0, gamma=cfg.gas.gamma, period=box["L"])
    q = uniform_perturbation(q, 1.0e-3, seed=cfg.seed)
    return dict(box=box, nodes1d=x, xyz=xyz, q=q, n=n, N=N)


def build_hex_advection_case(cfg: Config, n=None, N=None):
    """Mesh, node set, velocity and initial scalar u[K][Np] of the advection config."""
    n = cfg.n if n is None else n
    N = cfg.N if N is None else N
    box = hex_box(n, 1.0)
    x = gll_nodes(N)
    xyz = hex_nodes(box, x)
    u = advected_wave(xyz, 0.0, velocity=ADVECTION_VELOCITY)
    u = uniform_perturbation(u[None], 1.0e-3, seed=cfg.seed)[0]
    return dict(box=box, nodes1d=x, xyz=xyz, u=u, velocity=ADVECTION_VELOCITY, n=n, N=N)


def batched_cases(ncases=64, seed=0, n_min=2, n_max=20):
    """The batched workload: ncases independent periodic boxes of n^3 hexahedra x 6
    tetrahedra, n ~ U{n_min..n_max}, order N ~ U{1..4}, half of them Euler (isentropic
    vortex + U(+-1e-3)) and half Navier-Stokes (Taylor-Green Mach 0.1 + 1% noise, mu = 1e-3,
    Pr = 0.71), assigned by a seeded permutation.  Returns a list of dicts with the
    mesh, nodes, state, gas and a CFL time step per case (PCG64, ``seed``)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = rng.integers(n_min, n_max + 1, size=ncases)
    Ns = rng.integers(1, 5, size=ncases)
    viscous = np.zeros(ncases, dtype=bool)
    viscous[rng.permutation(ncases)[: ncases // 2]] = True
    out = []
    for i in range(ncases):
        n, N = int(ns[i]), int(Ns[i])
        verts, period = box_mesh(n, 1.0)
        rst = equispaced_tet_nodes(N)
        xyz = physical_nodes(verts, rst)
        if viscous[i]:
            q = taylor_green(xyz, gamma=1.4, mach=0.1, noise=0.01, seed=seed + i)
            gas = _NS_GAS
            dt = _tgv_dt(n, N)
        else:
            q = uniform_perturbation(isentropic_vortex(xyz, 0.0, gamma=1.4, period=period), 1.0e-3, seed=seed + i)
            gas = IdealGas(gamma=1.4, R=1.0)
            # |u| <= 1 + beta/(2 pi) e^(1/2) ~ 2.31, c <= sqrt(1.4) ~ 1.18 for the vortex
            dt = 0.3 * (1.0 / n) / ((N + 1) ** 2 * (2.31 + 1.19))
        out.append(dict(n=n, N=N, viscous=bool(viscous[i]), vertices=verts, period=period, ref_nodes=rst, q=q,
                        gas=gas, dt=dt, K=verts.shape[0], Np=rst.shape[0]))
    return out
