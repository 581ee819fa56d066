"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This package only *generates inputs*: meshes of periodic boxes split into
tetrahedra, reference-node coordinates, closed-form initial states, seeded
noise and seeded gas-model coefficients.  It holds none of the DG method's
arithmetic (no operators, fluxes, geometric factors, connectivity, equation of
state or time stepping); every consumer computes those itself.

The workloads follow the paper's runs: nodal DG on tetrahedra with
element-local DOFs (§1, Fig. 1), the isentropic vortex (§5.2), compressible
Navier-Stokes of a perfect gas with gamma = 1.4 (§5.3) and a multi-species
mixture (§4, §5).
"""

from .mesh import box_mesh, equispaced_tet_nodes, physical_nodes, n_nodes, n_face_nodes
from .states import (
    isentropic_vortex,
    taylor_green,
    uniform_perturbation,
    freestream,
    sin_shear,
    advected_wave,
    channel_flow,
    sod_fronts,
)
from .gas import IdealGas, Nasa7Mixture, seeded_nasa7_mixture
from .configs import CONFIGS, get_config

__all__ = [
    "box_mesh",
    "equispaced_tet_nodes",
    "physical_nodes",
    "n_nodes",
    "n_face_nodes",
    "isentropic_vortex",
    "taylor_green",
    "uniform_perturbation",
    "freestream",
    "sin_shear",
    "IdealGas",
    "Nasa7Mixture",
    "seeded_nasa7_mixture",
    "CONFIGS",
    "get_config",
]
