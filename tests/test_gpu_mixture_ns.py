"""GPU parity of the viscous mixture (species diffusion, enthalpy diffusion, heat conduction):
the FP64 right-hand side through the C ABI against the oracle (oracle/mixture_ns.py), with
temperatures from Newton on both sides, at 1e-11 per conserved variable; the viscous part on its
own (right-hand side minus the inviscid one) at 1e-9."""

import numpy as np
import pytest

import oracle.mixture_ns as mns
from oracle.euler import rhs_strong
from oracle.lsrk import lsrk4_stage
from oracle.thermo import Nasa7Gas
from tests._gpu import rel_err, torch_cuda
from tests._oracle_case import Disc
from workloads import box_mesh, equispaced_tet_nodes
from workloads.gas import mixture_primitive_state, seeded_nasa7_mixture

pytestmark = pytest.mark.gpu
TOL = 1e-11
MU, PR, SC = 0.5, 0.71, 0.6


def _setup(n, N, seed=1):
    torch = torch_cuda()
    from paper_2512_17101_gb300 import dg
    v, per = box_mesh(n, 1.0)
    d = Disc(v, per, N)
    mesh = dg.Mesh(v, per, N, equispaced_tet_nodes(N))
    mix = seeded_nasa7_mixture(7, seed=seed)
    gas_o = Nasa7Gas(W=mix.W, coeffs=mix.coeffs)
    gas = dg.Gas(model="nasa7", W=mix.W, nasa7=mix.coeffs, newton_tol=1e-10, newton_max_it=50, mu=MU, Pr=PR,
                 Sc=SC)
    Y, T, vel, p0 = mixture_primitive_state(d.xyz, 7, seed=seed)
    rho = p0 / (gas_o.R_mix(Y) * T)
    q0 = gas_o.conserved(rho, vel, Y, T)
    _, _, Yc, e = gas_o.split_state(q0)
    Tw, _, ok = gas_o.newton_temperature(e, Yc, np.full(e.shape, 1650.0))
    assert ok.all()
    return torch, dg, d, mesh, gas, gas_o, q0, Tw


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_viscous_mixture_rhs(N):
    torch, dg, d, mesh, gas, gas_o, q0, Tw = _setup(3, N)
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    T = torch.full(q0.shape[1:], 1650.0, device="cuda", dtype=torch.float64)
    dg.dg_rhs(mesh, gas, q, rhs, T_io=T)
    want = mns.rhs_ns_mixture(d.ref, d.geo, d.conn, q0, gas_o, Tw, MU, PR, SC)
    got = rhs.cpu().numpy()
    assert rel_err(got, want) <= TOL
    inviscid = rhs_strong(d.ref, d.geo, d.conn, q0, gas_o, T=Tw)
    assert rel_err(got - inviscid, want - inviscid) <= 1e-9
    assert mesh.status() == 0 and gas.status() == 0


def test_viscous_mixture_rk_stage():
    torch, dg, d, mesh, gas, gas_o, q0, Tw = _setup(3, 2, seed=2)
    dt = 1e-6
    q_in = torch.tensor(q0, device="cuda")
    q_out, k = torch.empty_like(q_in), torch.zeros_like(q_in)
    T = torch.full(q0.shape[1:], 1650.0, device="cuda", dtype=torch.float64)
    dg.dg_rk_stage(mesh, gas, 0, dt, q_in, q_out, k, T_io=T)
    f = lambda u: mns.rhs_ns_mixture(d.ref, d.geo, d.conn, u, gas_o, Tw, MU, PR, SC)
    want_q, want_k = lsrk4_stage(q0, np.zeros_like(q0), 0, dt, f)
    assert rel_err(k.cpu().numpy(), want_k) <= TOL
    assert rel_err(q_out.cpu().numpy() - q0, want_q - q0) <= TOL


def test_viscous_mixture_arguments():
    torch_cuda()
    from paper_2512_17101_gb300 import capi, dg
    mix = seeded_nasa7_mixture(7, seed=0)
    with pytest.raises(capi.DGError):  # a viscous mixture needs a Schmidt number
        dg.Gas(model="nasa7", W=mix.W, nasa7=mix.coeffs, mu=0.1, Pr=0.71)
    torch, dg, d, mesh, gas, gas_o, q0, Tw = _setup(2, 1)
    q = torch.tensor(q0, device="cuda")
    rhs = torch.empty_like(q)
    T = torch.full(q0.shape[1:], 1650.0, device="cuda", dtype=torch.float64)
    with pytest.raises(capi.DGError):  # the mixed-precision mixture form is inviscid
        dg.dg_rhs(mesh, gas, q, rhs, T_io=T, opts=dg._opts(precision=capi.DG_PREC_MIXED))
