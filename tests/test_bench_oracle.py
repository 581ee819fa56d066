"""The all-core oracle timing of bench.py computes the same stage as the single-process oracle:
element ranges with a two-deep halo (outflow faces beyond it) give the range's right-hand side of
the global mesh, for Euler and for Navier-Stokes (whose BR1 gradients reach one layer further)."""

import numpy as np
import pytest


@pytest.mark.parametrize("name,n", [("euler_small", 3), ("ns_viscous", 3)])
def test_all_core_oracle_stage_equals_single_process(name, n):
    import bench
    from oracle.lsrk import lsrk4_stage
    from workloads.configs import get_config
    cfg = get_config(name)
    run, dofs, desc = bench.oracle_stage_runner(cfg, n=n)
    from workloads.configs import build_case
    case = build_case(cfg, n=n)
    # single process: the stage-0 RK register of the whole mesh
    import oracle.euler as eu
    import oracle.ns as ns
    from oracle.geometry import connect, geometric_factors
    from oracle.refelem import build_reference
    from oracle.thermo import PerfectGas
    ref = build_reference(cfg.N, case["ref_nodes"])
    geo, conn = geometric_factors(case["vertices"]), connect(case["vertices"], case["period"], ref)
    gas = PerfectGas(cfg.gas.gamma, cfg.gas.R)
    f = (lambda u: ns.rhs_ns(ref, geo, conn, u, gas, cfg.gas.mu, cfg.gas.Pr)) if cfg.physics == "ns" else \
        (lambda u: eu.rhs_strong(ref, geo, conn, u, gas))
    _, k_want = lsrk4_stage(case["q"], np.zeros_like(case["q"]), 0, cfg.dt, f)
    _, _, _, k_got = bench.oracle_all_cores(cfg, 3, n=n)
    scale = np.abs(k_want).max(axis=(1, 2))[:, None, None]
    assert np.abs(k_got - k_want).max() <= 1e-12 * scale.max()
    assert (np.abs(k_got - k_want) / scale).max() <= 1e-11
