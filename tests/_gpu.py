"""Helpers for the GPU parity tests (CUDA path through the C ABI vs the oracle)."""

import numpy as np
import pytest


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    from paper_2512_17101_gb300 import capi
    import os
    if not os.path.exists(capi.LIB_PATH):
        __graft_entry__.build()
    return torch


def rel_err(got, want):
    """Max over variables of max|got_v - want_v| / max|want_v| (max-norm per conserved variable)."""
    got = np.asarray(got)
    want = np.asarray(want)
    errs = []
    for v in range(want.shape[0]):
        scale = np.abs(want[v]).max()
        errs.append(np.abs(got[v] - want[v]).max() / (scale if scale > 0 else 1.0))
    return max(errs)


def field_err(got, want):
    """Max over conserved fields of max|got - want| / max|want|, with the momentum components
    taken together as one vector field (rho, rho u, rho E, species); the error measure of the
    mixed-precision form."""
    got = np.asarray(got)
    want = np.asarray(want)
    groups = [[0], [1, 2, 3], [4]] + [[v] for v in range(5, want.shape[0])]
    errs = []
    for g in groups:
        scale = max(np.abs(want[v]).max() for v in g)
        errs.append(max(np.abs(got[v] - want[v]).max() for v in g) / (scale if scale > 0 else 1.0))
    return max(errs)


def component_err(got, want):
    """Per-component relative error max|got_v - want_v| / max|want_v| over the components whose own
    maximum is at least 1 % of their field's (rho, momentum vector, rho E, each species).  The mixed
    forms' bar is field_err; this is the stated second measure: a component much smaller than its
    field (rho w in the Taylor-Green states, where w = 0 initially) has an own-relative error set by
    the rounding of the other components, so components under 1 % of their field are left to
    field_err."""
    got = np.asarray(got)
    want = np.asarray(want)
    groups = [[0], [1, 2, 3], [4]] + [[v] for v in range(5, want.shape[0])]
    err = 0.0
    for g in groups:
        scale = max(np.abs(want[v]).max() for v in g)
        for v in g:
            m = np.abs(want[v]).max()
            if m > 0 and m >= 0.01 * scale:
                err = max(err, np.abs(got[v] - want[v]).max() / m)
    return err
