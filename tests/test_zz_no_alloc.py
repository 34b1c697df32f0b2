"""sphere_bie_apply_layer_noalloc: the raw layer operators for callers that
cannot allocate device memory (a memory manager owns the device, or their hot
loop bans allocation).  Its output must match sphere_bie_apply_operator with
eta = 0 -- the same self and far-field kernels -- within the FP64 tolerance of
the other parity tests, on consecutive calls that share its static scratch.
This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_1707_06551_gb300 import workloads as wl

TOL64 = 1e-10


@pytest.fixture(scope="module")
def sb():
    from paper_1707_06551_gb300 import build_lib
    build_lib.build()
    from paper_1707_06551_gb300 import sphere_bie
    return sphere_bie


def test_noalloc_rejects_oversize_before_device_work(sb):
    """Sizes beyond the static scratch are refused with a message (no GPU needed)."""
    z = ctypes.c_void_p(16)
    st = sb.lib().sphere_bie_apply_layer_noalloc(sb.SBIE_OP_S, 300, 10, z, z, z, ctypes.c_void_p(32), None)
    assert st == sb.SBIE_ERR_ARG
    assert "65536" in sb.sphere_bie_last_error(None)
    st = sb.lib().sphere_bie_apply_layer_noalloc(sb.SBIE_OP_MOBILITY, 2, 4, z, z, z, ctypes.c_void_p(32), None)
    assert st == sb.SBIE_ERR_ARG


@pytest.mark.gpu
def test_noalloc_matches_apply_operator_on_two_calls(sb):
    import torch
    cases = [("K", wl.small_suspension(7, 5, seed=4)), ("S", wl.small_suspension(5, 8, seed=9, radius_range=(0.6, 1.4)))]
    for call, (op, w) in enumerate(cases):
        c, a, p = w["centres"], w["radii"], w["p"]
        n = len(a)
        dens = np.random.default_rng(20 + call).normal(size=(n * (p + 1) * (2 * p + 2), 3))
        with sb.SphereBIE(c, a, p, eta=0.0) as s:
            ref = s.apply(op, dens)
        dc = torch.tensor(c, dtype=torch.float64, device="cuda")
        da = torch.tensor(a, dtype=torch.float64, device="cuda")
        dd = torch.tensor(dens, dtype=torch.float64, device="cuda")
        out = torch.full_like(dd, float("nan"))
        sb.sphere_bie_apply_layer_noalloc(op, n, p, dc, da, dd, out)
        got = out.cpu().numpy()
        err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        assert err < TOL64, (call, op, err)
