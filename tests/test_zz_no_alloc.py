"""sphere_bie_apply_layer_noalloc: the raw layer operators for callers that
cannot allocate device memory (a memory manager owns the device, or their hot
loop bans allocation).  Its output must match sphere_bie_apply_operator with
eta = 0 -- the same self and far-field kernels -- within the FP64 tolerance of
the other parity tests, on consecutive calls that share its static scratch,
up to the sizes it advertises (p = 24, exactly 65,536 nodes, 4,096 spheres).
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


def test_noalloc_binding_takes_cuda_tensors_only(sb):
    """The Python binding refuses host arrays before calling the library."""
    h = np.zeros((2, 3))
    with pytest.raises(ValueError, match="CUDA tensor"):
        sb.sphere_bie_apply_layer_noalloc("S", 2, 1, h, np.ones(2), np.zeros((16, 3)), np.zeros((16, 3)))


def _compare(sb, op, c, a, p, seed):
    import torch
    n = len(a)
    dens = np.random.default_rng(seed).normal(size=(n * (p + 1) * (2 * p + 2), 3))
    with sb.SphereBIE(c, a, p, eta=0.0) as s:
        ref = s.apply(op, dens)
    dc = torch.tensor(c, dtype=torch.float64, device="cuda")
    da = torch.tensor(a, dtype=torch.float64, device="cuda")
    dd = torch.tensor(dens, dtype=torch.float64, device="cuda")
    out = torch.full_like(dd, float("nan"))
    sb.sphere_bie_apply_layer_noalloc(op, n, p, dc, da, dd, out)
    got = out.cpu().numpy()
    return np.max(np.abs(got - ref)) / np.max(np.abs(ref))


@pytest.mark.gpu
def test_noalloc_matches_apply_operator_on_two_calls(sb):
    cases = [("K", wl.small_suspension(7, 5, seed=4)), ("S", wl.small_suspension(5, 8, seed=9, radius_range=(0.6, 1.4)))]
    for call, (op, w) in enumerate(cases):
        err = _compare(sb, op, w["centres"], w["radii"], w["p"], 20 + call)
        assert err < TOL64, (call, op, err)


@pytest.mark.gpu
def test_noalloc_at_its_advertised_limits(sb):
    """p = 24 (largest order, 90 KB of shared memory in the self kernel),
    exactly 65,536 nodes (128 spheres at p = 15) and 4,096 spheres (p = 1):
    each in turn on the shared scratch, against apply_operator."""
    w24 = wl.small_suspension(3, 24, seed=5, radius_range=(0.7, 1.3))
    w15 = wl.small_suspension(128, 15, seed=6, push=0.0)
    assert 128 * 16 * 32 == 65536
    g = np.arange(16) * 3.0
    lat = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    cases = [("D", w24["centres"], w24["radii"], 24), ("K", w15["centres"], w15["radii"], 15),
             ("S", lat, np.ones(4096), 1), ("D", w24["centres"], w24["radii"], 24)]
    for call, (op, c, a, p) in enumerate(cases):
        err = _compare(sb, op, c, a, p, 40 + call)
        assert err < TOL64, (call, op, p, err)


@pytest.mark.gpu
def test_noalloc_refuses_host_pointers(sb):
    """Host arrays passed through the C interface are refused with
    SBIE_ERR_ARG by the pointer check, before any kernel is queued."""
    import torch
    w = wl.small_suspension(3, 4, seed=1)
    n, p = 3, 4
    N = n * (p + 1) * (2 * p + 2)
    hc = np.ascontiguousarray(w["centres"])
    dc = torch.tensor(hc, dtype=torch.float64, device="cuda")
    da = torch.tensor(w["radii"], dtype=torch.float64, device="cuda")
    dd = torch.zeros((N, 3), dtype=torch.float64, device="cuda")
    out = torch.zeros_like(dd)
    hd = np.zeros((N, 3))
    P = ctypes.c_void_p
    st = sb.lib().sphere_bie_apply_layer_noalloc(sb.SBIE_OP_D, n, p, P(hc.ctypes.data), P(da.data_ptr()),
                                                 P(dd.data_ptr()), P(out.data_ptr()), None)
    assert st == sb.SBIE_ERR_ARG and "device" in sb.sphere_bie_last_error(None)
    st = sb.lib().sphere_bie_apply_layer_noalloc(sb.SBIE_OP_D, n, p, P(dc.data_ptr()), P(da.data_ptr()),
                                                 P(hd.ctypes.data), P(out.data_ptr()), None)
    assert st == sb.SBIE_ERR_ARG
    torch.cuda.synchronize()
