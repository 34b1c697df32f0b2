"""The C-ABI library builds, loads and exports every function the header
declares; host-side argument checks run without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1707_06551_gb300 import build_lib
    build_lib.build()
    from paper_1707_06551_gb300 import sphere_bie
    return sphere_bie


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(sphere_bie_\w+)\s*\(", txt))
    return sorted(names)


def test_header_declares_the_interface():
    names = declared_functions()
    for f in ("sphere_bie_create", "sphere_bie_apply_operator", "sphere_bie_solve_mobility",
              "sphere_bie_solve_resistance", "sphere_bie_destroy"):
        assert f in names


def test_every_declared_symbol_is_exported(lib):
    L = lib.lib()
    for name in declared_functions():
        assert hasattr(L, name), name


def test_default_opts(lib):
    o = lib.sphere_bie_default_opts()
    assert (o.p, o.eta, o.prec, o.tol, o.restart, o.max_iter, o.mem_kind) == (8, 1.0, 0, 1e-8, 60, 600, 0)


@pytest.mark.parametrize("case,status", [
    ("overlap", 2), ("p0", 1), ("p25", 1), ("radius", 1), ("nan", 1), ("learned", 1), ("tol", 1), ("empty", 1),
])
def test_create_rejects_bad_input_before_any_device_work(lib, case, status):
    c = np.array([[0.0, 0, 0], [3.0, 0, 0]])
    a = np.array([1.0, 1.0])
    o = lib.make_opts(4)
    if case == "overlap":
        c[1, 0] = 1.5
    elif case == "p0":
        o.p = 0
    elif case == "p25":
        o.p = 25
    elif case == "radius":
        a[1] = 0.0
    elif case == "nan":
        c[0, 1] = np.nan
    elif case == "learned":
        o.use_learned_precond = 1
    elif case == "tol":
        o.tol = 0.0
    h = ctypes.c_void_p()
    n = 0 if case == "empty" else 2
    st = lib.lib().sphere_bie_create(n, lib._ptr(c), lib._ptr(a), ctypes.byref(o), ctypes.byref(h))
    assert st == status
    assert not h.value
    assert len(lib.sphere_bie_last_error(None)) > 0


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lib.SphereBIEError) as e:
        lib.sphere_bie_create(np.zeros((1, 3)), np.ones(1), lib.make_opts(3))
    assert e.value.status == lib.SBIE_ERR_CUDA


def test_binding_rejects_wrong_dtypes(lib):
    with pytest.raises(ValueError):
        lib._ptr(np.zeros(3, dtype=np.float32))
    with pytest.raises(ValueError):
        lib._ptr(np.zeros((3, 3))[:, 0])


def test_create_batch_rejects_bad_input(lib):
    c = np.array([[0.0, 0, 0], [3.0, 0, 0], [10.0, 0, 0]])
    a = np.ones(3)
    o = lib.make_opts(4)
    h = ctypes.c_void_p()
    for ns, ps, status in (([2, 1], [4, 30], 1), ([2, 0], [4, 4], 1), ([0, 3], [4, 4], 1)):
        n = np.array(ns, dtype=np.int32)
        p = np.array(ps, dtype=np.int32)
        st = lib.lib().sphere_bie_create_batch(2, ctypes.c_void_p(n.ctypes.data), ctypes.c_void_p(p.ctypes.data),
                                               lib._ptr(c), lib._ptr(a), ctypes.byref(o), ctypes.byref(h))
        assert st == status
    c[1, 0] = 1.5  # overlap inside problem 0
    n = np.array([2, 1], dtype=np.int32)
    p = np.array([4, 6], dtype=np.int32)
    st = lib.lib().sphere_bie_create_batch(2, ctypes.c_void_p(n.ctypes.data), ctypes.c_void_p(p.ctypes.data),
                                           lib._ptr(c), lib._ptr(a), ctypes.byref(o), ctypes.byref(h))
    assert st == 2


def test_default_opts_use_graphs(lib):
    assert lib.sphere_bie_default_opts().use_graphs == 1


@pytest.mark.parametrize("case", ["missing", "not_a_net", "graphs"])
def test_create_rejects_bad_preconditioner_and_graph_options(lib, tmp_path, case):
    """Checked on the host before any device work: the weights file of the
    learned preconditioner is read at create, and use_graphs must be 0 or 1."""
    c = np.array([[0.0, 0, 0], [3.0, 0, 0]])
    a = np.array([1.0, 1.0])
    o = lib.make_opts(4)
    keep = None
    if case == "missing":
        o.use_learned_precond = 1
        keep = str(tmp_path / "absent.bin").encode()
        o.mlp_weights_path = keep
    elif case == "not_a_net":
        bad = tmp_path / "bad.bin"
        bad.write_bytes(b"SBIEPN00" + b"\0" * 64)
        o.use_learned_precond = 1
        keep = str(bad).encode()
        o.mlp_weights_path = keep
    else:
        o.use_graphs = 2
    h = ctypes.c_void_p()
    st = lib.lib().sphere_bie_create(2, lib._ptr(c), lib._ptr(a), ctypes.byref(o), ctypes.byref(h))
    assert st == lib.SBIE_ERR_ARG and not h.value
    msg = lib.sphere_bie_last_error(None)
    assert ("pair-network" in msg or "cannot read" in msg) if case != "graphs" else "use_graphs" in msg


@pytest.mark.parametrize("scheme", [2, -1, 7])
def test_create_rejects_bad_close_pair_scheme(lib, scheme):
    """near_scheme is 0 (direct) or 1 (rotated, Sec. 4.2), checked on the host
    before any device work, for single contexts and batches."""
    c = np.array([[0.0, 0, 0], [3.0, 0, 0]])
    a = np.array([1.0, 1.0])
    o = lib.make_opts(4, near_scheme=scheme)
    h = ctypes.c_void_p()
    st = lib.lib().sphere_bie_create(2, lib._ptr(c), lib._ptr(a), ctypes.byref(o), ctypes.byref(h))
    assert st == lib.SBIE_ERR_ARG and not h.value
    assert "near_scheme" in lib.sphere_bie_last_error(None)
    n = np.array([1, 1], dtype=np.int32)
    pp = np.array([4, 6], dtype=np.int32)
    st = lib.lib().sphere_bie_create_batch(2, ctypes.c_void_p(n.ctypes.data), ctypes.c_void_p(pp.ctypes.data),
                                           lib._ptr(c), lib._ptr(a), ctypes.byref(o), ctypes.byref(h))
    assert st == lib.SBIE_ERR_ARG and not h.value


@pytest.mark.parametrize("field,value", [("ops", 0), ("ops", 4), ("radius_max", 0.5), ("n_samples", 8),
                                         ("p", 3), ("val_frac", 0.95)])
def test_train_pair_network_rejects_bad_options(lib, tmp_path, field, value):
    o = lib.PairTrainOpts(64, 6, 0.01, 0.5, 1.0, 10, 32, 2e-3, 7, 0.1, 1, 1.0)
    setattr(o, field, value)
    info = lib.PairTrainInfo()
    st = lib.lib().sphere_bie_train_pair_network(ctypes.byref(o), str(tmp_path / "n.bin").encode(), ctypes.byref(info))
    assert st == lib.SBIE_ERR_ARG
    assert not (tmp_path / "n.bin").exists()


def test_every_context_entry_point_rejects_a_null_context(lib):
    """Each call that takes a context checks it before touching it (no device
    work, no crash); destroy(NULL) is a no-op and last_error(NULL) returns the
    library's own last message."""
    L = lib.lib()
    buf = (ctypes.c_double * 64)()
    n = ctypes.c_longlong(0)
    calls = {
        "num_nodes": lambda: L.sphere_bie_num_nodes(None, ctypes.byref(n)),
        "nodes": lambda: L.sphere_bie_nodes(None, buf, buf, buf),
        "apply_operator": lambda: L.sphere_bie_apply_operator(None, 0, buf, buf),
        "solve_mobility": lambda: L.sphere_bie_solve_mobility(None, buf, buf, buf, buf, None),
        "solve_resistance": lambda: L.sphere_bie_solve_resistance(None, buf, buf, None, None, buf, buf, None),
        "solve_porous": lambda: L.sphere_bie_solve_porous(None, None, None, buf, buf, None),
        "solve_squirmer": lambda: L.sphere_bie_solve_squirmer(None, buf, buf, buf, None),
        "apply_laplace": lambda: L.sphere_bie_apply_laplace(None, 0, buf, buf),
        "solve_mhd": lambda: L.sphere_bie_solve_mhd(None, buf, 0.5, buf, buf, buf, buf, None),
        "autotune": lambda: L.sphere_bie_autotune(None, 4, None),
        "profile": lambda: L.sphere_bie_profile(None, 1),
        "profile_read": lambda: L.sphere_bie_profile_read(None, None),
        "solution_density": lambda: L.sphere_bie_solution_density(None, buf),
        "precond_info": lambda: L.sphere_bie_precond_info(None, 4, None, None, None, None),
    }
    for name, call in calls.items():
        assert call() == lib.SBIE_ERR_ARG, name
    assert L.sphere_bie_destroy(None) == 0
    assert isinstance(L.sphere_bie_last_error(None), bytes)


def test_context_free_entry_points_reject_bad_arguments(lib):
    L = lib.lib()
    d = (ctypes.c_double * 8)(2.5)
    out = (ctypes.c_double * (73 * 73))()
    assert L.sphere_bie_pair_blocks(0, d, d, d, 10, 4, out) == lib.SBIE_ERR_ARG       # no pairs
    assert L.sphere_bie_pair_blocks(1, d, d, d, 3, 4, out) == lib.SBIE_ERR_ARG       # p below degree 4
    assert L.sphere_bie_pair_blocks(1, d, d, d, 10, 0, out) == lib.SBIE_ERR_ARG      # not a solve operator
    assert L.sphere_bie_pair_blocks(1, None, d, d, 10, 4, out) == lib.SBIE_ERR_ARG
    f = (ctypes.c_float * 8)()
    loss = ctypes.c_double(0)
    assert L.sphere_bie_pair_network_gradients(None, 1, f, f, f, ctypes.byref(loss)) == lib.SBIE_ERR_ARG
    assert L.sphere_bie_pair_network_gradients(f, 0, f, f, f, ctypes.byref(loss)) == lib.SBIE_ERR_ARG
    assert L.sphere_bie_pair_network_size(None) == lib.SBIE_ERR_ARG
