"""ctypes binding of include/sphere_bie.h (argument marshalling only).

Every function has the C name and forwards to libsphere_bie.so; arrays are
numpy float64 (host memory, opts.mem_kind = 0) or torch float64 CUDA tensors
(device memory, opts.mem_kind = 1), passed as raw pointers.  If the library
has not been built this module raises; there is no other implementation to
fall back to.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsphere_bie.so")

SBIE_OK, SBIE_ERR_ARG, SBIE_ERR_OVERLAP, SBIE_ERR_CUDA, SBIE_ERR_OOM = 0, 1, 2, 3, 4
SBIE_ERR_NOT_CONVERGED, SBIE_ERR_TIMEOUT, SBIE_ERR_NUMERIC = 5, 6, 7
STATUS_NAMES = {0: "SBIE_OK", 1: "SBIE_ERR_ARG", 2: "SBIE_ERR_OVERLAP", 3: "SBIE_ERR_CUDA", 4: "SBIE_ERR_OOM",
                5: "SBIE_ERR_NOT_CONVERGED", 6: "SBIE_ERR_TIMEOUT", 7: "SBIE_ERR_NUMERIC"}
SBIE_FP64, SBIE_MIXED, SBIE_FP64_DF = 0, 1, 2
SBIE_OP_S, SBIE_OP_D, SBIE_OP_K, SBIE_OP_MOBILITY, SBIE_OP_RESISTANCE = 0, 1, 2, 3, 4
SBIE_OP_POROUS, SBIE_OP_SQUIRMER = 5, 6
OPS = {"S": 0, "D": 1, "K": 2, "mobility": 3, "resistance": 4, "porous": 5, "squirmer": 6}
STAGES = ("far", "near", "self", "completion", "arnoldi", "precond", "far_kernel_f32", "far_kernel_f64")


class Opts(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("eta", ctypes.c_double), ("prec", ctypes.c_int), ("tol", ctypes.c_double),
                ("restart", ctypes.c_int), ("max_iter", ctypes.c_int), ("use_learned_precond", ctypes.c_int),
                ("mlp_weights_path", ctypes.c_char_p), ("mem_kind", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("use_graphs", ctypes.c_int), ("near_scheme", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("restarts", ctypes.c_int), ("refinements", ctypes.c_int),
                ("rel_residual_true", ctypes.c_double), ("t_setup_ms", ctypes.c_double),
                ("t_solve_ms", ctypes.c_double), ("n_near_pairs", ctypes.c_longlong),
                ("graph_cycles", ctypes.c_int), ("kernel_launches", ctypes.c_longlong),
                ("fp32_residual_updates", ctypes.c_int), ("fp32_op_err", ctypes.c_double),
                ("last_correction", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 8), ("launches", ctypes.c_longlong * 8),
                ("far_pairs_f32", ctypes.c_longlong), ("far_pairs_f64", ctypes.c_longlong),
                ("kernel_launches", ctypes.c_longlong), ("arnoldi_vectors", ctypes.c_longlong)]


class FarTuning(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int), ("targets_per_thread", ctypes.c_int), ("split", ctypes.c_int),
                ("tile", ctypes.c_int), ("ms", ctypes.c_double), ("candidates", ctypes.c_int),
                ("min_blocks", ctypes.c_int)]


class PairTrainOpts(ctypes.Structure):
    _fields_ = [("n_samples", ctypes.c_int), ("p", ctypes.c_int), ("gap_min", ctypes.c_double),
                ("gap_max", ctypes.c_double), ("radius", ctypes.c_double), ("epochs", ctypes.c_int),
                ("batch", ctypes.c_int), ("lr", ctypes.c_double), ("seed", ctypes.c_ulonglong),
                ("val_frac", ctypes.c_double), ("ops", ctypes.c_int), ("radius_max", ctypes.c_double)]


class PairTrainInfo(ctypes.Structure):
    _fields_ = [("train_loss", ctypes.c_double), ("val_rel_err", ctypes.c_double), ("t_data_s", ctypes.c_double),
                ("t_train_s", ctypes.c_double), ("n_train", ctypes.c_int), ("n_val", ctypes.c_int)]


class SphereBIEError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        L.sphere_bie_default_opts.argtypes = [ctypes.POINTER(Opts)]
        L.sphere_bie_create.argtypes = [ctypes.c_int, _P, _P, ctypes.POINTER(Opts), ctypes.POINTER(_P)]
        L.sphere_bie_create_batch.argtypes = [ctypes.c_int, _P, _P, _P, _P, ctypes.POINTER(Opts), ctypes.POINTER(_P)]
        L.sphere_bie_num_nodes.argtypes = [_P, ctypes.POINTER(ctypes.c_longlong)]
        L.sphere_bie_nodes.argtypes = [_P, _P, _P, _P]
        L.sphere_bie_apply_operator.argtypes = [_P, ctypes.c_int, _P, _P]
        L.sphere_bie_solve_mobility.argtypes = [_P, _P, _P, _P, _P, ctypes.POINTER(SolveInfo)]
        L.sphere_bie_solve_resistance.argtypes = [_P, _P, _P, _P, _P, _P, _P, ctypes.POINTER(SolveInfo)]
        L.sphere_bie_solve_porous.argtypes = [_P, _P, _P, _P, _P, ctypes.POINTER(SolveInfo)]
        L.sphere_bie_solve_squirmer.argtypes = [_P, _P, _P, _P, ctypes.POINTER(SolveInfo)]
        L.sphere_bie_apply_laplace.argtypes = [_P, ctypes.c_int, _P, _P]
        L.sphere_bie_solve_mhd.argtypes = [_P, _P, ctypes.c_double, _P, _P, _P, _P, ctypes.POINTER(SolveInfo)]
        L.sphere_bie_fp32_peak_probe.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        L.sphere_bie_destroy.argtypes = [_P]
        L.sphere_bie_last_error.argtypes = [_P]
        L.sphere_bie_last_error.restype = ctypes.c_char_p
        L.sphere_bie_profile.argtypes = [_P, ctypes.c_int]
        L.sphere_bie_profile_read.argtypes = [_P, ctypes.POINTER(Profile)]
        L.sphere_bie_train_pair_network.argtypes = [ctypes.POINTER(PairTrainOpts), ctypes.c_char_p,
                                                    ctypes.POINTER(PairTrainInfo)]
        L.sphere_bie_pair_blocks.argtypes = [ctypes.c_int, _P, _P, _P, ctypes.c_int, ctypes.c_int, _P]
        L.sphere_bie_pair_network_size.argtypes = [ctypes.POINTER(ctypes.c_longlong)]
        L.sphere_bie_solution_density.argtypes = [_P, _P]
        L.sphere_bie_precond_info.argtypes = [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                              ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                              ctypes.POINTER(ctypes.c_double)]
        L.sphere_bie_pair_network_gradients.argtypes = [_P, ctypes.c_int, _P, _P, _P, ctypes.POINTER(ctypes.c_double)]
        L.sphere_bie_autotune.argtypes = [_P, ctypes.c_int, ctypes.POINTER(FarTuning)]
        L.sphere_bie_apply_layer_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P, _P]
        for f in ("sphere_bie_default_opts", "sphere_bie_create", "sphere_bie_create_batch", "sphere_bie_num_nodes",
                  "sphere_bie_nodes",
                  "sphere_bie_apply_operator", "sphere_bie_solve_mobility", "sphere_bie_solve_resistance",
                  "sphere_bie_solve_porous", "sphere_bie_solve_squirmer", "sphere_bie_fp32_peak_probe",
                  "sphere_bie_apply_laplace", "sphere_bie_solve_mhd",
                  "sphere_bie_destroy", "sphere_bie_profile", "sphere_bie_profile_read",
                  "sphere_bie_apply_layer_noalloc", "sphere_bie_autotune", "sphere_bie_train_pair_network",
                  "sphere_bie_pair_blocks", "sphere_bie_pair_network_size", "sphere_bie_pair_network_gradients",
                  "sphere_bie_precond_info", "sphere_bie_solution_density"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a, nullable=False):
    """Raw pointer of a C-contiguous float64 numpy array or torch tensor."""
    if a is None:
        if nullable:
            return None
        raise ValueError("array required")
    if hasattr(a, "data_ptr"):  # torch tensor
        if str(a.dtype) != "torch.float64" or not a.is_contiguous():
            raise ValueError("torch tensors must be contiguous float64")
        return ctypes.c_void_p(a.data_ptr())
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]):
        raise ValueError("numpy arrays must be C-contiguous float64")
    return ctypes.c_void_p(a.ctypes.data)


def _check(ctx, status, allow=()):
    if status != SBIE_OK and status not in allow:
        msg = lib().sphere_bie_last_error(ctx).decode()
        raise SphereBIEError(status, msg)
    return status


def sphere_bie_default_opts():
    o = Opts()
    _check(None, lib().sphere_bie_default_opts(ctypes.byref(o)))
    return o


def make_opts(p, eta=1.0, prec=SBIE_FP64, tol=1e-8, restart=60, max_iter=600, mem_kind=0, stream=None, graphs=True,
              near_scheme=0):
    o = sphere_bie_default_opts()
    o.p, o.eta, o.prec, o.tol, o.restart, o.max_iter, o.mem_kind = p, eta, prec, tol, restart, max_iter, mem_kind
    o.stream = stream
    o.use_graphs = 1 if graphs else 0
    o.near_scheme = int(near_scheme)
    return o


def sphere_bie_create(centres, radii, opts):
    c = np.ascontiguousarray(centres, dtype=np.float64).reshape(-1, 3)
    a = np.ascontiguousarray(radii, dtype=np.float64).reshape(-1)
    if len(c) != len(a):
        raise ValueError("centres and radii disagree")
    h = _P()
    _check(None, lib().sphere_bie_create(len(a), _ptr(c), _ptr(a), ctypes.byref(opts), ctypes.byref(h)))
    return h


def sphere_bie_create_batch(centres_list, radii_list, p_list, opts):
    """One context for independent problems; arrays are concatenated in problem order."""
    n = np.ascontiguousarray([len(np.asarray(r).reshape(-1)) for r in radii_list], dtype=np.int32)
    p = np.ascontiguousarray(p_list, dtype=np.int32)
    c = np.ascontiguousarray(np.concatenate([np.asarray(x, float).reshape(-1, 3) for x in centres_list]))
    a = np.ascontiguousarray(np.concatenate([np.asarray(x, float).reshape(-1) for x in radii_list]))
    h = _P()
    _check(None, lib().sphere_bie_create_batch(len(n), ctypes.c_void_p(n.ctypes.data), ctypes.c_void_p(p.ctypes.data),
                                               _ptr(c), _ptr(a), ctypes.byref(opts), ctypes.byref(h)))
    return h


def sphere_bie_num_nodes(ctx):
    n = ctypes.c_longlong()
    _check(ctx, lib().sphere_bie_num_nodes(ctx, ctypes.byref(n)))
    return n.value


def sphere_bie_nodes(ctx):
    N = sphere_bie_num_nodes(ctx)
    x = np.zeros((N, 3))
    nr = np.zeros((N, 3))
    w = np.zeros(N)
    _check(ctx, lib().sphere_bie_nodes(ctx, _ptr(x), _ptr(nr), _ptr(w)))
    return x, nr, w


def sphere_bie_apply_operator(ctx, op, density, out):
    op = OPS[op] if isinstance(op, str) else int(op)
    _check(ctx, lib().sphere_bie_apply_operator(ctx, op, _ptr(density), _ptr(out)))
    return out


def sphere_bie_solve_mobility(ctx, forces, torques, vel, omega):
    info = SolveInfo()
    st = _check(ctx, lib().sphere_bie_solve_mobility(ctx, _ptr(forces), _ptr(torques), _ptr(vel), _ptr(omega),
                                                     ctypes.byref(info)), allow=(SBIE_ERR_NOT_CONVERGED,))
    d = info.as_dict()
    d["status"] = st
    return d


def sphere_bie_solve_resistance(ctx, vel, omega, bg_u0, bg_grad, forces, torques):
    info = SolveInfo()
    u0 = None if bg_u0 is None else np.ascontiguousarray(bg_u0, dtype=np.float64).reshape(3)
    G = None if bg_grad is None else np.ascontiguousarray(bg_grad, dtype=np.float64).reshape(3, 3)
    st = _check(ctx, lib().sphere_bie_solve_resistance(ctx, _ptr(vel), _ptr(omega), _ptr(u0, True), _ptr(G, True),
                                                       _ptr(forces), _ptr(torques), ctypes.byref(info)),
                allow=(SBIE_ERR_NOT_CONVERGED,))
    d = info.as_dict()
    d["status"] = st
    return d


def sphere_bie_solve_porous(ctx, bg_u0, bg_grad, forces, torques):
    info = SolveInfo()
    u0 = None if bg_u0 is None else np.ascontiguousarray(bg_u0, dtype=np.float64).reshape(3)
    G = None if bg_grad is None else np.ascontiguousarray(bg_grad, dtype=np.float64).reshape(3, 3)
    st = _check(ctx, lib().sphere_bie_solve_porous(ctx, _ptr(u0, True), _ptr(G, True), _ptr(forces), _ptr(torques),
                                                   ctypes.byref(info)), allow=(SBIE_ERR_NOT_CONVERGED,))
    d = info.as_dict()
    d["status"] = st
    return d


def sphere_bie_solve_squirmer(ctx, slip, vel, omega):
    info = SolveInfo()
    st = _check(ctx, lib().sphere_bie_solve_squirmer(ctx, _ptr(slip), _ptr(vel), _ptr(omega), ctypes.byref(info)),
                allow=(SBIE_ERR_NOT_CONVERGED,))
    d = info.as_dict()
    d["status"] = st
    return d


def sphere_bie_apply_layer_noalloc(op, n_spheres, p, centres, radii, density, out, stream=None):
    """CUDA float64 tensors only; see the header for limits and the shared scratch."""
    op = OPS[op] if isinstance(op, str) else int(op)
    for name, a in (("centres", centres), ("radii", radii), ("density", density), ("out", out)):
        if not (hasattr(a, "is_cuda") and a.is_cuda):
            raise ValueError(f"sphere_bie_apply_layer_noalloc: {name} must be a CUDA tensor")
    _check(None, lib().sphere_bie_apply_layer_noalloc(op, int(n_spheres), int(p), _ptr(centres), _ptr(radii),
                                                      _ptr(density), _ptr(out), stream))
    return out


LAPLACE_OPS = {"SL": 0, "DL": 1, "KL": 2}


def sphere_bie_apply_laplace(ctx, op, q, out):
    op = LAPLACE_OPS[op] if isinstance(op, str) else int(op)
    _check(ctx, lib().sphere_bie_apply_laplace(ctx, op, _ptr(q), _ptr(out)))
    return out


def sphere_bie_solve_mhd(ctx, H0, eta, forces, torques, vel, omega):
    info = SolveInfo()
    h = np.ascontiguousarray(H0, dtype=np.float64).reshape(3)
    st = _check(ctx, lib().sphere_bie_solve_mhd(ctx, _ptr(h), float(eta), _ptr(forces), _ptr(torques), _ptr(vel),
                                                _ptr(omega), ctypes.byref(info)), allow=(SBIE_ERR_NOT_CONVERGED,))
    d = info.as_dict()
    d["status"] = st
    return d


def sphere_bie_fp32_peak_probe():
    """Measured FP32 TFLOP/s of the current device and the probe launch (ms)."""
    t, ms = ctypes.c_double(0), ctypes.c_double(0)
    _check(None, lib().sphere_bie_fp32_peak_probe(ctypes.byref(t), ctypes.byref(ms)))
    return t.value, ms.value


def sphere_bie_destroy(ctx):
    if ctx:
        _check(None, lib().sphere_bie_destroy(ctx))


def sphere_bie_last_error(ctx=None):
    return lib().sphere_bie_last_error(ctx).decode()


def sphere_bie_autotune(ctx, op):
    op = OPS[op] if isinstance(op, str) else int(op)
    t = (FarTuning * 2)()
    _check(ctx, lib().sphere_bie_autotune(ctx, op, t))
    return {name: {k: getattr(t[i], k) for k, _ in FarTuning._fields_} for i, name in enumerate(("fp32", "df"))}


def sphere_bie_train_pair_network(path, n_samples=4096, p=10, gap_min=0.01, gap_max=0.5, radius=1.0, epochs=200,
                                  batch=256, lr=2e-3, seed=7, val_frac=0.1, ops=("resistance",), radius_max=None):
    bits = sum({"resistance": 1, "mobility": 2}[o] for o in ops)
    o = PairTrainOpts(n_samples, p, gap_min, gap_max, radius, epochs, batch, lr, seed, val_frac, bits,
                      radius if radius_max is None else radius_max)
    info = PairTrainInfo()
    _check(None, lib().sphere_bie_train_pair_network(ctypes.byref(o), str(path).encode(), ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in info._fields_}


def sphere_bie_pair_blocks(dist, a_src, a_tgt, p, op="resistance"):
    d = np.ascontiguousarray(dist, dtype=np.float64).reshape(-1)
    s = np.ascontiguousarray(np.broadcast_to(a_src, d.shape), dtype=np.float64)
    t = np.ascontiguousarray(np.broadcast_to(a_tgt, d.shape), dtype=np.float64)
    out = np.zeros((len(d), 73, 73))
    op = OPS[op] if isinstance(op, str) else int(op)
    _check(None, lib().sphere_bie_pair_blocks(len(d), _ptr(d), _ptr(s), _ptr(t), int(p), op, _ptr(out)))
    return out


def sphere_bie_solution_density(ctx, out):
    _check(ctx, lib().sphere_bie_solution_density(ctx, _ptr(out)))
    return out


def sphere_bie_precond_info(ctx, op="resistance"):
    op = OPS[op] if isinstance(op, str) else int(op)
    k, npairs, nd, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(ctx, lib().sphere_bie_precond_info(ctx, op, ctypes.byref(k), ctypes.byref(npairs), ctypes.byref(nd),
                                              ctypes.byref(ms)))
    return {"kind": k.value, "pairs": npairs.value, "dropped": nd.value, "setup_ms": ms.value}


def sphere_bie_pair_network_size():
    n = ctypes.c_longlong()
    _check(None, lib().sphere_bie_pair_network_size(ctypes.byref(n)))
    return n.value


def sphere_bie_pair_network_gradients(params, X, Y):
    params = np.ascontiguousarray(params, dtype=np.float32)
    X = np.ascontiguousarray(X, dtype=np.float32)
    Y = np.ascontiguousarray(Y, dtype=np.float32)
    g = np.zeros_like(params)
    loss = ctypes.c_double()
    fp = lambda a: ctypes.c_void_p(a.ctypes.data)
    _check(None, lib().sphere_bie_pair_network_gradients(fp(params), len(X), fp(X), fp(Y), fp(g), ctypes.byref(loss)))
    return loss.value, g


def sphere_bie_profile(ctx, enable):
    _check(ctx, lib().sphere_bie_profile(ctx, int(enable)))


def sphere_bie_profile_read(ctx):
    p = Profile()
    _check(ctx, lib().sphere_bie_profile_read(ctx, ctypes.byref(p)))
    return {"ms": dict(zip(STAGES, list(p.ms))), "launches": dict(zip(STAGES, list(p.launches))),
            "far_pairs_f32": p.far_pairs_f32, "far_pairs_f64": p.far_pairs_f64,
            "kernel_launches": p.kernel_launches, "arnoldi_vectors": p.arnoldi_vectors}


class SphereBIE:
    """Owning wrapper around a context (host memory interface).  With
    `batch=[(centres, radii, p), ...]` it holds a batch of problems."""

    def __init__(self, centres=None, radii=None, p=None, eta=1.0, prec=SBIE_FP64, tol=1e-8, restart=60, max_iter=600,
                 batch=None, precond=0, weights=None, graphs=True, near_scheme=0):
        self.opts = make_opts(p if p is not None else batch[0][2], eta, prec, tol, restart, max_iter, 0,
                              graphs=graphs, near_scheme=near_scheme)
        self.opts.use_learned_precond = precond
        self._wpath = None if weights is None else str(weights).encode()
        self.opts.mlp_weights_path = self._wpath
        if batch is None:
            self.ctx = sphere_bie_create(centres, radii, self.opts)
            self.n = len(np.asarray(radii).reshape(-1))
        else:
            self.ctx = sphere_bie_create_batch([x[0] for x in batch], [x[1] for x in batch], [x[2] for x in batch],
                                               self.opts)
            self.n = sum(len(np.asarray(x[1]).reshape(-1)) for x in batch)
        self.N = sphere_bie_num_nodes(self.ctx)

    def apply(self, op, density):
        d = np.ascontiguousarray(density, dtype=np.float64).reshape(-1, 3)
        out = np.zeros_like(d)
        return sphere_bie_apply_operator(self.ctx, op, d, out)

    def mobility(self, F, T):
        F = np.ascontiguousarray(F, dtype=np.float64).reshape(-1, 3)
        T = np.ascontiguousarray(T, dtype=np.float64).reshape(-1, 3)
        v = np.zeros_like(F)
        w = np.zeros_like(T)
        info = sphere_bie_solve_mobility(self.ctx, F, T, v, w)
        return v, w, info

    def resistance(self, v, w, u0=None, G=None):
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1, 3)
        w = np.ascontiguousarray(w, dtype=np.float64).reshape(-1, 3)
        F = np.zeros_like(v)
        T = np.zeros_like(w)
        info = sphere_bie_solve_resistance(self.ctx, v, w, u0, G, F, T)
        return F, T, info

    def porous(self, u0=None, G=None):
        F = np.zeros((self.n, 3))
        T = np.zeros((self.n, 3))
        info = sphere_bie_solve_porous(self.ctx, u0, G, F, T)
        return F, T, info

    def squirmer(self, slip):
        s = np.ascontiguousarray(slip, dtype=np.float64).reshape(-1, 3)
        v = np.zeros((self.n, 3))
        w = np.zeros((self.n, 3))
        info = sphere_bie_solve_squirmer(self.ctx, s, v, w)
        return v, w, info

    def laplace(self, op, q):
        qq = np.ascontiguousarray(q, dtype=np.float64).reshape(-1)
        return sphere_bie_apply_laplace(self.ctx, op, qq, np.zeros_like(qq))

    def mhd(self, H0, eta):
        F, T, v, w = (np.zeros((self.n, 3)) for _ in range(4))
        info = sphere_bie_solve_mhd(self.ctx, H0, eta, F, T, v, w)
        return F, T, v, w, info

    def nodes(self):
        return sphere_bie_nodes(self.ctx)

    def density(self):
        return sphere_bie_solution_density(self.ctx, np.zeros((self.N, 3)))

    def close(self):
        if self.ctx:
            sphere_bie_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
