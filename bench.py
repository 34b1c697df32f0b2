#!/usr/bin/env python
"""Benchmark: GMRES time-to-solve at a 1e-8 relative residual for the
resistance workload of 256 unit spheres at volume fraction 0.10 (20% pushed to
gaps 0.05-0.2), VSH order p = 10, in a background shear, mixed precision (FP32
far field and close-pair evaluation, FP64 residuals), plus the far-field pair
rate in FP32 and FP64.

One step = one complete solve: right-hand side, right-preconditioned GMRES
(learned pair preconditioner; each restart cycle one CUDA graph launch) with
FP64-accurate iterative refinement, forces and torques, with the geometry
resident on the device.  The pair network is trained once before anything is
timed; the solve without it, with exact pair blocks and the plain FP64 path
are reported alongside.
Under torchrun every rank solves its own replica (the solve does not shard);
the time reported is the maximum over ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line on rank 0.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GMRES time-to-solve at 1e-8 rel. residual; far-field pair-interactions/s vs FP64"
WORKLOAD = "resistance_256"
FLOP_PER_PAIR = {"S": 28, "D": 30, "K": 30}   # algorithmic flops per (target, source) pair
SM_COUNT_NOMINAL = 152
FP32_LANES_PER_SM = 128
# ncu DRAM traffic (read + write bytes per launch) of the FP32 far-field pair
# kernel on this workload, keyed by the hash of that kernel's source text and
# the tiling (threads x targets per thread / split / tile) it was measured
# with; reported only while both are unchanged.
NCU_TRAFFIC = {"df668ee33ebfad7f/64x4/14/256/mb8": 4257536,  # profiles/far_f32_kernel_resistance_256.md
               "df668ee33ebfad7f/64x4/33/128/mb8": 4912384}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched_512 solve of the headline line")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-precond", action="store_true")
    ap.add_argument("--no-graphs", action="store_true",
                    help="step each GMRES iteration from the host instead of one CUDA graph per restart cycle")
    ap.add_argument("--pair-samples", type=int, default=None,
                    help="two-sphere configurations the pair network is trained on "
                         "(default 4096; 100000 for dense_1024, 20000 for large_4096)")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=[WORKLOAD, "batched_512", "dense_1024", "large_4096", "lattice", "near_schemes"],
                    help="the other configurations print their own JSON line (not the headline)")
    ap.add_argument("--near-p", default="4,6,8,10,12,14,16",
                    help="orders of the near_schemes workload (comma-separated)")
    return ap.parse_args()


def far_source_hash():
    """Hash of the FP32 far-field kernel's source text (from its header comment
    to the double-float section of far.cu): measured traffic stays valid while
    this text is unchanged."""
    with open(os.path.join(ROOT, "paper_1707_06551_gb300", "csrc", "far.cu")) as f:
        src = f.read()
    i = src.index("// FP32 pair kernel on packed FP32x2 arithmetic")
    j = src.index("// ---- double-float", i)
    return hashlib.sha256(src[i:j].encode()).hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clocks / throttle reasons, sampled every 200 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.mark = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                self.rows.append((time.time(), parts))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0, t1):
        rows = [p for (t, p) in self.rows if t0 <= t <= t1] or [p for (_, p) in self.rows]
        if not rows:
            return None
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(p[1]) for p in rows if num(p[1]) is not None]
        mx = [num(p[2]) for p in rows if num(p[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for p in rows for i in range(4) if p[4 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def peak_fp32_tflops(sm_count, mhz):
    return sm_count * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12


def ncu_traffic(t32):
    """Measured DRAM bytes per launch of the FP32 far-field kernel for the
    tiling `t32` (the autotuner's FP32 choice), or None when that tiling or the
    kernel's source text differs from what was measured."""
    key = (f"{far_source_hash()}/{t32.get('threads')}x{t32.get('targets_per_thread')}/"
           f"{t32.get('split')}/{t32.get('tile')}/mb{t32.get('min_blocks')}")
    return NCU_TRAFFIC.get(key)


def self_vsh_rate(prof, n_nodes):
    """Throughput of the operator's self step (VSH analysis, signature,
    synthesis: the density read and the result written, 2 x 3 x N doubles per
    apply) from a profile of solves; None when the profile has no self step."""
    applies, ms = prof["launches"].get("self", 0), prof["ms"].get("self", 0.0)
    if not applies or not ms:
        return None
    per = 2 * 3 * n_nodes * 8
    return {"gb_per_s": per * applies / (ms * 1e-3) / 1e9, "ms_per_apply": ms / applies, "bytes_per_apply": per}


def load_peaks():
    """Measured peaks of the GB300s (HBM copy GB/s, cuBLAS bf16
    TFLOP/s), or the recipe's fallback figures."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]), "source": "measured"}
    except (OSError, ValueError, KeyError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


# Dense TF32 tensor rate relative to BF16 (nominal 1.1 vs 2.25 PFLOP/s per GPU).
TF32_PER_BF16 = 1.1 / 2.25
COMPLETION_FLOP = 32   # one Stokeslet + rotlet evaluation at one node
NEAR_FLOP = 20         # per (target node, source coefficient) term of a close pair


def stage_rooflines(prof, n, p, n_near, n_pairs, fp32_peak, peaks):
    """Achieved rate of each profiled stage against its roofline, from the
    stage times of the profiled solves and the algorithmic work per unit:
      near        ALU: per directed close pair npn x 3 (p+1)^2 x 20 FLOP;
      completion  ALU: N x n Stokeslet + rotlet evaluations x 32 FLOP;
      arnoldi     HBM: (4k + 4) 3N-vectors of FP64 per iteration with k basis vectors;
      self        tensor: 3 (3xTF32) x 2 x (3 npn)^2 x n FLOP per FP32 apply (the
                  stage also holds the FP64 coefficient analysis of the close pairs);
      precond     HBM: the FP32 pair and own inverses, the preconditioner GEMM's
                  split matrix and 4 nodal vectors per apply."""
    npn = (p + 1) * (2 * p + 2)
    N = n * npn
    ms, la = prof["ms"], prof["launches"]
    out = {}

    def rate(work, t_ms):
        return work / (t_ms * 1e-3) if t_ms > 0 else None

    if la.get("near") and ms.get("near"):
        w = n_near * npn * 3 * (p + 1) ** 2 * NEAR_FLOP * la["near"]
        a = rate(w, ms["near"]) / 1e12
        out["near"] = {"bound": "alu", "achieved": a, "peak": fp32_peak, "unit": "TFLOP/s", "frac": a / fp32_peak,
                       "flop_per_apply": w / la["near"], "ms_per_apply": ms["near"] / la["near"]}
    if la.get("completion") and ms.get("completion"):
        w = N * n * COMPLETION_FLOP * la["completion"]
        a = rate(w, ms["completion"]) / 1e12
        out["completion"] = {"bound": "alu", "achieved": a, "peak": fp32_peak, "unit": "TFLOP/s",
                             "frac": a / fp32_peak, "ms_per_apply": ms["completion"] / la["completion"]}
    if prof.get("arnoldi_vectors") and ms.get("arnoldi"):
        b = prof["arnoldi_vectors"] * 3 * N * 8
        a = rate(b, ms["arnoldi"]) / 1e9
        out["arnoldi"] = {"bound": "hbm", "achieved": a, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                          "frac": a / peaks["hbm_gbs"], "bytes": b, "note": "Krylov basis of one cycle fits L2"}
    if la.get("self") and ms.get("self"):
        K = 3 * npn
        w = 3 * 2 * K * K * n * la["self"]
        tf32_peak = peaks["bf16_tflops"] * TF32_PER_BF16
        a = rate(w, ms["self"]) / 1e12
        out["self"] = {"bound": "tensor", "achieved": a, "peak": tf32_peak, "unit": "TFLOP/s", "frac": a / tf32_peak,
                       "peak_basis": "bf16 %s x 1.1/2.25 (TF32 / BF16 nominal)" % peaks["source"],
                       "ms_per_apply": ms["self"] / la["self"]}
    if la.get("precond") and ms.get("precond") and n_pairs is not None:
        K = 3 * npn
        b = (n_pairs * 146 * 146 * 4 + n * 73 * 73 * 4 + 2 * (K + 73) * ((K + 31) // 32 * 32) * 4 + 4 * 3 * N * 8)
        a = rate(b * la["precond"], ms["precond"]) / 1e9
        out["precond"] = {"bound": "hbm", "achieved": a, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                          "frac": a / peaks["hbm_gbs"], "bytes_per_apply": b,
                          "ms_per_apply": ms["precond"] / la["precond"]}
    return out


def max_over_ranks(torch, dist, world, x, device):
    """The maximum of x over the ranks (N independent replicas are done when
    the slowest is); x itself on a single rank."""
    if world <= 1:
        return x
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def train_pair_network(sb, w, samples):
    """Exact two-sphere low-mode blocks for the workload's close-pair gaps
    (close if gap < eta 2 max(a), eta = 1) and the network trained on them."""
    import tempfile
    gap_max = 2.0 * float(max(w["radii"]))
    tmp = tempfile.mkdtemp()
    path = os.path.join(tmp, "pairnet.bin")
    tr = sb.sphere_bie_train_pair_network(path, n_samples=samples, p=w["p"], gap_min=0.01, gap_max=gap_max,
                                          radius=float(w["radii"][0]), epochs=200, seed=7)
    return {"path": path, "path_bytes": path.encode(), "dir": tmp,
            "report": {"samples": samples, "gap_range": [0.01, gap_max], "val_rel_err": tr["val_rel_err"],
                       "train_loss": tr["train_loss"], "data_s": tr["t_data_s"], "train_s": tr["t_train_s"]}}


def precond_compare(sb, torch, w, prec, stream, vel, om, F_ref, base, net):
    """The same resistance solve without the pair preconditioner and with
    exact pair blocks, next to the learned blocks of the timed solves."""
    p = w["p"]
    out = {"learned": {"iters": base["iters"], "refinements": base["refinements"]}, "network": net["report"]}
    for kind, name in ((0, "none"), (2, "exact")):
        o = sb.make_opts(p, prec=prec, tol=w["tol"], mem_kind=1, stream=stream.cuda_stream)
        o.use_learned_precond = kind
        t0 = time.perf_counter()
        ctx = sb.sphere_bie_create(w["centres"], w["radii"], o)
        t_create = time.perf_counter() - t0
        if prec == sb.SBIE_MIXED:
            sb.sphere_bie_autotune(ctx, "resistance")
        F = torch.zeros_like(F_ref)
        T = torch.zeros_like(F_ref)
        sb.sphere_bie_solve_resistance(ctx, vel, om, w["u0"], w["G"], F, T)  # warm-up
        torch.cuda.synchronize()
        ts = []
        for _ in range(2):
            t0 = time.perf_counter()
            info = sb.sphere_bie_solve_resistance(ctx, vel, om, w["u0"], w["G"], F, T)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        pi = sb.sphere_bie_precond_info(ctx)
        out[name] = {"iters": info["iters"], "refinements": info["refinements"], "status": info["status"],
                     "rel_residual_true": info["rel_residual_true"], "time_to_solve_s": min(ts),
                     "create_s": t_create, "precond_setup_s": pi["setup_ms"] / 1e3, "pairs": pi["pairs"],
                     "pairs_out_of_range": pi["dropped"],
                     "force_rel_diff_vs_learned": float((F - F_ref).abs().max() / F_ref.abs().max())}
        sb.sphere_bie_destroy(ctx)
    return out


def graph_compare(sb, torch, wl, w, prec, stream, vel, om, F_ref, t_graph, net):
    """Time-to-solve with each GMRES iteration stepped from the host, against
    the graph-launched cycles of the timed solves; and both on the small
    8-sphere mobility problem, where launch and synchronisation overhead
    dominate."""
    out = {}
    p = w["p"]
    o = sb.make_opts(p, prec=prec, tol=w["tol"], mem_kind=1, stream=stream.cuda_stream, graphs=False)
    if net is not None:
        o.use_learned_precond = 1
        o.mlp_weights_path = net["path_bytes"]
    ctx = sb.sphere_bie_create(w["centres"], w["radii"], o)
    if prec == sb.SBIE_MIXED:
        sb.sphere_bie_autotune(ctx, "resistance")
    F = torch.zeros_like(F_ref)
    T = torch.zeros_like(F_ref)
    sb.sphere_bie_solve_resistance(ctx, vel, om, w["u0"], w["G"], F, T)
    ts = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = sb.sphere_bie_solve_resistance(ctx, vel, om, w["u0"], w["G"], F, T)
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    sb.sphere_bie_destroy(ctx)
    out[WORKLOAD] = {"graph_s": t_graph, "host_stepped_s": statistics.mean(ts), "iters_host_stepped": info["iters"]}
    m8 = wl.mobility_8()
    dev = F_ref.device
    f8 = torch.tensor(m8["forces"], dtype=torch.float64, device=dev)
    t8 = torch.tensor(m8["torques"], dtype=torch.float64, device=dev)
    v8, w8 = torch.zeros_like(f8), torch.zeros_like(t8)
    res = {}
    for graphs in (True, False):
        o = sb.make_opts(m8["p"], prec=sb.SBIE_FP64, tol=m8["tol"], mem_kind=1, stream=stream.cuda_stream,
                         graphs=graphs)
        ctx = sb.sphere_bie_create(m8["centres"], m8["radii"], o)
        sb.sphere_bie_solve_mobility(ctx, f8, t8, v8, w8)
        ts = []
        for _ in range(10):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = sb.sphere_bie_solve_mobility(ctx, f8, t8, v8, w8)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        sb.sphere_bie_destroy(ctx)
        res[graphs] = (statistics.median(ts), info)
    out["mobility_8"] = {"graph_s": res[True][0], "host_stepped_s": res[False][0], "iters": res[True][1]["iters"],
                         "graph_cycles": res[True][1]["graph_cycles"],
                         "kernels_per_solve": res[True][1]["kernel_launches"]}
    return out


def batched_quick(sb, torch, wl, local):
    """One mixed-precision, graph-launched solve of all 512 problems of
    batched_512 in one context (after a warm-up solve that captures the cycle
    graphs), CUDA events on the library's stream: the batched configuration in
    the headline run.  `bench.py --workload batched_512` measures it in full."""
    import numpy as np
    probs = wl.batched_512()
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream()
    cl = [q["centres"] for q in probs]
    rl = [q["radii"] for q in probs]
    pl = [q["p"] for q in probs]
    F = torch.tensor(np.concatenate([q["forces"] for q in probs]), dtype=torch.float64, device=dev)
    T = torch.tensor(np.concatenate([q["torques"] for q in probs]), dtype=torch.float64, device=dev)
    v, om = torch.zeros_like(F), torch.zeros_like(T)
    o = sb.make_opts(pl[0], prec=sb.SBIE_MIXED, tol=1e-8, mem_kind=1, stream=stream.cuda_stream)
    ctx = sb.sphere_bie_create_batch(cl, rl, pl, o)
    sb.sphere_bie_autotune(ctx, "mobility")
    fn = lambda: sb.sphere_bie_solve_mobility(ctx, F, T, v, om)
    fn()
    ts, info = _timed_solves(torch, stream, fn, 1)
    sb.sphere_bie_destroy(ctx)
    return {"time_to_solve_s": ts[0], "problems_per_s": len(probs) / ts[0], "problems": len(probs),
            "spheres": int(sum(len(r) for r in rl)), "iters": info["iters"],
            "rel_residual_true": info["rel_residual_true"], "graph_cycles": info["graph_cycles"],
            "precision": "mixed", "tol": 1e-8}


GOLDEN_SOLVE = os.path.join(ROOT, "tests", "golden", "resistance_256_oracle_solve.json")
ORACLE_GROUPS = 64  # target-sphere groups handed to the worker processes


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


_og = None  # the oracle's geometry in a worker process


def _oracle_init(root):
    global _og
    if root not in sys.path:
        sys.path.insert(0, root)
    from oracle import operators as ops
    from paper_1707_06551_gb300 import workloads as wl
    w = wl.resistance_256()
    _og = ops.Geometry(w["centres"], w["radii"], w["p"])


def _oracle_group(args):
    """The oracle's resistance operator (Eq. 5.19) on one group of target spheres."""
    import numpy as np
    from oracle import operators as ops
    x, group = args
    out = ops.apply_at(_og, "resistance", x, group)
    return group, out[np.concatenate([np.arange(_og.sl(i).start, _og.sl(i).stop) for i in group])]


def oracle_pool(cores):
    """A pool of `cores` worker processes, each holding the oracle's geometry of
    the timed workload (spawned: no worker inherits a CUDA context)."""
    import multiprocessing as mp
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"  # inherited by the workers: one BLAS thread each
    return mp.get_context("spawn").Pool(cores, initializer=_oracle_init, initargs=(ROOT,))


def _oracle_mobility_8():
    """The oracle's full GMRES solve of the 8-sphere mobility problem (p = 6,
    tol 1e-10), timed in a worker process (one core)."""
    from oracle import operators as ops
    from oracle import solve as osolve
    from paper_1707_06551_gb300 import workloads as wl
    m8 = wl.mobility_8()
    g8 = ops.Geometry(m8["centres"], m8["radii"], m8["p"])
    t0 = time.perf_counter()
    _, _, info = osolve.solve_mobility(g8, m8["forces"], m8["torques"], tol=m8["tol"])
    return {"solve_s": time.perf_counter() - t0, "iters": int(info["iters"]), "cores": 1,
            "rel_residual": float(info["rel_residual"])}


def oracle_apply(pool, x, groups):
    """Oracle operator rows of the target-sphere groups, one group per task."""
    return pool.map(_oracle_group, [(x, g) for g in groups])


def golden_solve():
    """Operator-apply count and result of the oracle's own FP64 GMRES solve of
    the timed workload (tests/golden/make_resistance_256_solve.py), or None."""
    try:
        with open(GOLDEN_SOLVE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


def cpu_baseline():
    """The oracle as it stands on every host core: one full resistance_256
    operator apply (all 256 target spheres, all nodes; worker processes over
    target-sphere groups, BLAS single-threaded) and a full oracle GMRES solve of
    the 8-sphere mobility problem (serial), both timed in full.  The solve
    time of the timed workload is the full apply time x the operator applies of
    the oracle's own solve of it (recorded by the golden-solve script)."""
    import numpy as np
    cores = host_cores()
    n = 256
    groups = [list(range(i, n, ORACLE_GROUPS)) for i in range(ORACLE_GROUPS)]
    x = np.random.default_rng(0).normal(size=(n * 242, 3))
    with oracle_pool(cores) as pool:
        pool.map(abs, range(cores))  # workers up and geometry built before the clock starts
        t0 = time.perf_counter()
        rows = oracle_apply(pool, x, groups)
        t_apply = time.perf_counter() - t0
        m8 = pool.apply(_oracle_mobility_8)
    assert sum(len(g) for g, _ in rows) == n
    gs = golden_solve()
    applies = gs["operator_applies"] if gs else None
    return {"apply_s": t_apply, "cores": cores, "applies": applies,
            "solve_iters": gs["iters"] if gs else None, "mobility_8": m8}


def run_reference(args):
    """The oracle on every host core, on the timed workload.  Step s is the
    resistance operator on the target spheres i = s (mod 4), i.e. one quarter
    of a full apply (four consecutive steps make one full apply); the
    time-to-solve is 4 x the mean step time x the operator applies of the
    oracle's own FP64 GMRES solve of this workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    gs = golden_solve()
    if gs is None:
        print(json.dumps({"impl": "reference", "unavailable": "oracle solve record missing: run "
                          "tests/golden/make_resistance_256_solve.py"}))
        return
    cores = host_cores()
    n = 256
    quarters = [[list(range(i, n, ORACLE_GROUPS)) for i in range(q, ORACLE_GROUPS, 4)] for q in range(4)]
    x = np.random.default_rng(0).normal(size=(n * 242, 3))
    ts = []
    with oracle_pool(cores) as pool:
        pool.map(abs, range(cores))
        for s in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            oracle_apply(pool, x, quarters[s % 4])
            if s >= args.warmup:
                ts.append(time.perf_counter() - t0)
    step = statistics.mean(ts)
    applies = gs["operator_applies"]
    per_solve = 4 * step * applies
    sample = (f"each step: the oracle's resistance operator on 64 of the 256 target spheres (a quarter of one "
              f"full apply, quarters in turn) on {cores} host cores; time-to-solve = 4 x mean step x {applies} "
              f"operator applies of the oracle's own FP64 GMRES solve of this workload "
              f"({gs['iters']} iterations at tol {gs['tol']}, recorded by tests/golden/make_resistance_256_solve.py)")
    line = {"impl": "reference", "metric": METRIC, "value": per_solve, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "step": "a quarter of one full oracle operator apply (value is the time-to-solve built from it)",
            "config": {"workload": WORKLOAD, "n_spheres": 256, "p": 10, "nodes": 61952, "tol": 1e-8,
                       "precision": "fp64 (oracle, plain GMRES)", "preconditioner": "none",
                       "parallelism": "replicas x1"},
            "cpu_baseline": {"value": per_solve, "unit": "s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": per_solve, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---- the other configurations (python bench.py --workload NAME) -------------

def _timed_solves(torch, stream, fn, n):
    """n solves timed with CUDA events on the library's stream; returns the
    times (s) and the last solve's info."""
    ts, info = [], None
    for _ in range(n):
        with torch.cuda.stream(stream):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        info = fn()
        with torch.cuda.stream(stream):
            e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    return ts, info


def _clocks(local):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    idx = vis.split(",")[local] if vis and vis.split(",")[0].strip().isdigit() else str(local)
    return ClockSampler(idx)


def run_lattice(args, sb, torch, wl, local):
    """Operator-apply scaling on the cubic lattices of Sec. 6: the double layer
    and the single layer's traction, applied by the FP32 operator of the mixed
    path and (up to 2e11 far-field pairs) by the FP64-accurate double-float
    operator, for loosely (q = 1) and densely (q = 4) packed mono- and
    polydisperse lattices of 1 to 16 units per side, p = 4 and 8.  Times are
    CUDA events on the library's stream around one apply (mean of 3 after one
    warm-up), densities resident on the device."""
    import math
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream()
    series = []
    for poly in (False, True):
        for q in (1, 4):
            for p in (4, 8):
                rec = {"lattice": "poly" if poly else "mono", "q": q, "p": p, "n_b": [], "nodes": [],
                       "far_pairs": [], "D_fp32_s": [], "K_fp32_s": [], "D_df_s": [], "K_df_s": []}
                for m in (1, 2, 4, 8, 16):
                    w = wl.lattice(m, q, poly)
                    n = len(w["radii"])
                    npn = (p + 1) * (2 * p + 2)
                    x = torch.randn((n * npn, 3), dtype=torch.float64, device=dev)
                    y = torch.zeros_like(x)
                    far_pairs = None
                    for prec, tag in ((sb.SBIE_MIXED, "fp32"), (sb.SBIE_FP64_DF, "df")):
                        o = sb.make_opts(p, prec=prec, mem_kind=1, stream=stream.cuda_stream)
                        ctx = sb.sphere_bie_create(w["centres"], w["radii"], o)
                        if tag == "fp32":
                            sb.sphere_bie_profile(ctx, 1)
                            sb.sphere_bie_apply_operator(ctx, "D", x, y)
                            prof = sb.sphere_bie_profile_read(ctx)
                            sb.sphere_bie_profile(ctx, 0)
                            far_pairs = prof["far_pairs_f32"]
                        if tag == "df" and far_pairs > 2e11:
                            rec["D_df_s"].append(None)
                            rec["K_df_s"].append(None)
                            sb.sphere_bie_destroy(ctx)
                            continue
                        if n * npn >= 100000:
                            sb.sphere_bie_autotune(ctx, "D")
                            sb.sphere_bie_autotune(ctx, "K")
                        for op in ("D", "K"):
                            sb.sphere_bie_apply_operator(ctx, op, x, y)
                            ts, _ = _timed_solves(torch, stream, lambda: sb.sphere_bie_apply_operator(ctx, op, x, y), 3)
                            rec[f"{op}_{tag}_s"].append(statistics.mean(ts))
                        sb.sphere_bie_destroy(ctx)
                    rec["n_b"].append(n)
                    rec["nodes"].append(n * npn)
                    rec["far_pairs"].append(far_pairs)
                    del x, y
                # log-log slope between the two largest lattices
                for key in ("D_fp32_s", "K_fp32_s"):
                    t = rec[key]
                    rec[key.replace("_s", "_slope_last")] = (math.log(t[-1] / t[-2]) /
                                                             math.log(rec["n_b"][-1] / rec["n_b"][-2]))
                series.append(rec)
    return {"metric": "operator apply time vs number of spheres (lattice scaling test)", "unit": "s",
            "higher_is_better": False, "n_gpus": 1, "dtype": "f32 (mixed path operator) / f64-accurate (df)",
            "data": "synthetic", "config": {"workload": "lattice", "units_per_side": [1, 2, 4, 8, 16],
                                            "q": [1, 4], "p": [4, 8], "eta": 1.0},
            "series": series}


def run_near_schemes(args, sb, torch, wl, local):
    """Close-pair stage of one operator apply on dense_1024 (1,024 spheres,
    13,940 directed close pairs) by the direct evaluation at the target nodes
    (near_scheme 0) and by the rotated, FFT-accelerated scheme of Sec. 4.2
    (near_scheme 1), for p = 4 ... 16 and the three layer operators: in FP64
    (the FP64-accurate operator, far field in double-float arithmetic; keys
    without suffix) and in FP32 (the FP32 operator of the mixed path; keys
    `_f32`).  Stage times are CUDA events of the library's profiler (one apply
    after one warm-up) on a smooth density (a random rigid motion of each
    sphere plus four plane waves with wave numbers up to 1,
    `workloads.smooth_density`); `rel_diff` is the largest difference of the
    two schemes' applies relative to the largest value (the rotated scheme
    projects each close-pair field onto degree <= p on the target sphere)."""
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream()
    w = wl.dense_1024()
    rows = []
    for p in [int(v) for v in args.near_p.split(",")]:
        npn = (p + 1) * (2 * p + 2)
        rec = {"p": p}
        outs = {}
        x = None
        for prec, suf in ((sb.SBIE_FP64_DF, ""), (sb.SBIE_MIXED, "_f32")):
            for scheme in (0, 1):
                o = sb.make_opts(p, prec=prec, mem_kind=1, stream=stream.cuda_stream, near_scheme=scheme)
                ctx = sb.sphere_bie_create(w["centres"], w["radii"], o)
                if x is None:
                    nodes, _, _ = sb.sphere_bie_nodes(ctx)
                    x = torch.tensor(wl.smooth_density(nodes, w["centres"], npn, seed=p), dtype=torch.float64,
                                     device=dev)
                for op in ("S", "D", "K"):
                    y = torch.zeros_like(x)
                    sb.sphere_bie_apply_operator(ctx, op, x, y)
                    torch.cuda.synchronize(dev)
                    sb.sphere_bie_profile(ctx, 1)
                    sb.sphere_bie_apply_operator(ctx, op, x, y)
                    prof = sb.sphere_bie_profile_read(ctx)
                    sb.sphere_bie_profile(ctx, 0)
                    rec[f"{op}_near_ms_{'rotated' if scheme else 'direct'}{suf}"] = prof["ms"]["near"]
                    outs[(suf, scheme, op)] = y.clone()
                sb.sphere_bie_destroy(ctx)
            for op in ("S", "D", "K"):
                a, b = outs[(suf, 0, op)], outs[(suf, 1, op)]
                rec[f"{op}_rel_diff{suf}"] = float((a - b).abs().max() / a.abs().max())
                rec[f"{op}_speedup{suf}"] = rec[f"{op}_near_ms_direct{suf}"] / rec[f"{op}_near_ms_rotated{suf}"]
        for op in ("S", "D", "K"):  # FP32 rotated scheme against the FP64 one
            a, b = outs[("", 1, op)], outs[("_f32", 1, op)]
            rec[f"{op}_rotated_f32_vs_f64"] = float((a - b).abs().max() / a.abs().max())
        rows.append(rec)
        del x, outs
    return {"metric": "close-pair stage time per operator apply, direct vs rotated scheme (FP64 and FP32)",
            "unit": "ms", "higher_is_better": False, "n_gpus": 1, "dtype": "f64 / f32", "data": "synthetic",
            "config": {"workload": "near_schemes", "geometry": "dense_1024", "spheres": len(w["radii"]),
                       "p": [r["p"] for r in rows]},
            "rows": rows}


def run_workload(args, sb, torch, wl, local):
    if args.workload == "lattice":
        return run_lattice(args, sb, torch, wl, local)
    if args.workload == "near_schemes":
        return run_near_schemes(args, sb, torch, wl, local)
    if args.workload == "batched_512":
        return run_batched(args, sb, torch, wl, local)
    if args.workload == "dense_1024":
        return run_dense(args, sb, torch, wl, local)
    return run_large(args, sb, torch, wl, local)


def run_batched(args, sb, torch, wl, local):
    """512 independent mobility problems of uneven size and order in one
    context: one solve advances every problem, each restart cycle one CUDA
    graph launch, stopped problems skipped by the far field."""
    import numpy as np
    probs = wl.batched_512()
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream()
    cl = [q["centres"] for q in probs]
    rl = [q["radii"] for q in probs]
    pl = [q["p"] for q in probs]
    F = torch.tensor(np.concatenate([q["forces"] for q in probs]), dtype=torch.float64, device=dev)
    T = torch.tensor(np.concatenate([q["torques"] for q in probs]), dtype=torch.float64, device=dev)
    v, om = torch.zeros_like(F), torch.zeros_like(T)
    nodes = int(sum(len(r) * (p + 1) * (2 * p + 2) for r, p in zip(rl, pl)))
    out = {"metric": "batched mobility time-to-solve at 1e-8 rel. residual (all problems)", "unit": "s",
           "higher_is_better": False, "n_gpus": 1, "dtype": "f32+f64", "data": "synthetic",
           "config": {"workload": "batched_512", "problems": len(probs), "spheres": int(sum(len(r) for r in rl)),
                      "nodes": nodes, "p_values": sorted(set(pl)), "precision": "mixed", "tol": 1e-8}}
    res = {}
    for graphs in (True, False):
        o = sb.make_opts(pl[0], prec=sb.SBIE_MIXED, tol=1e-8, mem_kind=1, stream=stream.cuda_stream, graphs=graphs)
        ctx = sb.sphere_bie_create_batch(cl, rl, pl, o)
        t0 = time.perf_counter()
        sb.sphere_bie_autotune(ctx, "mobility")
        t_tune = time.perf_counter() - t0
        fn = lambda: sb.sphere_bie_solve_mobility(ctx, F, T, v, om)
        fn()  # warm-up (captures the cycle graphs)
        sampler = _clocks(local)
        if graphs:
            sampler.start()
        w0 = time.time()
        ts, info = _timed_solves(torch, stream, fn, args.steps if graphs else 1)
        w1 = time.time()
        res[graphs] = {"time_to_solve_s": statistics.mean(ts), "iters": info["iters"],
                       "refinements": info["refinements"], "rel_residual_true": info["rel_residual_true"],
                       "graph_cycles": info["graph_cycles"], "kernel_launches": info["kernel_launches"],
                       "autotune_s": t_tune}
        if graphs:
            sampler.stop()
            out["clocks"] = sampler.summary(w0, w1)
            sb.sphere_bie_profile(ctx, 1)
            fn()
            prof = sb.sphere_bie_profile_read(ctx)
            sb.sphere_bie_profile(ctx, 0)
            res[graphs]["stage_ms_profiled_solve"] = prof["ms"]
            res[graphs]["far_pairs_per_s_fp32"] = (prof["far_pairs_f32"] / (prof["ms"]["far_kernel_f32"] * 1e-3)
                                                   if prof["ms"]["far_kernel_f32"] > 0 else None)
            vb, wb = v.clone(), om.clone()
        sb.sphere_bie_destroy(ctx)
    # the same problems one context at a time (no batching), graph cycles
    t_sep, it_sep = 0.0, 0
    for q in probs:
        o = sb.make_opts(q["p"], prec=sb.SBIE_MIXED, tol=1e-8, mem_kind=0)
        ctx = sb.sphere_bie_create(q["centres"], q["radii"], o)
        vq, wq = np.zeros_like(q["forces"]), np.zeros_like(q["torques"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        iq = sb.sphere_bie_solve_mobility(ctx, q["forces"], q["torques"], vq, wq)
        t_sep += time.perf_counter() - t0
        it_sep = max(it_sep, iq["iters"])
        sb.sphere_bie_destroy(ctx)
    # FP64-accurate batched solve (double-float far field), one solve
    o = sb.make_opts(pl[0], prec=sb.SBIE_FP64_DF, tol=1e-8, mem_kind=1, stream=stream.cuda_stream)
    ctx = sb.sphere_bie_create_batch(cl, rl, pl, o)
    sb.sphere_bie_autotune(ctx, "mobility")
    ts, idf = _timed_solves(torch, stream, lambda: sb.sphere_bie_solve_mobility(ctx, F, T, v, om), 1)
    sb.sphere_bie_destroy(ctx)
    out["value"] = res[True]["time_to_solve_s"]
    out["problems_per_s"] = len(probs) / out["value"]
    out["graphs"] = res[True]
    out["host_stepped"] = res[False]
    out["one_context_per_problem"] = {"total_time_s": t_sep, "max_iters": it_sep,
                                      "note": "512 separate solves, host buffers, one after another"}
    out["fp64_df_batched"] = {"time_to_solve_s": ts[0], "iters": idf["iters"],
                              "rel_residual_true": idf["rel_residual_true"],
                              "velocity_rel_diff_vs_mixed": float((v - vb).abs().max() / v.abs().max())}
    return out


def _plain_fp64_apply_s(sb, torch, w, stream, op):
    """One FP64 operator apply (the plain FP64 path's unit of work)."""
    o = sb.make_opts(w["p"], prec=sb.SBIE_FP64, tol=1e-8, mem_kind=1, stream=stream.cuda_stream)
    ctx = sb.sphere_bie_create(w["centres"], w["radii"], o)
    N = sb.sphere_bie_num_nodes(ctx)
    x = torch.randn((N, 3), dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    sb.sphere_bie_apply_operator(ctx, op, x, y)
    ts, _ = _timed_solves(torch, stream, lambda: sb.sphere_bie_apply_operator(ctx, op, x, y), 1)
    sb.sphere_bie_destroy(ctx)
    return ts[0]


def _precond_runs(sb, torch, w, stream, op, solve, net_path, steps, exact=True):
    out = {}
    kinds = [(1, "learned"), (0, "none")] + ([(2, "exact")] if exact else [])
    for kind, name in kinds:
        o = sb.make_opts(w["p"], prec=sb.SBIE_MIXED, tol=w.get("tol", 1e-8), mem_kind=1, stream=stream.cuda_stream)
        o.use_learned_precond = kind
        o.mlp_weights_path = net_path if kind == 1 else None
        ctx = sb.sphere_bie_create(w["centres"], w["radii"], o)
        if name == "learned":  # later contexts of the same geometry take the tuned tilings at create
            sb.sphere_bie_autotune(ctx, op)
        t0 = time.perf_counter()
        solve(ctx)  # builds the preconditioner and captures the cycle graphs
        torch.cuda.synchronize()
        t_first = time.perf_counter() - t0
        n = steps if kind == 1 else 1
        ts, info = _timed_solves(torch, stream, lambda: solve(ctx), n)
        pi = sb.sphere_bie_precond_info(ctx, op)
        out[name] = {"time_to_solve_s": statistics.mean(ts), "iters": info["iters"],
                     "refinements": info["refinements"], "rel_residual_true": info["rel_residual_true"],
                     "first_solve_s": t_first, "precond_setup_s": pi["setup_ms"] / 1e3, "pairs": pi["pairs"],
                     "pairs_out_of_range": pi["dropped"], "graph_cycles": info["graph_cycles"]}
        sb.sphere_bie_destroy(ctx)
    return out


def run_dense(args, sb, torch, wl, local):
    """1024 unit spheres at volume fraction 0.30, every sphere pushed to a
    gap log-uniform in [0.01, 0.5]; mobility with random forces and torques;
    the pair network trained on exact mobility blocks of two-sphere
    configurations."""
    import tempfile
    w = wl.dense_1024()
    w["tol"] = 1e-8
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream()
    samples = args.pair_samples or 100000
    path = os.path.join(tempfile.mkdtemp(), "pairnet.bin")
    tr = sb.sphere_bie_train_pair_network(path, n_samples=samples, p=w["p"], gap_min=0.01, gap_max=2.0,
                                          radius=1.0, epochs=200, seed=11, ops=("mobility",))
    F = torch.tensor(w["forces"], dtype=torch.float64, device=dev)
    T = torch.tensor(w["torques"], dtype=torch.float64, device=dev)
    v, om = torch.zeros_like(F), torch.zeros_like(T)
    runs = _precond_runs(sb, torch, w, stream, "mobility",
                         lambda ctx: sb.sphere_bie_solve_mobility(ctx, F, T, v, om), path.encode(), args.steps)
    f64 = _plain_fp64_apply_s(sb, torch, w, stream, "K")
    n = len(w["radii"])
    return {"metric": "mobility time-to-solve at 1e-8 rel. residual, learned pair preconditioner", "unit": "s",
            "value": runs["learned"]["time_to_solve_s"], "higher_is_better": False, "n_gpus": 1,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "dense_1024", "n_spheres": n, "p": w["p"],
                       "nodes": n * (w["p"] + 1) * (2 * w["p"] + 2), "precision": "mixed", "tol": 1e-8},
            "network": {"samples": samples, "val_rel_err": tr["val_rel_err"], "data_s": tr["t_data_s"],
                        "train_s": tr["t_train_s"], "operator": "mobility", "gap_range": [0.01, 2.0]},
            "solves": runs,
            "plain_fp64": {"apply_s": f64,
                           "lower_bound_solve_s": f64 * runs["none"]["iters"],
                           "note": "one FP64 apply x the unpreconditioned iteration count (no FP64 solve run)"}}


def run_large(args, sb, torch, wl, local):
    """4096 spheres, radii U[0.8, 1.2], volume fraction 0.20, p = 12, resistance
    in a random linear background flow; learned pair preconditioner (radius
    range in training) against no preconditioner; the plain FP64 path by its
    apply time."""
    import tempfile
    w = wl.large_4096()
    w["tol"] = 1e-8
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream()
    samples = args.pair_samples or 20000
    path = os.path.join(tempfile.mkdtemp(), "pairnet.bin")
    tr = sb.sphere_bie_train_pair_network(path, n_samples=samples, p=w["p"], gap_min=0.01, gap_max=2.4,
                                          radius=0.8, radius_max=1.2, epochs=200, seed=13)
    vel = torch.tensor(w["vel"], dtype=torch.float64, device=dev)
    om = torch.tensor(w["omega"], dtype=torch.float64, device=dev)
    F, T = torch.zeros_like(vel), torch.zeros_like(om)
    runs = _precond_runs(sb, torch, w, stream, "resistance",
                         lambda ctx: sb.sphere_bie_solve_resistance(ctx, vel, om, w["u0"], w["G"], F, T),
                         path.encode(), 1, exact=False)
    n = len(w["radii"])
    return {"metric": "resistance time-to-solve at 1e-8 rel. residual, learned pair preconditioner", "unit": "s",
            "value": runs["learned"]["time_to_solve_s"], "higher_is_better": False, "n_gpus": 1,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "large_4096", "n_spheres": n, "p": w["p"],
                       "nodes": n * (w["p"] + 1) * (2 * w["p"] + 2), "precision": "mixed", "tol": 1e-8},
            "network": {"samples": samples, "val_rel_err": tr["val_rel_err"], "data_s": tr["t_data_s"],
                        "train_s": tr["t_train_s"], "operator": "resistance", "radius_range": [0.8, 1.2],
                        "gap_range": [0.01, 2.4]},
            "solves": runs}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1707_06551_gb300 import build_lib
    if local == 0:
        build_lib.build()
    if world > 1:
        dist.barrier()
    from paper_1707_06551_gb300 import sphere_bie as sb
    from paper_1707_06551_gb300 import workloads as wl

    if args.workload != WORKLOAD:
        if rank == 0:
            print(json.dumps(run_workload(args, sb, torch, wl, local)))
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return
    if args.pair_samples is None:
        args.pair_samples = 4096
    w = wl.resistance_256()
    n, p = len(w["radii"]), w["p"]
    prec = sb.SBIE_MIXED if args.prec == "mixed" else sb.SBIE_FP64
    stream = torch.cuda.Stream()
    opts = sb.make_opts(p, prec=prec, tol=w["tol"], mem_kind=1, stream=stream.cuda_stream, graphs=not args.no_graphs)
    # The pair network of the learned preconditioner is trained once, before
    # anything is timed (a model-loading step: it depends on p and the radii,
    # not on the suspension), on exact blocks for this workload's close-pair gaps.
    net = None
    if not args.no_precond:
        net = train_pair_network(sb, w, args.pair_samples)
        opts.use_learned_precond = 1
        opts.mlp_weights_path = net["path_bytes"]
    t_c0 = time.perf_counter()
    ctx = sb.sphere_bie_create(w["centres"], w["radii"], opts)
    t_create = time.perf_counter() - t_c0
    t_c0 = time.perf_counter()
    tuning = sb.sphere_bie_autotune(ctx, "resistance") if prec == sb.SBIE_MIXED else None
    t_tune = time.perf_counter() - t_c0
    dev = torch.device("cuda", local)
    vel = torch.tensor(w["vel"], dtype=torch.float64, device=dev)
    om = torch.tensor(w["omega"], dtype=torch.float64, device=dev)
    F = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    T = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MiB > 129 MB L2

    def step():
        return sb.sphere_bie_solve_resistance(ctx, vel, om, w["u0"], w["G"], F, T)

    infos = []
    for _ in range(args.warmup):
        infos.append(step())
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    smi_index = vis.split(",")[local] if vis and vis.split(",")[0].strip().isdigit() else str(local)
    sampler = ClockSampler(smi_index)
    sampler.start()
    time.sleep(0.5)

    def timed(n):
        ts, inf = [], []
        for _ in range(n):
            with torch.cuda.stream(stream):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            info = step()
            with torch.cuda.stream(stream):
                e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
            inf.append(info)
        return ts, inf

    t_wall0 = time.time()
    # the NVTX range lets a profiler select the launches of the timed solves
    # (ncu --nvtx --nvtx-include "timed_solves/")
    torch.cuda.nvtx.range_push("timed_solves")
    times, timed_infos = timed(args.steps)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    t_wall1 = time.time()
    infos += timed_infos
    sampler.stop()
    clocks = sampler.summary(t_wall0, t_wall1)
    t_step = statistics.mean(times)
    launches_timed = sum(i["kernel_launches"] for i in timed_infos)
    # Per-stage and per-kernel times come from the same solves run again with
    # profiling on: CUDA events cannot be recorded inside the graph launches
    # of the timed solves, so profiled solves step the same device iteration
    # from the host (same kernels and launch configurations).
    sb.sphere_bie_profile(ctx, 1)
    prof_times, _ = timed(args.steps)
    torch.cuda.synchronize()
    prof = sb.sphere_bie_profile_read(ctx)
    sb.sphere_bie_profile(ctx, 0)
    t_step = max_over_ranks(torch, dist if world > 1 else None, world, t_step, dev)
    last = infos[-1]

    # far-field kernel roofline (FP32 pair kernel, the hot loop of the solve)
    l32 = prof["launches"]["far_kernel_f32"]
    ms32 = prof["ms"]["far_kernel_f32"]
    pairs32 = prof["far_pairs_f32"]
    l64 = prof["launches"]["far_kernel_f64"]
    ms64 = prof["ms"]["far_kernel_f64"]
    pairs64 = prof["far_pairs_f64"]
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    clk_max = (clocks or {}).get("sm_max_mhz") or 2070.0
    peak = peak_fp32_tflops(sm_count, clk_max)
    probe_tf, probe_ms = sb.sphere_bie_fp32_peak_probe()
    roof = None
    if l32 > 0 and ms32 > 0:
        flop_launch = pairs32 / l32 * FLOP_PER_PAIR["D"]
        achieved = flop_launch / (ms32 / l32 * 1e-3) / 1e12
        traffic = ncu_traffic((tuning or {}).get("fp32") or {})
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": "far_f32_kernel<D>",
                "peak_basis": f"{sm_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {clk_max:.0f} MHz (derived)",
                "peak_probe": probe_tf, "frac_of_probe": achieved / probe_tf,
                "probe": "packed FP32x2 FMA chains on every SM (sphere_bie_fp32_peak_probe), best of 3",
                "flop_per_pair": FLOP_PER_PAIR["D"], "pairs_per_launch": pairs32 // l32,
                "ms_per_launch": ms32 / l32}
    far = {"pairs_per_s_fp32": pairs32 / (ms32 * 1e-3) if ms32 > 0 else None,
           "pairs_per_s_df": pairs64 / (ms64 * 1e-3) if ms64 > 0 else None,
           "pairs_per_s_fp64": None,
           "df_launches_per_solve": l64 / args.steps, "fp32_launches_per_solve": l32 / args.steps}
    stage_ms = {k: v / args.steps for k, v in prof["ms"].items()}
    self_vsh = self_vsh_rate(prof, n * (p + 1) * (2 * p + 2))
    n_pairs = None
    if net is not None:
        n_pairs = sb.sphere_bie_precond_info(ctx)["pairs"]
    stages = stage_rooflines(prof, n, p, last["n_near_pairs"], n_pairs, peak, load_peaks())

    # plain FP64 path on the same workload (comparison; outside the timed region)
    fp64 = None
    if not args.no_fp64_compare and prec == sb.SBIE_MIXED:
        o64 = sb.make_opts(p, prec=sb.SBIE_FP64, tol=w["tol"], mem_kind=1, stream=stream.cuda_stream)
        c64 = sb.sphere_bie_create(w["centres"], w["radii"], o64)
        # native FP64 far-field pair rate: one profiled FP64 apply
        x64 = torch.randn((n * (p + 1) * (2 * p + 2), 3), dtype=torch.float64, device=dev)
        y64 = torch.zeros_like(x64)
        sb.sphere_bie_profile(c64, 1)
        sb.sphere_bie_apply_operator(c64, "resistance", x64, y64)
        p64 = sb.sphere_bie_profile_read(c64)
        sb.sphere_bie_profile(c64, 0)
        if p64["ms"]["far_kernel_f64"] > 0:
            far["pairs_per_s_fp64"] = p64["far_pairs_f64"] / (p64["ms"]["far_kernel_f64"] * 1e-3)
        del x64, y64
        F64 = torch.zeros_like(F)
        T64 = torch.zeros_like(T)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        i64 = sb.sphere_bie_solve_resistance(c64, vel, om, w["u0"], w["G"], F64, T64)
        torch.cuda.synchronize()
        fp64 = {"time_to_solve_s": time.perf_counter() - t0, "iters": i64["iters"],
                "rel_residual_true": i64["rel_residual_true"],
                "force_rel_diff_vs_mixed": float((F64 - F).abs().max() / F64.abs().max())}
        sb.sphere_bie_destroy(c64)
        # FP64-accurate path with the double-float far field
        odf = sb.make_opts(p, prec=sb.SBIE_FP64_DF, tol=w["tol"], mem_kind=1, stream=stream.cuda_stream)
        cdf = sb.sphere_bie_create(w["centres"], w["radii"], odf)
        sb.sphere_bie_autotune(cdf, "resistance")
        Fdf = torch.zeros_like(F)
        Tdf = torch.zeros_like(T)
        sb.sphere_bie_solve_resistance(cdf, vel, om, w["u0"], w["G"], Fdf, Tdf)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        idf = sb.sphere_bie_solve_resistance(cdf, vel, om, w["u0"], w["G"], Fdf, Tdf)
        torch.cuda.synchronize()
        fp64["df_path"] = {"time_to_solve_s": time.perf_counter() - t0, "iters": idf["iters"],
                           "rel_residual_true": idf["rel_residual_true"],
                           "force_rel_diff_vs_fp64": float((Fdf - F64).abs().max() / F64.abs().max())}
        sb.sphere_bie_destroy(cdf)

    pre = None
    if net is not None:
        pre = precond_compare(sb, torch, w, prec, stream, vel, om, F, last, net)

    # end to end through the public API with host buffers: create (geometry
    # upload, tables, close-pair lists), solve, read forces/torques, destroy
    e2e_times = []
    hF = np.zeros((n, 3))
    hT = np.zeros((n, 3))
    for _ in range(args.e2e_steps):
        oh = sb.make_opts(p, prec=prec, tol=w["tol"], mem_kind=0)
        if net is not None:
            oh.use_learned_precond = 1
            oh.mlp_weights_path = net["path_bytes"]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ch = sb.sphere_bie_create(w["centres"], w["radii"], oh)
        sb.sphere_bie_solve_resistance(ch, w["vel"], w["omega"], w["u0"], w["G"], hF, hT)
        sb.sphere_bie_destroy(ch)
        e2e_times.append(time.perf_counter() - t0)
    h2d = 8 * (w["centres"].size + w["radii"].size + w["vel"].size + w["omega"].size + 3 + 9)
    d2h = 8 * (hF.size + hT.size)
    t_e2e = None
    if args.e2e_steps > 0:
        t_e2e = max_over_ranks(torch, dist if world > 1 else None, world, statistics.mean(e2e_times), dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline()
        applies = cb["applies"]
        cpu = {"value": cb["apply_s"] * applies if applies else None, "unit": "s", "cores": cb["cores"],
               "kind": "oracle",
               "sample": (f"one full resistance_256 operator apply by the oracle (all 256 target spheres, all "
                          f"61,952 nodes) on {cb['cores']} host cores, timed in full: {cb['apply_s']:.1f} s; "
                          f"x {applies} operator applies of the oracle's own FP64 GMRES solve of this workload "
                          f"({cb['solve_iters']} iterations at tol 1e-8)"),
               "timed_in_full": {"resistance_256_apply_s": cb["apply_s"], "mobility_8_solve": cb["mobility_8"]}}

    graphs_cmp = None if args.no_graphs else graph_compare(sb, torch, wl, w, prec, stream, vel, om, F, t_step, net)
    batched = None if (args.no_batched or args.no_graphs or rank != 0) else batched_quick(sb, torch, wl, local)
    launches_per_step = launches_timed / args.steps
    if rank == 0:
        line = {
            "metric": METRIC, "value": t_step, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64" if prec == sb.SBIE_MIXED else "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_spheres": n, "p": p, "nodes": n * (p + 1) * (2 * p + 2),
                       "precision": args.prec, "tol": w["tol"], "close_pairs": last["n_near_pairs"],
                       "preconditioner": ("learned pair network (trained before the timed region)"
                                          if net is not None else "none"),
                       "l2": "256 MiB buffer written between timed steps", "parallelism": f"replicas x{world}"},
            "solve": {"iters": last["iters"], "refinements": last["refinements"],
                      "fp32_residual_updates": last["fp32_residual_updates"], "fp32_op_err": last["fp32_op_err"],
                      "last_correction": last["last_correction"],
                      "rel_residual_true": last["rel_residual_true"], "status": last["status"],
                      "create_s": t_create, "autotune_s": t_tune, "far_tiling": tuning},
            "roofline": roof, "far_field": far, "stage_ms_per_step": stage_ms, "self_vsh": self_vsh,
            "stage_rooflines": stages, "fp32_peak_probe": {"tflops": probe_tf, "ms": probe_ms},
            "fp64_path": fp64,
            "pair_preconditioner": pre,
            "clocks": clocks, "gpu_launches": int(launches_timed),
            "gpu_launches_per_step": launches_per_step,
            "timed_solves": {"gmres_cycles_as_cuda_graphs": not args.no_graphs,
                             "graph_cycles_per_step": sum(i["graph_cycles"] for i in timed_infos) / args.steps},
            "profiled_solves": {"steps": args.steps, "mean_s": statistics.mean(prof_times),
                                "note": "stage and kernel times (roofline, far_field, stage_ms_per_step) come from "
                                        "these host-stepped solves with CUDA events per stage"},
            "graphs_vs_host_stepped": graphs_cmp,
            "batched_512": batched,
            "e2e": ({"value": t_e2e, "unit": "s", "h2d_bytes_per_step": h2d,
                     "d2h_bytes_per_step": d2h, "includes": "create + solve + destroy, host buffers"}
                    if t_e2e is not None else None),
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    sb.sphere_bie_destroy(ctx)
    if net is not None:
        try:
            os.remove(net["path"])
            os.rmdir(net["dir"])
        except OSError:
            pass
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
