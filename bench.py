"""Benchmark: MG-GCR time per solve at ||r||/||b|| < 1e-10 on GB300.

Default workload (N=1): 32^4 lattice, naive staggered operator on seeded
synthetic links Proj_SU3(exp(0.3 i H)), mass 0.001, twelve Gaussian
right-hand sides solved together by one smg_multi_solve per step; K-cycle
multigrid with Table 1's two coarsenings (4^4 then 2^4 aggregates, 64 / 32
near-null vectors from 1000 CGNE iterations) and an SVD-deflated Chebyshev
CA-GCR coarsest level (48 singular vectors), level-1 inner GCR to 0.05 or
16 iterations and Table 1's 0.25 or 8 below it, FP32 arithmetic with FP16
storage of links, KD blocks, near-null vectors and coarse stencils (the
12-system coarse apply on the tensor cores), FP64 outer GCR.  Other
workloads: --config 1 (8^4, FP64), 2 (16^4 HISQ-shaped), 4 (24^3 x 48
HISQ-shaped, 8 masses x 4 sources).

A step is one complete batched solve (the outer GCR of every system until its
FP64-recomputed residual is below 1e-10) with the sources already in device
memory; `value` is the step time divided by the systems it solves.  The
multigrid setup is built once before timing and reported separately.  L2 is
flushed (a 512 MB write) before every timed step.  `e2e` repeats the
measurement through the C ABI with pinned host buffers (host->device copy of
the sources and device->host copy of the solutions inside the timed region).
The same algorithm in plain FP64 (same near-null vectors, FP64 operators,
one system at a time, no CUDA graph) is timed beside it for the
mixed+batched vs FP64 comparison the metric names.

`--impl reference` times the FP64 CPU oracle instead (rank 0, host cores).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "MG-GCR time/solve at |r|/|b|<1e-10 and coarse-apply GB/s, mixed+batched vs FP64"
UNIT = "s/solve"
WORKLOADS = {
    1: "8^4 naive staggered, m=0.1, 2-level KD-MG (4^4 aggregates, 24 vectors), FP64, 1 RHS",
    2: "16^4 HISQ-shaped, m=0.01, 3-level KD-MG (4^4/2^4 aggregates, 24/32 vectors), truncated level-1 operator, "
       "FP32 + FP16 storage, FP64 outer GCR, 1 RHS",
    3: "32^4 naive staggered, m=0.001, 12 Gaussian RHS solved together, KD-MG with Table 1's levels "
       "(4^4/2^4 aggregates, 64/32 vectors, SVD-deflated Chebyshev CA-GCR coarsest level with 48 singular vectors), "
       "FP32 + FP16 storage (12-system coarse apply on tcgen05), FP64 outer GCR",
    4: "24^3x48 HISQ-shaped, 8 masses log-spaced 0.001-0.05 x 4 sources = 32 systems in one batch, KD-MG with "
       "Table 1's levels (4^4/2^4 aggregates, 64/32 vectors, SVD-deflated Chebyshev CA-GCR coarsest level with 48 "
       "singular vectors, operators of the lightest mass), truncated level-1 operator, FP32 + FP16 storage, "
       "FP64 outer GCR",
}
# Solver recipe of each workload (its inputs come from inputs.CONFIGS): the
# level-1 inner rule, the rule of the coarse levels (0 = the same), the
# near-null CGNE cap and the level-1 operator.  Table 1's "0.25 or 8
# iterations" serves the heavier masses; at m = 0.001 the outer GCR stalls
# near 1e-2 with it at level 1 (GPU and oracle probes); the level-1 rule
# 0.05 / 16 with near-null vectors from 1000 CGNE iterations and Table 1's
# rule on the coarse levels converges (32^4: 12 outer iterations, 0.74 s per
# system, against 10 and 1.13 s with 0.05 / 16 on every level).
SOLVER = {
    1: dict(inner=(0.25, 8), coarse_inner=(0.0, 0), setup_maxiter=2000, truncate_naik=0),
    2: dict(inner=(0.25, 8), coarse_inner=(0.0, 0), setup_maxiter=2000, truncate_naik=1),
    3: dict(inner=(0.05, 16), coarse_inner=(0.25, 8), setup_maxiter=1000, truncate_naik=0, coarsest_deflate=48),
    4: dict(inner=(0.05, 16), coarse_inner=(0.25, 8), setup_maxiter=1000, truncate_naik=1, coarsest_deflate=48),
}
# Outer GCR iterations a solve of the workload takes with this algorithm,
# measured by the GPU path with the same recipe; scales the oracle's
# per-iteration time in --impl reference (no GPU runs there).
REF_OUTER_ITERS = {1: 10, 2: 31, 3: 12, 4: 16}


# ------------------------------------------------------------------ helpers
def log(msg):
    """Progress on stderr (the JSON line stays the only stdout output)."""
    sys.stderr.write(f"[bench {time.strftime('%H:%M:%S')}] {msg}\n")
    sys.stderr.flush()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x, tdist, device):
    """Largest value of x over the process group (timing of the slowest rank)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def replica_value(tmax, steps, world_size):
    """Seconds per solve of the whole job: every rank solves `steps` systems
    independently (replicas, weak scaling), the job takes the slowest rank's time."""
    return tmax / (steps * world_size)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------- GPU problem
def problem(cfg, torch, dev, rank=0, dims=None):
    """Gauge field, mass and near-null starts of a workload on the device, its
    sources on the host ([nrhs][V][3]; replica `rank` draws its own) and the
    masses of the batch."""
    from paper_2212_12559_gb300 import binding, inputs
    c = inputs.config_inputs(cfg, dims=tuple(dims) if dims else None)
    dims = c["dims"]
    V = int(np.prod(dims))
    s = binding.Solver(dims)
    s.set_stream(torch.cuda.current_stream(dev).cuda_stream)
    s.set_gauge(torch.from_numpy(c["fat"]).to(dev),
                None if c["naik"] is None else torch.from_numpy(c["naik"]).to(dev), c["c_naik"])
    s.set_mass(c["mass"])
    nv = c["nvec"]
    phi0 = [torch.from_numpy(inputs.gaussian_fields(nv[0], V, 3, c["nullvec_seed"])).to(dev)]
    cdims = dims
    for l in range(1, len(nv)):
        cdims = tuple(d // a for d, a in zip(cdims, c["agg"][l - 1]))
        phi0.append(torch.from_numpy(
            inputs.gaussian_fields(nv[l], int(np.prod(cdims)), 2 * nv[l - 1], c["nullvec_seed"] + 10 * l)).to(dev))
    k = SOLVER[cfg].get("coarsest_deflate", 0)
    if k > 0:
        cdims = tuple(d // a for d, a in zip(cdims, c["agg"][-1]))
        phi0.append(torch.from_numpy(inputs.gaussian_fields(binding.deflation_block(k), int(np.prod(cdims)),
                                                            2 * nv[-1], c["nullvec_seed"] + 99)).to(dev))
    src = c["sources"]
    if rank > 0:
        src = np.stack([inputs.gaussian_field(V, 3, c["seeds"][1] + 1000 * rank + r) for r in range(src.shape[0])])
    masses = np.array([c["mass"]]) if c["masses"] is None else inputs.log_masses(0.001, 0.05, 8)
    return c, s, phi0, src, masses


def solver_params(binding, c, cfg, precision, use_graph, args, persistent=1):
    rec = SOLVER[cfg]
    prec = {"double": binding.PREC_DOUBLE, "single": binding.PREC_SINGLE, "mixed": binding.PREC_HALF}[precision]
    inner = (args.inner_tol, args.inner_maxiter) if args.inner_tol > 0 else rec["inner"]
    return binding.default_params(
        n_coarse=len(c["nvec"]), agg=c["agg"], nvec=c["nvec"], precision=prec, use_graph=use_graph,
        persistent=persistent, setup_maxiter=args.setup_maxiter if args.setup_maxiter > 0 else rec["setup_maxiter"],
        max_outer=args.max_outer, truncate_naik=rec["truncate_naik"], inner_tol=float(inner[0]),
        inner_maxiter=int(inner[1]), coarse_inner_tol=float(rec["coarse_inner"][0]),
        coarse_inner_maxiter=int(rec["coarse_inner"][1]), coarsest_deflate=int(rec.get("coarsest_deflate", 0)))


def coarse_bytes(N, nsys, store_bytes=4, scale=True):
    """Algorithmic bytes of one coarse-site apply: 9 N^2 stencil entries, row
    scales, the site's input vector (read once) and its output vector."""
    return 9 * N * N * store_bytes + (4 * N if scale else 0) + 2 * N * 8 * nsys


def dslash_bytes(hisq, nsys, store_bytes=4):
    """Per fine site: 4 (8 with Naik) 3x3 links at storage precision (read once
    for the batch), input and output colour vectors in FP32 (each read /
    written once per system)."""
    nl = 8 if hisq else 4
    return nl * 9 * store_bytes + 2 * 3 * 8 * nsys


def kd_bytes(nsys, store_bytes=4):
    """Per fine site: 48^2/16 = 144 complex block entries, 3 FP32 row scales,
    input and output colour vectors."""
    return 144 * store_bytes + 3 * 4 + 2 * 3 * 8 * nsys


def transfer_bytes(nvec, ndof, nsys, store_bytes=4):
    """Per fine site of a restriction or prolongation: the site's ndof x nvec
    prolongator entries (read once for the batch) and its ndof components of
    every system; the coarse side is V/agg as large and left out."""
    return ndof * nvec * store_bytes + ndof * 8 * nsys


# ------------------------------------------------------ coarse apply alone
COARSE_SHAPES = {
    # coarse level of a workload: extents, components per site
    "8^4xN128": ((8, 8, 8, 8), 128),     # 32^4 / 4^4 aggregates, 64 vectors: 2.42 GB FP16 stencil
    "6^3x12xN48": ((6, 6, 6, 12), 48),   # 24^3x48 / 4^4 aggregates, 24 vectors: 215 MB
    "4^4xN48": ((4, 4, 4, 4), 48),       # 16^4 / 4^4 aggregates, 24 vectors: 21.5 MB (L2-resident)
}


def coarse_roofline(binding, solver, shape, nsys, nrep, hbm):
    """Times the 9-point coarse apply on a synthetic FP16 stencil of a coarse
    level's shape; returns a roofline dict (algorithmic bytes: 9 N^2 complex
    FP16 entries + N FP32 row scales per site, input and output FP32 vectors
    of nsys systems, each counted once)."""
    cd, N = COARSE_SHAPES[shape]
    Vc = int(np.prod(cd))
    ms = solver.bench_coarse_apply(cd, N, nsys, binding.PREC_HALF, nrep)
    alg = coarse_bytes(N, nsys) * Vc
    ach = alg / (ms * 1e-3) / 1e9
    flops = 8 * 9 * N * N * nsys * Vc
    return {"shape": shape, "N": N, "coarse_sites": Vc, "nrhs": nsys, "ms_per_launch": ms,
            "alg_bytes_per_launch": alg, "achieved_GBs": ach, "frac_of_hbm": ach / hbm,
            "TFLOPs": flops / (ms * 1e-3) / 1e12}


def run_coarse_only(args):
    """Coarse apply alone on the workloads' coarse-level shapes (profiling aid)."""
    import torch
    from paper_2212_12559_gb300 import binding
    torch.cuda.set_device(0)
    s = binding.Solver((4, 4, 4, 4))
    hbm, _ = measured_peaks()
    shapes = [args.shape] if args.shape else list(COARSE_SHAPES)
    for sh in shapes:
        for nsys in args.nrhs:
            print(json.dumps(coarse_roofline(binding, s, sh, nsys, args.nrep, hbm)), flush=True)
    return 0


# --------------------------------------------------------- oracle sample
def oracle_sample(cfg, n_iter, out_path, dims):
    """Runs in a child process with one BLAS thread: times the oracle's outer
    GCR iterations (K-cycle + M) of the workload's operator and level
    structure on the extents `dims` (setup with unrefined random near-null
    vectors, not timed)."""
    from oracle.dirac import Staggered
    from oracle.lattice import Lattice
    from oracle.mg import MGParams, MultigridSolver
    from paper_2212_12559_gb300 import inputs
    c = inputs.config_inputs(cfg, dims=tuple(dims))
    V = int(np.prod(dims))
    op = Staggered(Lattice(dims), c["fat"], c["naik"], c["c_naik"], c["mass"])
    nv = c["nvec"]
    phi0 = [inputs.gaussian_fields(nv[0], V, 3, c["nullvec_seed"])]
    cdims = tuple(dims)
    for l in range(1, len(nv)):
        cdims = tuple(d // a for d, a in zip(cdims, c["agg"][l - 1]))
        phi0.append(inputs.gaussian_fields(nv[l], int(np.prod(cdims)), 2 * nv[l - 1], c["nullvec_seed"] + 10 * l))
    rec = SOLVER[cfg]
    t0 = time.perf_counter()
    mg = MultigridSolver(op, MGParams(agg=c["agg"], nvec=nv, setup_maxiter=0,
                                      truncate_naik=bool(rec["truncate_naik"]), inner_tol=rec["inner"][0],
                                      inner_maxiter=rec["inner"][1], coarse_inner_tol=rec["coarse_inner"][0],
                                      coarse_inner_maxiter=rec["coarse_inner"][1]), phi0)
    t_setup = time.perf_counter() - t0
    b = c["sources"][0]
    times = []
    for _ in range(n_iter):
        t0 = time.perf_counter()
        z = mg.precondition(b)
        op.M(z)
        times.append(time.perf_counter() - t0)
    with open(out_path, "w") as f:
        json.dump({"iter_times": times, "setup_s": t_setup, "V": V}, f)


def oracle_full_solve(cfg, out_path):
    """Runs in a child process with one BLAS thread: one complete oracle
    setup (CGNE near-null vectors) and solve of a workload."""
    from oracle.dirac import Staggered
    from oracle.lattice import Lattice
    from oracle.mg import MGParams, MultigridSolver
    from paper_2212_12559_gb300 import inputs
    c = inputs.config_inputs(cfg)
    dims = c["dims"]
    V = int(np.prod(dims))
    op = Staggered(Lattice(dims), c["fat"], c["naik"], c["c_naik"], c["mass"])
    rec = SOLVER[cfg]
    t0 = time.perf_counter()
    mg = MultigridSolver(op, MGParams(agg=c["agg"], nvec=c["nvec"], setup_maxiter=rec["setup_maxiter"],
                                      inner_tol=rec["inner"][0], inner_maxiter=rec["inner"][1]),
                         [inputs.gaussian_fields(c["nvec"][0], V, 3, c["nullvec_seed"])])
    t1 = time.perf_counter()
    x, it, res = mg.solve(c["sources"][0], 1e-10)
    t2 = time.perf_counter()
    with open(out_path, "w") as f:
        json.dump({"setup_s": t1 - t0, "solve_s": t2 - t1, "iters": it, "residual": res, "V": V}, f)


def run_child(args_list, timeout):
    """Runs this script in a child process on the host cores only (one BLAS
    thread, no GPU visible); returns the JSON the child wrote."""
    import tempfile
    fd, out = tempfile.mkstemp(suffix=".json")
    os.close(fd)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT"):
        env.pop(k, None)
    cmd = [sys.executable, os.path.abspath(__file__)] + args_list + [out]
    try:
        r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=timeout)
        if r.returncode != 0:
            raise RuntimeError("oracle child failed: " + r.stderr[-2000:])
        with open(out) as f:
            return json.load(f)
    finally:
        if os.path.exists(out):
            os.remove(out)


def sample_dims(cfg):
    """Extents of the oracle sample: the workload's own level structure and
    aspect ratio on the smallest lattice that keeps them: per direction the
    product of the aggregate extents times the workload's coarsest extent
    divided by the common factor of those extents (32^4 -> 8^4,
    24^3 x 48 -> 8^3 x 16)."""
    import math
    from paper_2212_12559_gb300 import inputs
    c = inputs.CONFIGS[cfg]
    dims = list(c["dims"])
    q = [math.prod(a[mu] for a in c["agg"]) for mu in range(4)]
    base = [d // qq for d, qq in zip(dims, q)]
    g = math.gcd(*base)
    return tuple(qq * (b // g) for qq, b in zip(q, base))


# --------------------------------------------------------------------- arms
def run_reference(args):
    """The FP64 CPU oracle on the host cores: each step one oracle outer-GCR
    iteration of the workload on the reduced lattice, scaled by volume and by
    the outer iterations per solve the GPU path needs."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    cfg = args.config
    from paper_2212_12559_gb300 import inputs
    dims = sample_dims(cfg)
    V = int(np.prod(inputs.CONFIGS[cfg]["dims"]))
    n = args.steps + args.warmup
    d = run_child(["--_oracle-sample", str(cfg), str(n), *[str(x) for x in dims]], 3600)
    vol = V / d["V"]
    iters = REF_OUTER_ITERS[cfg]
    per_solve = [t * vol * iters for t in d["iter_times"][args.warmup:]]
    value = statistics.mean(per_solve)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[cfg], "oracle_sample_dims": list(dims), "oracle_setup_s": d["setup_s"]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} oracle outer-GCR iterations (K-cycle + M) of this workload's "
                                   f"operator and level structure on {'x'.join(map(str, dims))}, scaled by volume "
                                   f"x{vol:.0f} and by the {iters} outer iterations a solve takes on the GPU path; "
                                   f"oracle setup with unrefined near-null vectors, not timed"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def timed_batches(torch, s, b, masses, steps, flush):
    """Per-step seconds (CUDA events on the solver's stream, L2 flushed before
    each) of `steps` batched solves; returns (times, infos of the last step)."""
    times, infos = [], None
    st = torch.cuda.current_stream()
    for _ in range(steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        _, infos = s.multi_solve(b, masses, 1e-10)
        e1.record(st)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    return times, infos


def kernel_rooflines(binding, s, c, nsys, hbm):
    """Live CUDA-event timings of the solve's kernel families on the workload's
    own operators (smg_time_kernel: nrep launches on the solver's stream, the
    autotuner's kernel for the shape) with their algorithmic bytes."""
    V = int(np.prod(c["dims"]))
    hisq = c["naik"] is not None
    out = {}
    nv0 = c["nvec"][0]
    cd = [d // a for d, a in zip(c["dims"], c["agg"][0])]
    Vc, N = int(np.prod(cd)), 2 * nv0
    for name, kern, l, nbytes in (
            ("coarse_apply_level2", binding.K_COARSE, 0, coarse_bytes(N, nsys) * Vc),
            ("dslash", binding.K_DSLASH, 0, dslash_bytes(hisq, nsys, 4) * V),
            ("kd_apply", binding.K_KD, 0, kd_bytes(nsys) * V),
            ("restrict_level1", binding.K_RESTRICT, 0, transfer_bytes(nv0, 3, nsys) * V),
            ("prolong_level1", binding.K_PROLONG, 0, transfer_bytes(nv0, 3, nsys) * V)):
        ms = s.time_kernel(kern, l, nsys, 20)
        ach = nbytes / (ms * 1e-3) / 1e9
        out[name] = {"ms_per_launch": ms, "alg_bytes_per_launch": nbytes, "achieved_GBs": ach, "frac": ach / hbm}
    return out


def run_ours(args):
    import torch
    import torch.distributed as tdist
    from paper_2212_12559_gb300 import binding

    ws, rank, local = dist_env()
    if ws > 1:
        tdist.init_process_group("nccl", init_method="env://")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    cfg = args.config
    log(f"workload {cfg}: building inputs")
    c, s, phi0, src, masses = problem(cfg, torch, dev, rank=rank, dims=args.dims)
    V = int(np.prod(c["dims"]))
    p = solver_params(binding, c, cfg, c["precision"], args.graph, args)
    log(f"inputs ready (dims {c['dims']}); setup")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.mg_setup(p, phi0)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    setup_iters = [s.setup_iterations(l) for l in range(len(c["nvec"]))]
    setup_phases = [{k: round(v, 3) for k, v in s.setup_times(l).items()} for l in range(len(c["nvec"]))]
    log(f"setup {t_setup:.1f} s, CGNE iterations {setup_iters}")
    b = torch.from_numpy(src).to(dev)
    nsys = b.shape[0] * len(masses)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        t0 = time.perf_counter()
        _, inf = s.multi_solve(b, masses, 1e-10)
        log(f"warm-up step {time.perf_counter() - t0:.2f} s, outer {inf[0].iterations}, "
            f"max residual {max(i.true_residual for i in inf):.2e}")
    # timed region: K batched solves, L2 flushed before each
    if ws > 1:
        tdist.barrier()
    torch.cuda.synchronize()
    launches0 = binding.kernel_launches()
    clocks = ClockSampler(local)
    clocks.start()
    t_wall0 = time.perf_counter()
    if args.profile:
        torch.cuda.profiler.start()
    times, infos = timed_batches(torch, s, b, masses, args.steps, flush)
    torch.cuda.synchronize()
    if args.profile:
        torch.cuda.profiler.stop()
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    launches = binding.kernel_launches() - launches0
    if ws > 1:
        tdist.barrier()
    total = sum(times)
    tmax = max_over_ranks(total, tdist, dev) if ws > 1 else total
    value = tmax / (args.steps * nsys * ws)
    conv = all(i.converged for i in infos)
    res = max(i.true_residual for i in infos)
    log(f"timed: {statistics.mean(times):.3f} s per step of {nsys} systems, outer {infos[0].iterations}, "
        f"max residual {res:.2e}")

    # end to end through the C ABI with pinned host buffers
    bh = torch.from_numpy(src).pin_memory()
    xh = torch.empty((len(masses),) + tuple(bh.shape), dtype=torch.complex128).pin_memory()
    e2e_times = []
    for _ in range(args.e2e_steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, einf = s.multi_solve(bh, masses, 1e-10, x=xh)
        e2e_times.append(time.perf_counter() - t0)
    e2e = statistics.mean(e2e_times) / nsys if e2e_times else None

    hbm, peak_kind = measured_peaks()
    roof, kern = None, {}
    if rank == 0:
        # the solve's kernel families on this workload's operators; the line's
        # roofline is the family with the largest share of the solve's device
        # time (the launch list in profiles/ names it)
        kern = kernel_rooflines(binding, s, c, min(nsys, 16), hbm)
        top = DOMINANT.get(cfg, "coarse_apply_level2")
        k = kern[top]
        roof = {"bound": "hbm", "kernel": top, "achieved": k["achieved_GBs"], "peak": hbm, "unit": "GB/s",
                "frac": k["frac"], "traffic": NCU_TRAFFIC.get(cfg), "peak_kind": peak_kind + " HBM copy bandwidth",
                "ms_per_launch": k["ms_per_launch"], "alg_bytes_per_launch": k["alg_bytes_per_launch"],
                "systems_per_launch": min(nsys, 16), "others": {n: v for n, v in kern.items() if n != top}}

    # the same algorithm in plain FP64 on the same GPU: same near-null vectors
    # (loaded from the mixed setup), FP64 operators, one system at a time
    fp64 = None
    if rank == 0 and args.compare_fp64 and c["precision"] != "double":
        import tempfile
        path = os.path.join(tempfile.mkdtemp(), "setup.smg")
        s.save_setup(path)
        s64 = binding.Solver(c["dims"])
        s64.set_stream(torch.cuda.current_stream(dev).cuda_stream)
        s64.set_gauge(torch.from_numpy(c["fat"]).to(dev),
                      None if c["naik"] is None else torch.from_numpy(c["naik"]).to(dev), c["c_naik"])
        s64.set_mass(c["mass"])
        fp64 = {}
        for graph in ((1, 0) if args.fp64_both else (1,)):
            p64 = solver_params(binding, c, cfg, "double", graph, args, persistent=0)
            s64.load_setup(path, p64)
            b1 = b[:1]
            m1 = masses[:1]
            if graph:
                s64.multi_solve(b1, m1, 1e-10)       # warm-up: the graph capture
            t64, inf64 = timed_batches(torch, s64, b1, m1, args.fp64_steps, flush)
            key = "graph" if graph else "no_graph"
            fp64[key] = {"s_per_solve": statistics.mean(t64), "outer_iters": inf64[0].iterations,
                         "converged": bool(inf64[0].converged), "true_residual": inf64[0].true_residual}
            fp64["speedup_mixed_batched_vs_fp64_" + key] = fp64[key]["s_per_solve"] / value
            log(f"FP64 ({key}): {fp64[key]['s_per_solve']:.2f} s/solve, outer {inf64[0].iterations}")
        s64.close()
        os.remove(path)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        try:
            dims = sample_dims(cfg)
            d = run_child(["--_oracle-sample", str(cfg), str(args.cpu_iters), *[str(x) for x in dims]], 900)
            vol = V / d["V"]
            per_iter = statistics.mean(d["iter_times"]) * vol
            it_per_solve = infos[0].iterations
            cpu = {"value": per_iter * it_per_solve, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"{args.cpu_iters} oracle outer-GCR iterations (K-cycle + M) of this workload's operator "
                             f"and level structure on {'x'.join(map(str, dims))} ({d['V']} sites), scaled by volume "
                             f"x{vol:.0f} to {per_iter:.2f} s per iteration and by the {it_per_solve} outer "
                             f"iterations a solve takes here; oracle setup ({d['setup_s']:.1f} s, unrefined "
                             f"near-null vectors) not timed"}
        except Exception as e:  # report, do not hide
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {e}"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.mean(times) * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if c["precision"] == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[cfg], "dims": list(c["dims"]), "systems_per_step": nsys,
                       "masses": [float(m) for m in masses], "nvec": c["nvec"], "agg": [list(a) for a in c["agg"]],
                       "precision": c["precision"],
                       "storage": ("FP16 links, KD blocks, near-null vectors and coarse stencils (FP32 scales); "
                                   "FP32 preconditioner vectors; FP64 outer GCR and true residuals")
                       if c["precision"] == "mixed" else "FP64 throughout",
                       "inner": [p.inner_tol, p.inner_maxiter],
                       "coarse_inner": [p.coarse_inner_tol or p.inner_tol, p.coarse_inner_maxiter or p.inner_maxiter],
                       "setup_maxiter": p.setup_maxiter, "cuda_graph": bool(args.graph),
                       "l2": "flushed (512 MB write) before every timed step", "setup_s": t_setup,
                       "setup_cgne_iters": setup_iters, "setup_phases_s": setup_phases,
                       "outer_iters": infos[0].iterations,
                       "all_converged": conv, "max_true_residual": res, "timed_wall_s": t_wall,
                       "parallelism": f"replicas x{ws}", "tuned_kernels": binding.tune_table()},
            "e2e": None if e2e is None else {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": int(bh.numel() * 16),
                                              "d2h_bytes_per_step": int(xh.numel() * 16)},
            "gpu_launches": launches // max(1, args.steps),
            "clocks": clk,
            "roofline": roof,
            "cpu_baseline": cpu,
        }
        if fp64 is not None:
            line["config"]["fp64_gpu"] = fp64
        print(json.dumps(line))
    if ws > 1:
        tdist.destroy_process_group()
    return 0


# Kernel family with the largest share of the solve's device time (ncu launch
# list of the workload, profiles/), and its DRAM traffic per launch from one
# ncu capture when it still describes the current kernel (else None).
DOMINANT = {3: "coarse_apply_level2", 4: "coarse_apply_level2", 2: "dslash", 1: "kd_apply"}
# DRAM bytes (read + write) per launch of the dominant kernel from one ncu
# capture of that kernel at the workload's shape, while the kernel is
# unchanged since (profiles/coarse_umma_tcgen05_N128_4096sites_12rhs.md:
# 2.597 GB read + 0.053 GB written against 2.519 GB algorithmic)
NCU_TRAFFIC = {3: 2597469000 + 53360384}


def main():
    if len(sys.argv) > 1 and sys.argv[1] == "--_oracle-sample":
        cfg, n = int(sys.argv[2]), int(sys.argv[3])
        dims = tuple(int(x) for x in sys.argv[4:8])
        oracle_sample(cfg, n, sys.argv[8], dims)
        return 0
    if len(sys.argv) > 1 and sys.argv[1] == "--_oracle-full":
        oracle_full_solve(int(sys.argv[2]), sys.argv[3])
        return 0
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=3, choices=[1, 2, 3, 4])
    ap.add_argument("--graph", type=int, default=1)
    ap.add_argument("--compare-fp64", type=int, default=1)
    ap.add_argument("--fp64-steps", type=int, default=1, help="timed FP64 single-system solves per variant")
    ap.add_argument("--fp64-both", action="store_true",
                    help="time the FP64 arm without the CUDA graph too (default: with the graph only)")
    ap.add_argument("--e2e-steps", type=int, default=1, help="batches timed end to end through host buffers")
    ap.add_argument("--profile", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop (ncu --profile-from-start off)")
    ap.add_argument("--inner-tol", type=float, default=0.0,
                    help="level-1 inner GCR tolerance (0: the workload's recipe)")
    ap.add_argument("--inner-maxiter", type=int, default=16)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-iters", type=int, default=2)
    ap.add_argument("--oracle-full-solve", action="store_true",
                    help="with --impl reference: time one complete oracle setup + solve of the workload instead")
    ap.add_argument("--setup-maxiter", type=int, default=0, help="near-null CGNE cap (0: the workload's recipe)")
    ap.add_argument("--max-outer", type=int, default=500, help="outer GCR cap; lower only to bound profiler runs")
    ap.add_argument("--dims", type=int, nargs=4, default=None, help="other lattice extents (probing only)")
    ap.add_argument("--coarse-only", action="store_true",
                    help="time only the coarse apply on the workloads' coarse-level shapes")
    ap.add_argument("--shape", default=None, choices=[None] + list(COARSE_SHAPES))
    ap.add_argument("--nrhs", type=int, nargs="+", default=[1, 12])
    ap.add_argument("--nrep", type=int, default=10)
    args = ap.parse_args()
    if args.impl == "reference":
        if args.oracle_full_solve:
            d = run_child(["--_oracle-full", str(args.config)], 7200)
            print(json.dumps({"impl": "reference", "kind": "oracle full setup + solve", "workload":
                              WORKLOADS[args.config], "cores": 1, **d}))
            return 0
        return run_reference(args)
    if args.coarse_only:
        return run_coarse_only(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
