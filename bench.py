"""Benchmark of the INV-ASKIT hot path on GB300: factorization + solve per step.

One step = iaskit_factor (tree, kNN, sampling, skeletonization, leaf LU, W and Z
for every level) followed by iaskit_solve of the workload's right-hand sides.
The metric is right-hand sides solved per second with the factorization counted
in every step (RHS/s); the JSON line also carries the factor time, the
solve-only rate and the sampled eps_M of both forms (equal accuracy).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload C4]

The default workload is C4 (N = 1,048,576 points in d = 64 on a 6-dimensional
manifold, m 512, s_max 256, tau 1e-6, lambda 1e-3, 8 RHS).  The metric's own
configuration, C5 (N = 4M, d = 8, lambda 1e-4), has no FP64 solve that reaches its
residual target and does not fit the mixed form in HBM; --workload C5 runs it anyway.

--impl reference times the FP64 CPU oracle (the baseline) on a bounded sample of
the same workload and extrapolates it to the full N with per-phase complexity
models (labelled "extrapolated").  Under torchrun with N > 1 every rank factors its
own copy of the workload (independent replicas, weak scaling); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from workloads import batched_problems, make_points, make_rhs, workload  # noqa: E402

METRIC = "factor s + RHS solves/s at N=4M,d=8: chosen form vs FP64 plain, resid<=1e-10"
UNIT = "RHS/s (factor+solve per step)"
SM_COUNT = 152
FP64_FMA_PER_CLK_PER_SM = 2          # GB300: FP64 pipe width per SM and clock
CPU_SAMPLE_N = 2048                  # oracle sample: same generator and parameters, smaller N
EPS_M_ROWS = 1000                    # rows of the sampled eps_M (eq. error, Sec. III)
COMPARE_STEPS = 3                    # timed steps of the FP64 plain form beside the chosen one


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        if self.gpu < 0:
            return self
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ ranks (torchrun, N > 1)
def dist_init(backend: str):
    """The process group of a torchrun launch (RANK, WORLD_SIZE, MASTER_ADDR/PORT from the
    environment); None for a single process."""
    if int(os.environ.get("WORLD_SIZE", "1")) <= 1:
        return None
    import torch.distributed as dist
    dist.init_process_group(backend)
    return dist


def max_over_ranks(dist, x: float, device) -> float:
    """The largest x over the ranks (x itself for a single process)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist) -> None:
    if dist is not None:
        dist.barrier()


def batch_seed(rank: int) -> int:
    """Seed of rank's batch of independent problems: every rank factors a batch of its
    own (weak scaling, no data-path exchange); rank 0's is the single-GPU batch."""
    import inspect
    return inspect.signature(batched_problems).parameters["seed"].default + 1000 * rank


# ----------------------------------------------------------------- CPU oracle leg
def _depth(N: int, m: int) -> int:
    L = 0
    while -(-N // (1 << L)) > m:
        L += 1
    return L


# Per-phase growth models of the oracle (the method's complexities, Sec. II-C): tree
# N log N; brute-force kNN N^2; skeletonization one ID per non-root node (2^(L+1) - 2
# nodes, each of bounded size); factorization T^f = O(s^2 N log^2 N), i.e. N L^2 at
# fixed s; solve O(N log N), N L.
def _phase_growth(N: int, m: int) -> dict:
    L = max(_depth(N, m), 1)
    return {"tree": N * np.log2(max(N, 2)), "knn": float(N) * N, "skeletonize": float(2 ** (L + 1) - 2),
            "factorize": float(N) * L * L, "solve": float(N) * L}


def oracle_phases(w, N_sample: int, nrhs: int) -> dict:
    """One factor + solve of the oracle on N_sample points of the workload's generator
    (same parameters), each phase timed; returns seconds per phase."""
    import oracle
    from oracle.askit import skeletonize
    if w.kind == "batched":
        # the batch's first problem (its h and lambda), its first N_sample points
        X, h, lam = batched_problems(count=64)[0]
        X = np.ascontiguousarray(X[:N_sample])
        ws = w.scaled(len(X), h=h, lam=lam)
    else:
        ws = w.scaled(N_sample)
        X = make_points(ws)
    u = make_rhs(ws, nrhs=nrhs)
    t = {}
    t0 = time.perf_counter()
    tree = oracle.build_tree(X, ws.m)
    t1 = time.perf_counter()
    knn = oracle.knn_bruteforce(X, ws.kappa)
    t2 = time.perf_counter()
    sk = skeletonize(X, tree, knn, ws.h, ws.s_max, ws.tol, samp_factor=ws.samp_factor)
    t3 = time.perf_counter()
    F = oracle.factorize(sk, ws.lam)
    t4 = time.perf_counter()
    oracle.solve(F, u)
    t5 = time.perf_counter()
    return {"tree": t1 - t0, "knn": t2 - t1, "skeletonize": t3 - t2, "factorize": t4 - t3, "solve": t5 - t4}


def extrapolate(phases: dict, N_sample: int, N_full: int, m: int) -> float:
    """Seconds of the oracle at N_full from its phases at N_sample and the models above."""
    gs, gf = _phase_growth(N_sample, m), _phase_growth(N_full, m)
    return float(sum(phases[k] * gf[k] / gs[k] for k in phases))


def _full_sizes(w):
    if w.kind == "batched":
        return [len(p[0]) for p in batched_problems(count=64)]
    return [w.N]


def cpu_baseline_subprocess(wname: str, N_sample: int, nrhs: int, steps: int) -> dict:
    """Runs the oracle in a child process with every host core in its BLAS pool."""
    cores = os.cpu_count() or 1
    env = dict(os.environ, OMP_NUM_THREADS=str(cores), OPENBLAS_NUM_THREADS=str(cores),
               MKL_NUM_THREADS=str(cores))
    code = (f"import sys, json; sys.path.insert(0, {ROOT!r}); import bench; "
            f"from workloads import workload; w = workload({wname!r}); "
            f"ts = [bench.oracle_phases(w, {N_sample}, {nrhs}) for _ in range({steps})]; "
            f"print(json.dumps(ts))")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True)
    if r.returncode != 0:
        return {"error": r.stderr[-400:]}
    return {"phases": json.loads(r.stdout.strip().splitlines()[-1]), "cores": cores}


def cpu_estimate(w, phases: dict) -> tuple:
    """(RHS/s of the oracle at the workload's full size, seconds per step, sample text):
    the sampled phases extrapolated to every problem of the workload."""
    sizes = _full_sizes(w)
    N_s = min(CPU_SAMPLE_N, min(sizes))
    secs = sum(extrapolate(phases, N_s, n, w.m) for n in sizes)
    rhs = w.nrhs * len(sizes)
    what = (f"extrapolated: oracle factor+solve of N={N_s} points of the {w.name} generator "
            f"(same h, lambda, m, s_max, tol, {w.nrhs} RHS), each phase scaled to "
            + (f"N={sizes[0]}" if len(sizes) == 1 else f"each of the {len(sizes)} problems' N")
            + " by its complexity (tree N log N, kNN N^2, skeletonization per node, "
              "factorization N L^2, solve N L; L = tree depth)")
    if w.kind == "batched":
        what = what.replace(f"N={N_s} points of the {w.name} generator",
                            f"the first {N_s} points of the batch's first problem")
    return rhs / secs, secs, what


def cpu_baseline_entry(w) -> dict:
    """The line's cpu_baseline: one sampled oracle run on all host cores, extrapolated."""
    res = cpu_baseline_subprocess(w.name, min(CPU_SAMPLE_N, min(_full_sizes(w))), w.nrhs, 1)
    if "error" in res:
        return {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                "sample": "failed: " + res["error"][-200:]}
    value, secs, what = cpu_estimate(w, res["phases"][0])
    return {"value": value, "unit": UNIT, "cores": res["cores"], "kind": "oracle", "extrapolated": True,
            "seconds_per_step": secs,
            "sampled_phases_s": {k: round(v, 3) for k, v in res["phases"][0].items()}, "sample": what}


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    res = cpu_baseline_subprocess(w.name, min(CPU_SAMPLE_N, min(_full_sizes(w))), w.nrhs,
                                  args.warmup + args.steps)
    if "error" in res:
        print(json.dumps({"impl": "reference", "unavailable": "oracle failed: " + res["error"][-200:]}))
        return 0
    per = [cpu_estimate(w, ph) for ph in res["phases"][args.warmup:]]
    total = float(sum(p[1] for p in per))
    rhs = w.nrhs * len(_full_sizes(w))
    value = rhs * len(per) / total
    sample_s = float(sum(sum(ph.values()) for ph in res["phases"][args.warmup:]))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(per),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_of(w), "same_config": True, "extrapolated": True,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": res["cores"], "kind": "oracle",
                         "sample": per[0][2] + f"; sampled oracle time {sample_s:.1f} s over "
                                   f"{len(per)} steps"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def config_of(w):
    if w.kind == "batched":
        return {"workload": "C3: 64 independent problems, N log-uniform in [2048, 65536], d=16, "
                            "uniform; h in {0.3,0.6,1.2}, lambda in {1e-1,1e-3}",
                "problems": 64, "d": 16, "leaf_m": w.m, "s_max": w.s_max, "tol": w.tol,
                "nrhs_per_problem": w.nrhs, "kappa": w.kappa,
                "l2": "inputs and working set larger than L2 (no flush needed)"}
    kinds = {"gmm": f"{w.ncomp}-component Gaussian mixture, axis std in [{w.std_lo}, {w.std_hi}]",
             "manifold": "random 2-layer tanh image of N(0, I_6) plus 0.01 noise",
             "uniform": "uniform on the unit cube"}
    return {"workload": f"{w.name}: N={w.N}, d={w.d}, {kinds.get(w.kind, w.kind)}", "N": w.N, "d": w.d, "h": w.h,
            "lambda": w.lam, "leaf_m": w.m, "s_max": w.s_max, "tol": w.tol, "nrhs": w.nrhs,
            "kappa": w.kappa, "path": "plain FP64",
            "l2": "inputs and working set larger than L2 (no flush needed)"}


# ------------------------------------------------------------------- GPU leg
FP32_LANES_PER_SM = 128              # GB300: FP32 FMA lanes per SM
PEAK_CLASS = {                       # kernel classes whose arithmetic is FP32
    "kernel_blocks_f32", "cpqr_id_f32", "getrf_f32", "getrs_f32", "getri_f32"}
PAIR_INSTR_PER_MAC = 12              # FP32 instructions of one FP32-pair multiply-add
FP64_EQUIV_NOTE = {                  # classes whose flops count FP64 work done partly elsewhere
    "kernel_blocks_sliced": "FP64-equivalent flops (2d + 3 per entry, the FP64 Gram form's); the dot "
                            "products run on the BF16 tensor cores from exact digits, so the fraction of "
                            "the FP64 pipe can exceed 1"}
HBM_CLASS = {                        # memory-bound classes: algorithmic bytes / time vs HBM
    "operator_slices",               # FP64 operator blocks as BF16 digits (14 B per entry) on the tensor cores
    "slice_split"}
TENSOR_CLASS = {                     # tensor-core classes: nominal dense rate / bf16's
    "knn": (1.1 / 2.25, "TF32"),     # tcgen05 3xTF32 distance tiles, algorithmic work once
    "gemm_f32": (1.1 / 2.25, "TF32"),  # tcgen05 3xTF32 tiles (FP32 CUDA-core tiles with gemm_tc=0)
    "mlp_bf16": (1.0, "BF16"),
}


def measure_gemm_peaks() -> dict:
    """Dense TF32 and FP64 rates of this GPU, measured in this run with the library GEMM
    (torch.matmul on cuBLAS: FP32 operands with TF32 allowed, 8192^3; FP64, 4096^3),
    best of 10 after 3 warm-ups, CUDA events: the denominators of the tensor (TF32) and
    FP64 roofline fractions, as MEASURED_PEAKS.json's bf16 figure is for BF16."""
    import torch
    out = {}
    saved = torch.backends.cuda.matmul.allow_tf32
    try:
        torch.backends.cuda.matmul.allow_tf32 = True
        for name, dt, n in (("tf32_tflops", torch.float32, 8192), ("fp64_tflops", torch.float64, 4096)):
            a = torch.randn(n, n, dtype=dt, device="cuda")
            b = torch.randn(n, n, dtype=dt, device="cuda")
            for _ in range(3):
                torch.matmul(a, b)
            best = float("inf")
            for _ in range(10):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            out[name] = 2.0 * n ** 3 / (best / 1e3) / 1e12
            del a, b
        torch.cuda.empty_cache()
    finally:
        torch.backends.cuda.matmul.allow_tf32 = saved
    return out


def roof_peak(kernel: str, pk: dict, src: str, gp: dict = None) -> tuple:
    """(bound, peak TFLOP/s, how) for a kernel class; gp = measure_gemm_peaks()."""
    gp = gp or {}
    if kernel in TENSOR_CLASS:
        ratio, dt = TENSOR_CLASS[kernel]
        if dt == "TF32" and gp.get("tf32_tflops"):
            return ("tensor", gp["tf32_tflops"],
                    f"measured in this run: cuBLAS TF32 GEMM 8192^3 {gp['tf32_tflops']:.0f} TFLOP/s (burst)")
        return ("tensor", pk["bf16_tflops"] * ratio,
                f"{src} bf16 {pk['bf16_tflops']:.0f} TFLOP/s x nominal {dt}/BF16 ratio {ratio:.3f}")
    if kernel not in PEAK_CLASS and kernel != "gemm_pair" and gp.get("fp64_tflops"):
        return ("alu", gp["fp64_tflops"],
                f"measured in this run: cuBLAS FP64 GEMM 4096^3 {gp['fp64_tflops']:.2f} TFLOP/s (burst)")
    peak, how = alu_peak_tflops(kernel, pk.get("sm_max_mhz", 2070.0))
    return ("alu", peak, f"{how} ({src} max clock)")


def class_roof(kernel: str, v: dict, pk: dict, src: str, gp: dict = None):
    """(bound, achieved, peak, unit, how) of one kernel class from its summed event time
    and algorithmic work (bytes for the memory-bound classes, else flops); None without."""
    if v["ms"] <= 0:
        return None
    if kernel in HBM_CLASS and v.get("bytes", 0) > 0:
        return ("hbm", v["bytes"] / (v["ms"] / 1e3) / 1e9, pk["hbm_gbs"], "GB/s",
                f"{src} HBM copy bandwidth {pk['hbm_gbs']:.0f} GB/s")
    if v["flops"] <= 0:
        return None
    bound, peak, how = roof_peak(kernel, pk, src, gp)
    return (bound, v["flops"] / (v["ms"] / 1e3) / 1e12, peak, "TFLOP/s", how)


def alu_peak_tflops(kernel: str, sm_mhz: float) -> tuple:
    if kernel == "gemm_pair":          # 2 algorithmic flops per pair multiply-add
        return (SM_COUNT * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / PAIR_INSTR_PER_MAC / 1e12,
                f"derived: {SM_COUNT} SMs x {FP32_LANES_PER_SM} FP32 instr/clk x {sm_mhz:.0f} MHz "
                f"/ {PAIR_INSTR_PER_MAC} instr per pair multiply-add x 2 flops")
    if kernel in PEAK_CLASS:
        return (SM_COUNT * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12,
                f"derived: {SM_COUNT} SMs x {FP32_LANES_PER_SM} FP32 FMA/clk x {sm_mhz:.0f} MHz")
    return (SM_COUNT * FP64_FMA_PER_CLK_PER_SM * 2 * sm_mhz * 1e6 / 1e12,
            f"derived: {SM_COUNT} SMs x {FP64_FMA_PER_CLK_PER_SM} FP64 FMA/clk x {sm_mhz:.0f} MHz")


def batched_measure(w, form, steps, warmup, dist, rank, local, sample_clocks=True, with_e2e=True):
    """C3: all problems in one batched factor + solve per step vs one call per problem.
    Under torchrun every rank factors a batch of 64 problems of its own (weak scaling, no
    data-path exchange); the time is the largest over the ranks."""
    import torch
    import paper_1602_01376_gb300 as ia
    world = int(os.environ.get("WORLD_SIZE", "1"))
    probs = batched_problems(count=64, seed=batch_seed(rank))
    Ns = [len(p[0]) for p in probs]
    hs = [p[1] for p in probs]
    lams = [p[2] for p in probs]
    Xall = torch.from_numpy(np.ascontiguousarray(np.concatenate([p[0] for p in probs]))).cuda()
    rng = np.random.default_rng(w.seed + 7)
    U0 = torch.from_numpy(np.concatenate([rng.standard_normal(n * w.nrhs) for n in Ns])).cuda()
    U = torch.empty_like(U0)
    ia.iaskit_set_option("precision", 1 if form == "mixed" else 0)
    ia.iaskit_set_option("refine", 400 if form == "mixed" else 20)
    ia.iaskit_set_option("refine_tol", 1e-10)
    Xs = [Xall[sum(Ns[:q]):sum(Ns[:q + 1])] for q in range(len(Ns))]
    offs = np.concatenate([[0], np.cumsum([n * w.nrhs for n in Ns])])

    def step_batched():
        ia.iaskit_factor_batched_device(Xall, Ns, hs, lams, w.m, w.s_max, w.tol)
        U.copy_(U0)
        ia.iaskit_solve_batched_device(U, w.nrhs)

    def step_single():
        for q in range(len(Ns)):
            ia.iaskit_factor_device(Xs[q], hs[q], lams[q], w.m, w.s_max, w.tol)
            Uq = U[offs[q]:offs[q + 1]].view(w.nrhs, Ns[q])
            Uq.copy_(U0[offs[q]:offs[q + 1]].view(w.nrhs, Ns[q]))
            ia.iaskit_solve_device(Uq)

    def timed(fn, clocks_on):
        for _ in range(warmup):
            fn()
        ia.iaskit_set_option("profile", 1)
        l0 = ia.iaskit_stats()["launches"]
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(dist)
        torch.cuda.synchronize()
        with ClockSampler(local if clocks_on else -1) as clk:
            ev0.record()
            for _ in range(steps):
                fn()
            ev1.record()
            torch.cuda.synchronize()
        barrier(dist)
        st = ia.iaskit_stats()
        ia.iaskit_set_option("profile", 0)
        ms = max_over_ranks(dist, ev0.elapsed_time(ev1), "cuda")
        return ms, st, clk.summary(), st["launches"] - l0

    ms_b, st_b, clocks, launches = timed(step_batched, sample_clocks)
    ms_s, st_s, _, launches_s = timed(step_single, False)
    nrhs_total = w.nrhs * len(Ns)
    # residual of the batched solution against the operator, every problem and column
    step_batched()
    AU = torch.empty_like(U)
    ia.iaskit_apply_device(U, AU, w.nrhs)
    resid, above = 0.0, 0
    for q in range(len(Ns)):
        a, b = offs[q], offs[q + 1]
        r = (U0[a:b] - AU[a:b]).view(w.nrhs, Ns[q]).norm(dim=1) / U0[a:b].view(w.nrhs, Ns[q]).norm(dim=1)
        resid = max(resid, float(r.max()))
        above += int(float(r.max()) > 1e-10)
    st_last = ia.iaskit_stats()
    out = {"ms": ms_b, "stats": st_b, "clocks": clocks, "launches": launches, "ms_single": ms_s,
           "launches_single": launches_s, "resid": resid, "above": above, "st_last": st_last,
           "nrhs_total": nrhs_total, "Ns": Ns, "world": world}
    if with_e2e:
        # end to end: host points and right-hand sides through iaskit_factor_batched / solve_batched
        Xh = [np.ascontiguousarray(p[0]) for p in probs]
        Uh = [np.ascontiguousarray(U0[offs[q]:offs[q + 1]].cpu().numpy().reshape(w.nrhs, Ns[q]).T)
              for q in range(len(Ns))]
        barrier(dist)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ia.iaskit_factor_batched(Xh, hs, lams, w.m, w.s_max, w.tol)
        ia.iaskit_solve_batched(Uh)
        out["e2e_s"] = max_over_ranks(dist, time.perf_counter() - t0, "cuda")
    return out


def batched_summary(w, res, steps):
    """The C3 figures of a batched_measure result (shared by the C3 line and the C3 entry
    of the default line)."""
    st = res["st_last"]
    world = res["world"]
    return {
        "value": world * res["nrhs_total"] * steps / (res["ms"] / 1e3), "unit": UNIT,
        "ms_per_step": res["ms"] / steps, "steps": steps, "residual": res["resid"],
        "problems_above_1e-10": res["above"], "refine_stagnated_columns": st.get("refine_stagnated"),
        "stagnated": st.get("stagnated"), "refine_gmres_iters": st.get("refine_iters"),
        "fp64_problems": st.get("fp64_problems"), "fp64_operator_problems": st.get("fp64_operator_problems"),
        "operator_upgrades": st.get("operator_upgrades"), "gpu_launches": res["launches"],
        "compare_per_problem": {"value": world * res["nrhs_total"] * steps / (res["ms_single"] / 1e3),
                                "ms_per_step": res["ms_single"] / steps,
                                "gpu_launches": res["launches_single"]},
    }


def run_batched(args, w, form):
    import torch
    import paper_1602_01376_gb300 as ia
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = dist_init("nccl")
    ia.load()
    ia.iaskit_set_stream(None)
    res = batched_measure(w, form, args.steps, args.warmup, dist, rank, local)
    if rank != 0:
        dist.destroy_process_group()
        return 0
    kern = res["stats"]["kernels"]
    top = max(kern, key=lambda k: kern[k]["ms"])
    pk, src = peaks()
    roof = None
    cr = class_roof(top, kern[top], pk, src, measure_gemm_peaks())
    if cr is not None:
        bound, achieved, peak, unit, how = cr
        roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak, "traffic": None, "kernel": top,
                "peak_source": how, "launches": kern[top]["calls"],
                "ms_total": kern[top]["ms"]}
    world = res["world"]
    cfg = config_of(w)
    cfg["path"] = "batched " + form
    if world > 1:
        cfg["ranks"] = f"{world} ranks, each its own batch of 64 problems (seed + 1000 rank)"
    summ = batched_summary(w, res, args.steps)
    line = {
        "metric": METRIC, "value": summ["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": summ["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if form == "mixed" else "f64",
        "data": "synthetic", "config": cfg, "clocks": res["clocks"], "roofline": roof,
        "kernel_ms_per_step": {k: round(v["ms"] / args.steps, 3) for k, v in kern.items() if v["ms"] > 0},
        "e2e": {"value": world * res["nrhs_total"] / res["e2e_s"], "unit": UNIT,
                "h2d_bytes_per_step": 8 * sum(res["Ns"]) * (16 + w.nrhs),
                "d2h_bytes_per_step": 8 * sum(res["Ns"]) * w.nrhs},
    }
    for k in ("residual", "problems_above_1e-10", "refine_stagnated_columns", "stagnated", "refine_gmres_iters",
              "fp64_problems", "fp64_operator_problems", "operator_upgrades", "gpu_launches", "compare_per_problem"):
        line[k] = summ[k]
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_entry(w)
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="C4")
    ap.add_argument("--form", choices=["mixed", "fp64"], default="mixed",
                    help="form timed for the headline value (mixed = the chosen form)")
    ap.add_argument("--no-compare", action="store_true", help="skip timing the other form")
    ap.add_argument("--N", type=int, default=None, help="override N (testing only)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the C3 entry of the default line")
    args = ap.parse_args()
    w = workload(args.workload, N=args.N)
    if args.impl == "reference":
        return run_reference(args, w)
    if w.kind == "batched":
        return run_batched(args, w, args.form)

    import torch
    import paper_1602_01376_gb300 as ia

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = dist_init("nccl")

    ia.load()
    ia.iaskit_set_stream(None)                     # legacy default stream = torch's default
    X = torch.from_numpy(make_points(w)).cuda()
    U0 = torch.from_numpy(np.ascontiguousarray(make_rhs(w).T)).cuda()   # (nrhs, N): N x nrhs col-major
    U = torch.empty_like(U0)
    args_f = (w.h, w.lam, w.m, w.s_max, w.tol)

    def set_form(form):
        # both forms refine against the FP64 operator to the metric's 1e-10; the FP64
        # factorization usually needs no correction, the FP32 one a few GMRES-IR steps
        ia.iaskit_set_option("precision", 1 if form == "mixed" else 0)
        ia.iaskit_set_option("refine", 400 if form == "mixed" else 20)
        ia.iaskit_set_option("refine_tol", 1e-10)

    def step():
        ia.iaskit_factor_device(X, *args_f)
        U.copy_(U0)
        ia.iaskit_solve_device(U)

    # sampled eps_M (eq. error, S = 0) of the current factorization: ||K w - K~ w|| / ||K w||
    # on EPS_M_ROWS seeded rows, K w by exact kernel sums (iaskit_predict), K~ w by the
    # operator apply minus lambda w
    erng = np.random.default_rng(w.seed + 11)
    e_rows = torch.from_numpy(np.sort(erng.choice(w.N, EPS_M_ROWS, replace=False))).cuda()
    e_w = torch.from_numpy(erng.standard_normal(w.N)).cuda()

    def eps_M():
        T = X[e_rows].contiguous()
        Kw = torch.empty(EPS_M_ROWS, dtype=torch.float64, device="cuda")
        ia.iaskit_predict_device(T, e_w, Kw)
        Aw = torch.empty_like(e_w)
        ia.iaskit_apply_device(e_w, Aw)
        Ktw = (Aw - w.lam * e_w)[e_rows]
        return float((Kw - Ktw).norm() / Kw.norm())

    def measure(form, sample_clocks, steps, warmup):
        set_form(form)
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        AU = torch.empty_like(U)
        ia.iaskit_apply_device(U, AU)             # residual against the FP64 operator
        resid = float(((U0 - AU).norm(dim=1) / U0.norm(dim=1)).max())
        ia.iaskit_set_option("profile", 1)
        launches0 = ia.iaskit_stats()["launches"]
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(dist)
        torch.cuda.synchronize()
        with ClockSampler(local if sample_clocks else -1) as clk:
            ev0.record()
            for _ in range(steps):
                step()
            ev1.record()
            torch.cuda.synchronize()
        barrier(dist)
        ms = max_over_ranks(dist, ev0.elapsed_time(ev1), "cuda")
        stats = ia.iaskit_stats()
        ia.iaskit_set_option("profile", 0)
        return {"ms": ms, "stats": stats, "resid": resid, "clocks": clk.summary(),
                "launches": stats["launches"] - launches0, "eps_M": eps_M(), "steps": steps}

    chosen = measure(args.form, True, args.steps, args.warmup)
    other_form = "fp64" if args.form == "mixed" else "mixed"
    other = None if args.no_compare else measure(other_form, False, min(args.steps, COMPARE_STEPS),
                                                 min(args.warmup, 1))
    set_form(args.form)
    value = world * w.nrhs * args.steps / (chosen["ms"] / 1e3)

    # refactor for a new lambda (Sec. II-C): tree, kNN lists, skeletons and P are kept,
    # the leaf LUs, U, W and Z formed again; timed alternating lambda x 10 and lambda
    ia.iaskit_factor_device(X, *args_f)
    ia.iaskit_refactor(w.lam * 10.0)
    torch.cuda.synchronize()
    n_ref = 4
    t0 = time.perf_counter()
    for k in range(n_ref):
        ia.iaskit_refactor(w.lam if k % 2 == 0 else w.lam * 10.0)
    torch.cuda.synchronize()
    refactor_ms = (time.perf_counter() - t0) * 1e3 / n_ref
    ia.iaskit_refactor(w.lam)
    U.copy_(U0)
    ia.iaskit_solve_device(U)
    AU = torch.empty_like(U)
    ia.iaskit_apply_device(U, AU)
    refactor_resid = float(((U0 - AU).norm(dim=1) / U0.norm(dim=1)).max())

    # end to end through the host API: pinned host inputs in, solution out
    Xh = torch.from_numpy(make_points(w)).pin_memory()
    U_src = torch.from_numpy(np.ascontiguousarray(make_rhs(w).T))       # (nrhs, N)
    Uh = torch.empty((w.nrhs, w.N), dtype=torch.float64).pin_memory()
    Uh.copy_(U_src)
    Xh_np, Uh_view = Xh.numpy(), Uh.numpy()
    lib = ia.load()
    e2e_steps = max(1, min(args.steps, 2))
    barrier(dist)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        rc = lib.iaskit_factor(Xh_np.ctypes.data, w.N, w.d, *args_f)
        if rc != 0:
            raise RuntimeError(ia.iaskit_last_error())
        rc = lib.iaskit_solve(Uh_view.ctypes.data, w.nrhs)
        if rc != 0:
            raise RuntimeError(ia.iaskit_last_error())
        Uh.copy_(U_src)                            # restore the right-hand sides
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(dist, time.perf_counter() - t0, "cuda")
    e2e_value = world * w.nrhs * e2e_steps / e2e_s

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    pk, src = peaks()
    kern = chosen["stats"]["kernels"]
    top = max(kern, key=lambda k: kern[k]["ms"])
    clocks = chosen["clocks"]
    roof = None
    gp = measure_gemm_peaks()
    cr = class_roof(top, kern[top], pk, src, gp)
    if cr is not None:
        bound, achieved, peak, unit, how = cr
        roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak, "traffic": None, "kernel": top,
                "peak_source": how,
                "launches": kern[top]["calls"], "ms_total": kern[top]["ms"]}
        # every class against the peak of its pipe and type (HBM for the memory-bound ones)
        roof["by_class"] = {}
        for k, v in kern.items():
            ck = class_roof(k, v, pk, src, gp)
            if ck is not None:
                b_k, a_k, p_k, u_k, _ = ck
                roof["by_class"][k] = {"ms_per_step": round(v["ms"] / args.steps, 3), "achieved": round(a_k, 3),
                                       "peak": round(p_k, 2), "unit": u_k, "frac": round(a_k / p_k, 4),
                                       "bound": b_k}
                if k in FP64_EQUIV_NOTE:
                    roof["by_class"][k]["note"] = FP64_EQUIV_NOTE[k]
        roof["measured_peaks"] = gp
    st = chosen["stats"]
    cfg = config_of(w)
    cfg["path"] = ("mixed: FP32 factorization, FP64 pivots and operator, refined to 1e-10; "
                   "neighbour + uniform row sampling" if args.form == "mixed" else "plain FP64")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": chosen["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if args.form == "mixed" else "f64", "data": "synthetic",
        "config": cfg,
        "factor_s": st["ms"]["factor"] / 1e3, "solve_rhs_per_s": w.nrhs / (st["ms"]["solve"] / 1e3),
        "residual": chosen["resid"],
        "eps_M": {"chosen": chosen["eps_M"], "fp64_plain": other["eps_M"] if other else None,
                  "rows": EPS_M_ROWS,
                  "what": "||K w - K~ w|| / ||K w|| on seeded rows (eq. error, S = 0), K w by exact "
                          "kernel sums, w ~ N(0,1): equal accuracy needs chosen <= fp64_plain"},
        "refine_sweeps": st.get("refine_sweeps"),
        "refine_gmres_iters": st.get("refine_iters"), "refine_stagnated_columns": st.get("refine_stagnated"),
        "fp64_problems": st.get("fp64_problems"),
        "fp64_operator_problems": st.get("fp64_operator_problems"),
        "operator_upgrades": st.get("operator_upgrades"),
        "knn_exact_fallback_rows": st.get("knn_fallback"),
        "gpu_launches": chosen["launches"], "clocks": clocks, "roofline": roof,
        "kernel_ms_per_step": {k: round(v["ms"] / args.steps, 3) for k, v in kern.items() if v["ms"] > 0},
        "kernel_tflops": {k: round(v["flops"] / (v["ms"] / 1e3) / 1e12, 3)
                          for k, v in kern.items() if v["ms"] > 0 and v["flops"] > 0},
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": 8 * w.N * (w.d + w.nrhs), "d2h_bytes_per_step": 8 * w.N * w.nrhs},
    }
    line["refactor"] = {"ms": refactor_ms, "factor_ms": st["ms"]["factor"],
                        "factor_over_refactor": st["ms"]["factor"] / refactor_ms,
                        "residual_after": refactor_resid,
                        "what": "iaskit_refactor alternating lambda x 10 and lambda (host wall "
                                "clock, synchronized); then a solve at lambda"}
    if other is not None:
        so = other["stats"]
        line["compare_" + other_form] = {
            "value": world * w.nrhs * other["steps"] / (other["ms"] / 1e3),
            "steps": other["steps"], "warmup": min(args.warmup, 1),
            "sampled_steps": other["steps"] < args.steps,
            "ms_per_step": other["ms"] / other["steps"], "factor_s": so["ms"]["factor"] / 1e3,
            "solve_rhs_per_s": w.nrhs / (so["ms"]["solve"] / 1e3), "residual": other["resid"],
            "kernel_ms_per_step": {k: round(v["ms"] / other["steps"], 3)
                                   for k, v in so["kernels"].items() if v["ms"] > 0}}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_entry(w)
    if not args.no_batched:
        # the batching workload (C3: 64 independent problems in one batched launch per
        # level) on the same GPU, a few steps, beside the headline line
        wb = workload("C3")
        bsteps = min(args.steps, COMPARE_STEPS)
        res = batched_measure(wb, "mixed", bsteps, 1, None, 0, local, sample_clocks=False, with_e2e=False)
        line["batched_C3"] = dict(batched_summary(wb, res, bsteps), warmup=1,
                                  workload=config_of(wb)["workload"])
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
