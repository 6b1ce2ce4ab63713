#!/usr/bin/env python
"""Benchmark of the shift-and-invert eigensolution on one GB300 per rank.

Workload (the 2D configuration of Table 3's 256^2 p=3 row, with rIGA blocks
of 16 elements): Laplace on the unit square, Dirichlet, B-spline degree 3,
256x256 elements, C0 separator lines every 16 elements (N = 82,369), lowest
100 eigenpairs in two spectrum slices of 50 (sigma = 0, then the check shift
after the 50th), FP64 fronts.  One step = riga_eigs (factorizations,
Lanczos, Rayleigh-Ritz, inertia checks, residuals), the eigensolution the
paper times; the numeric assembly is timed apart (assembly_ms) and the
symbolic analysis is once per mesh pattern.  The end-to-end figure (e2e)
includes the assembly and the host copies.  Metric: converged eigenpairs per
second at residual <= 1e-10.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl riga|reference]
                    [--precision fp64|fp32] [--mesh riga|iga]

Under torchrun each rank solves its own copy (replicas: the single eigenproblem
does not shard); value = pairs of all ranks / max step time over ranks.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# the CPU baseline is the single-threaded oracle: pin BLAS before numpy loads
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

METRIC = "eigenpairs/s at resid<=1e-10"
RESID_TOL = 1e-10


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="riga", choices=["riga", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "tf32", "bf16"])
    ap.add_argument("--mesh", default="riga", choices=["riga", "iga", "c3", "c3s", "c4"],
                    help="riga / iga: the 2D 256^2 p=3 meshes (100 pairs, 2 slices); c3: 3D 64^3 p=2 rIGA bs8, "
                         "50 pairs; c4: batch of 512 2D rIGA problems with random coefficients, 20 pairs each")
    ap.add_argument("--block", type=int, default=2, choices=[0, 1, 2, 4],
                    help="Lanczos block size (riga_set_eig_block; 0 = automatic)")
    ap.add_argument("--fp64-update", default="tc", choices=["fma", "tc"],
                    help="Schur updates of FP64 fronts: FP64 FMA on the CUDA cores, or digit slices on the tensor cores")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-mixed", action="store_true", help="skip the low-precision-front (mixed) leg")
    ap.add_argument("--mixed-precision", default="tf32", choices=["fp32", "tf32"],
                    help="fronts of the mixed leg: tf32 (Schur updates on the tensor cores) or fp32 (FFMA)")
    ap.add_argument("--no-profile-pass", action="store_true", help="skip the phase-timing pass")
    ap.add_argument("--c3-steps", type=int, default=2,
                    help="timed steps of the 3D 64^3 p=2 rIGA workload (50 pairs), FP64 path and mixed path, "
                         "reported as the 'c3' object of the default run (0 = skip)")
    ap.add_argument("--trace-out", default="solve_trace.npz",
                    help="--mode trace: file for the per-item solve trace (npz)")
    ap.add_argument("--sweep-dim", type=int, default=2, help="--mode bs-sweep: 2 (256^2 p=3) or 3 (32^3 p=2)")
    ap.add_argument("--sweep-pairs", type=int, default=100, help="--mode bs-sweep: eigenpairs per eigensolve")
    ap.add_argument("--interval-pairs", type=int, default=1024,
                    help="--mode interval: about this many eigenpairs (the interval [0, hi) with hi from Weyl's law)")
    ap.add_argument("--mode", default="eigs", choices=["eigs", "solve", "factor", "trace", "bs-sweep", "interval"],
                    help="eigs: the benchmark; solve / factor: a short program (one factorization and "
                         "--steps solves, or --steps factorizations) of the same workload, for profilers")
    return ap.parse_args()


def workload(mesh_kind):
    from paper_2009_08167_gb300.inputs import config_c2, config_c3, config_c4
    if mesh_kind == "c4":
        import numpy as np
        probs = config_c4()
        return {"batch": True, "meshes": [p["mesh"] for p in probs], "coefK": [np.exp(p["a"]) for p in probs],
                "k": probs[0]["k"], "slice": probs[0]["k"], "sigma": 0.0}
    if mesh_kind == "c3":
        cfg = config_c3()
        cfg["slice"] = cfg["k"]
        return cfg
    if mesh_kind == "c3s":
        # the 3D family at 32^3 elements (N = 42,875, fronts up to 1820
        # variables): kernel profiles on a case a few GB in size
        from paper_2009_08167_gb300.inputs import Mesh
        return dict(mesh=Mesh(3, 32, 2, 8), k=50, sigma=0.0, slice=50)
    cfg = config_c2(riga=(mesh_kind == "riga"))
    return cfg


def config_dict(args, cfg, extra=None):
    if cfg.get("batch"):
        ms = cfg["meshes"]
        d = {
            "workload": f"batch{len(ms)}_laplace2d_riga_ne32-128_p2-3_bs8-16_lognormal-coef_k{cfg['k']}",
            "problems": len(ms), "pairs_per_problem": cfg["k"], "elements_per_side": "U{32..128}",
            "degree": "{2,3}", "block_size": "{8,16}", "coefficient": "exp(a_e), a_e~N(0,0.5^2)",
            "factor_precision": "fp64", "l2": "flushed between timed steps (512 MiB write)",
            "parallelism": f"replicas{args.gpus}",
        }
        if extra:
            d.update(extra)
        return d
    m = cfg["mesh"]
    d = {
        "workload": f"laplace{m.dim}d_p{m.p}_{'x'.join(str(v) for v in m.ne)}_{'riga_bs%d' % m.bs if m.bs else 'iga'}_k{cfg['k']}_slices{cfg['k'] // cfg['slice']}",
        "dim": m.dim, "elements_per_side": m.ne[0], "degree": m.p, "block_size": m.bs, "leaf_extent": m.leaf_extent,
        "pairs": cfg["k"], "slice": cfg["slice"], "factor_precision": args.precision, "fp64_update": args.fp64_update, "lanczos_block": args.block,
        "l2": "flushed between timed steps (512 MiB write)",
        "parallelism": f"replicas{args.gpus}",
    }
    if extra:
        d.update(extra)
    return d


# ------------------------------------------------------------------ clocks
class Clocks:
    def __init__(self, index):
        self.path = tempfile.mktemp(suffix=".csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def ncu_traffic(phase):
    """DRAM bytes per launch of the phase's kernel from the committed ncu
    summary (profiles/ncu_traffic.txt: '<phase> <bytes_per_call> <source>'),
    as (bytes, source), or None when the file has no line for the phase (a
    kernel changed since its counters were taken has its line removed)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        body, _, note = line.partition("#")
        parts = body.split()
        if len(parts) >= 2 and parts[0] == phase:
            src = " ".join(parts[2:]) or note.strip()
            return float(parts[1]), "ncu dram__bytes_read.sum + dram__bytes_write.sum, profiles/ncu_traffic.txt (" + src + ")"
    return None


# ------------------------------------------------------------- oracle leg
def oracle_sample(cfg):
    """The FP64 oracle as it stands (shift-invert Lanczos with banded LDL^T)
    on a bounded sample of the workload's family: 2D meshes at 48x48 elements
    with the workload's degree and C0 lines (100 pairs); 3D meshes at 10^3
    elements with the workload's degree and C0 planes (up to 50 pairs; the
    banded 3D factorization grows too fast for larger samples).  Returns
    (pairs/s, seconds, description)."""
    import numpy as np
    from oracle import assembly, eigen
    from paper_2009_08167_gb300.inputs import Mesh
    w = cfg["mesh"]
    if w.dim == 3:
        m, k = Mesh(3, 10, w.p, w.bs), min(int(cfg["k"]), 50)
        shape = "10x10x10"
    else:
        m, k = Mesh(2, 48, w.p, w.bs), 100
        shape = "48x48"
    fam = f"rIGA bs{w.bs}" if w.bs else "IGA"
    t0 = time.perf_counter()
    K, M = assembly.assemble_kron(m.dim, m.ne, m.p, m.mults)
    lam, U, info = eigen.lanczos_shift_invert(K, M, k, 0.0, tol=1e-12, seed=1)
    rho = eigen.residual_rho(K, M, lam, U)
    dt = time.perf_counter() - t0
    ok = int(np.sum(rho <= RESID_TOL))
    desc = (f"oracle shift-invert Lanczos + banded LDL^T, {m.dim}D p={m.p} {fam} at {shape} elements (N={K.n}), "
            f"{ok} of {k} pairs at resid<=1e-10, {dt:.1f} s, 1 thread of numpy/BLAS")
    return ok / dt, dt, desc


def oracle_sample_batch(cfg, budget_s=15.0):
    """The oracle as it stands on a bounded sample of the batch: its problems
    from the smallest up until about budget_s seconds of CPU work (larger
    problems take the banded oracle up to ~100 s each, so the sample favours
    the oracle).  Returns (pairs/s, seconds, description)."""
    import numpy as np
    from oracle import assembly, eigen
    t0 = time.perf_counter()
    ok = done = 0
    order = sorted(range(len(cfg["meshes"])), key=lambda i: (int(np.prod(cfg["meshes"][i].ne)), i))
    for i in order:
        m, c = cfg["meshes"][i], cfg["coefK"][i]
        K, M = assembly.assemble_coef(m.dim, m.ne, m.p, m.mults, c, None)
        lam, U, info = eigen.lanczos_shift_invert(K, M, cfg["k"], cfg["sigma"], tol=1e-12, seed=1)
        ok += int(np.sum(eigen.residual_rho(K, M, lam, U) <= RESID_TOL))
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    desc = (f"oracle shift-invert Lanczos + banded LDL^T on the {done} smallest problems of the batch, "
            f"{ok} pairs at resid<=1e-10, {dt:.1f} s, 1 thread of numpy/BLAS")
    return ok / dt, dt, desc


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def run_reference(args, rank, world):
    if rank != 0:
        return
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    cfg = workload(args.mesh)
    sample = (lambda: oracle_sample_batch(cfg)) if cfg.get("batch") else (lambda: oracle_sample(cfg))
    for _ in range(args.warmup):
        sample()
    vals, secs = [], []
    desc = ""
    for _ in range(args.steps):
        v, dt, desc = sample()
        vals.append(v)
        secs.append(dt)
    value = statistics.mean(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "eigenpairs/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(args, cfg),
        "cpu_baseline": {"value": value, "unit": "eigenpairs/s", "cores": 1, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "eigenpairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def roofline(prof, q=None):
    """Roofline of the dominant phase of one profiled step (device time of
    the phase's launches, CUDA events on the library's stream), in the class
    the hot-path table assigns to it: the f/b solve, the SpMVs and the
    reorthogonalization are HBM-bound (algorithmic bytes: for the solve
    2 nnz(L) s_f + 4 N 8 b per launch with b right-hand sides, as the library
    records them; peak: the measured copy bandwidth, else the fallback), the
    fronts are bound by the FP64 rate on the FP64 path.  The FP64-pipe
    fraction of the same phase (algorithmic flops over the measured FP64
    rate) is reported beside it, labelled as such."""
    pk, pk_kind = peaks()
    dom = max(prof, key=lambda p: prof[p]["ms"])
    pr = prof[dom]
    if pr["ms"] <= 0:
        return None
    t = pr["ms"] / 1e3
    calls = max(1, pr["calls"])
    gbs = pr["bytes"] / t / 1e9
    tfl = pr["flops"] / t / 1e12
    out = {"phase": dom, "ms_per_call": pr["ms"] / calls, "calls": pr["calls"],
           "fp64_pipe_frac": tfl / FP64_PEAK_TFLOPS if pr["flops"] > 0 else None,
           "fp64_peak_tflops": FP64_PEAK_TFLOPS, "fp64_peak_source": FP64_PEAK_SOURCE}
    tr = ncu_traffic(dom)
    if dom == "factor":
        out.update({"bound": "alu", "achieved": tfl, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": tfl / FP64_PEAK_TFLOPS, "peak_source": FP64_PEAK_SOURCE,
                    "algorithmic_flops_per_call": pr["flops"] / calls, "traffic": tr[0] if tr else None,
                    "traffic_source": tr[1] if tr else None})
        return out
    out.update({"bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": gbs / pk["hbm_gbs"],
                "peak_source": pk_kind + " copy bandwidth", "algorithmic_bytes_per_call": pr["bytes"] / calls,
                "traffic": tr[0] if tr else None, "traffic_source": tr[1] if tr else None})
    return out


def aggregate(ms, pairs, world, dist=None, device="cpu"):
    """Whole-job throughput of replicas: the slowest rank's step time (max
    over ranks) and the pairs of all ranks (each rank solves its own copy).
    Returns (value in pairs/s, max ms per step)."""
    import torch
    ms_t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if dist is not None and world > 1:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
    ms_max = float(ms_t.item())
    return world * pairs / (ms_max / 1e3), ms_max


# Rates measured on a GB300 with a timed probe (CUDA events, clocks untouched):
# independent FMA chains on every SM for FP64 / FP32, back-to-back tcgen05.mma
# (M128 N256, operands in shared memory) for TF32.  The FP64 figure equals the
# nominal 2 DFMA per clock per SM at 2.07 GHz.
FP64_PEAK_TFLOPS = 1.255
FP64_PEAK_SOURCE = "measured (DFMA probe; nominal 1.25)"
FP32_PEAK_TFLOPS = 73.1
TF32_PEAK_TFLOPS = 1212.0


def fp64_front_peak(fp64_update):
    """Ceiling of FP64 fronts' updates: the measured FP64 FMA rate on the CUDA
    cores, or, with the digit-slice tensor-core update, the measured BF16
    tensor rate over the 36 BF16 products one FP64 multiply-add costs there
    (8 x 8 digit pairs down to level 7), as (TFLOP/s, source)."""
    if fp64_update == "tc":
        pk, kind = peaks()
        return pk["bf16_tflops"] / 36.0, kind + " bf16 tensor rate / 36 (digit-slice emulation of FP64)"
    return FP64_PEAK_TFLOPS, FP64_PEAK_SOURCE


def fronts_rate(prof, flops_plain, n_fact, peak, peak_source="measured probe"):
    """Front TFLOP/s of one profiled step: the plain multifrontal flops per
    factorization (lower triangle, FMA = 2, no padding and no augmentation)
    times the factorizations, over the factor phase's device time; also with
    the augmentation's flops counted (the work the kernels actually do)."""
    pr = prof.get("factor")
    if not pr or pr["ms"] <= 0 or n_fact <= 0:
        return None
    t = pr["ms"] / 1e3
    plain = flops_plain * n_fact / t / 1e12
    return {"tflops": plain, "peak": peak, "frac": plain / peak, "unit": "TFLOP/s",
            "tflops_incl_augmentation": pr["flops"] / t / 1e12, "factorizations": n_fact,
            "factor_ms": pr["ms"], "peak_source": peak_source}


# ------------------------------------------------------------------ riga leg
def run_riga_batch(args, rank, world, local_rank, cfg):
    """The batch workload: one step = numeric assembly of every problem +
    riga_eigs_batch (FP64)."""
    import numpy as np
    import torch
    from paper_2009_08167_gb300 import riga

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    meshes, cK, k = cfg["meshes"], cfg["coefK"], cfg["k"]
    R = riga.Riga(local_rank, stream)
    R.set_fp64_update(1 if args.fp64_update == "tc" else 0)
    R.set_eig_options(extra=2, seed=11)
    R.assemble_batch(meshes, cK)  # symbolic analysis of every pattern: once, untimed
    tuned_trail, tuned_ms = R.autotune()  # front tile shapes for this batch: once, untimed
    q = R.query()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def step():
        return R.eigs_batch(k, cfg["sigma"], RESID_TOL)

    # numeric assembly (new coefficients in, matrices out): reported apart
    # from the timed eigensolution, as the paper counts it
    asm_ms = []
    for _ in range(3):
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        R.assemble_batch(meshes, cK)
        a1.record(stream)
        a1.synchronize()
        asm_ms.append(a0.elapsed_time(a1))
    for _ in range(args.warmup):
        step()
    barrier()
    clk = Clocks(local_rank)
    launches0 = R.launches()
    times = []
    t_wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ev, rs, nc = step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    barrier()
    t_wall = time.perf_counter() - t_wall0
    clocks = clk.stop()
    launches = (R.launches() - launches0) // max(1, args.steps)
    pairs = int(np.sum(rs <= RESID_TOL))
    ms = statistics.mean(times)
    value, ms_max = aggregate(ms, pairs, world, dist, dev)
    st = R.stats()
    # end to end: host wall clock around the same public calls (coefficients
    # host -> device inside assembly, eigenvalues and residuals back)
    h2d = int(sum(c.nbytes for c in cK) + sum(np.asarray(mm, dtype=np.int32).nbytes for m in meshes for mm in m.mults))
    d2h = 8 * 2 * len(meshes) * k + 4 * len(meshes)
    e2e_times = []
    for _ in range(0 if args.no_e2e else max(1, min(args.steps, 3))):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        R.assemble_batch(meshes, cK)
        _, rsh, _ = step()
        e2e_times.append(time.perf_counter() - t0)
    e2e_val = world * int(np.sum(rsh <= RESID_TOL)) / statistics.mean(e2e_times) if e2e_times else None
    R.profile(True)
    if not args.no_profile_pass:
        step()
    prof = R.profile_get()
    R.profile(False)
    roof = roofline(prof, q)
    fronts = fronts_rate(prof, q["flops_fact"], R.stats()["n_fact"], *fp64_front_peak(args.fp64_update))
    phases = {p: {"ms": round(v["ms"], 3), "calls": v["calls"], "launches": v["launches"]} for p, v in prof.items() if v["calls"]}
    # the mixed path on the same batch: low-precision fronts, FP64 refinement
    mixed = None
    if not args.no_mixed:
        mprec = riga.RIGA_TF32 if args.mixed_precision == "tf32" else riga.RIGA_FP32
        R.set_eig_options(precision=mprec, extra=2, seed=11)
        for _ in range(max(1, args.warmup)):
            step()
        mt = []
        rs_m = None
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, rs_m, _ = step()
            e1.record(stream)
            e1.synchronize()
            mt.append(e0.elapsed_time(e1))
        okm = int(np.sum(rs_m <= RESID_TOL))
        mixed = {"value": world * okm / (statistics.mean(mt) / 1e3), "unit": "eigenpairs/s",
                 "ms_per_step": statistics.mean(mt), "converged_pairs": okm, "max_resid": float(np.nanmax(rs_m)),
                 "dtype": ("f32 fronts with tf32 tensor-core updates" if args.mixed_precision == "tf32" else "f32 fronts")
                          + ", f64 refinement/Lanczos/inertia"}
        R.set_eig_options(precision=riga.RIGA_FP64, extra=2, seed=11)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, dt, desc = oracle_sample_batch(cfg)
        cpu = {"value": v, "unit": "eigenpairs/s", "cores": 1, "kind": "oracle", "sample": desc}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "eigenpairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded meshes and coefficients)",
            "config": config_dict(args, cfg, {"N_total": q["N"], "nnz_total": q["nnz"], "nnzL_total": q["nnzL"],
                                              "flops_fact": q["flops_fact"]}),
            "converged_pairs": pairs, "max_resid": float(np.nanmax(rs)),
            "e2e": {"value": e2e_val, "unit": "eigenpairs/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches), "roofline": roof, "fronts": fronts, "phases_ms_one_step": phases,
            "mixed_path": mixed,
            "autotune": {"small_trail": tuned_trail, "factor_ms_per_candidate": dict(zip([0, 128, 256, 512, 1024, 4096], tuned_ms))},
            "assembly_ms": statistics.median(asm_ms),
            "counts_per_step": {"n_fact": st["n_fact"], "n_solve": st["n_solve"], "n_matvec": st["n_matvec"],
                                "lanczos_steps": st["lanczos_steps"]},
            "clocks": clocks, "wall_s_timed": t_wall, "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    R.close()
    if dist is not None:
        dist.destroy_process_group()


def run_riga(args, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_2009_08167_gb300 import riga

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    prec = {"fp64": riga.RIGA_FP64, "fp32": riga.RIGA_FP32, "tf32": riga.RIGA_TF32, "bf16": riga.RIGA_BF16}[args.precision]
    cfg = workload(args.mesh)
    if cfg.get("batch"):
        return run_riga_batch(args, rank, world, local_rank, cfg)
    mesh, k = cfg["mesh"], cfg["k"]
    R = riga.Riga(local_rank, stream)
    R.set_fp64_update(1 if args.fp64_update == "tc" else 0)
    R.set_eig_options(slice=cfg["slice"], precision=prec, extra=2, seed=11)
    R.set_eig_block(args.block)
    R.assemble(mesh)  # symbolic analysis: once per pattern, untimed
    q = R.query()
    N = q["N"]
    # front tile shapes by measurement (untimed setup), where the factorization
    # is cheap enough to run 24 times (2D; the 3D mesh keeps the default)
    tuned = None
    if q["flops_fact"] < 1e11:
        t, tms = R.autotune()
        tuned = {"small_trail": t, "factor_ms_per_candidate": dict(zip([0, 128, 256, 512, 1024, 4096], tms))}
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def step_device():
        return R.eigs(k, cfg["sigma"], RESID_TOL, vectors=True, device_out=True)

    # numeric assembly: reported apart from the timed eigensolution, as the
    # paper counts it
    asm_ms = []
    for _ in range(3):
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        R.assemble(mesh)
        a1.record(stream)
        a1.synchronize()
        asm_ms.append(a0.elapsed_time(a1))
    for _ in range(args.warmup):
        step_device()
    barrier()
    clk = Clocks(local_rank)
    launches0 = R.launches()
    times = []
    rs = None
    t_wall0 = time.perf_counter()
    torch.cuda.nvtx.range_push("timed")  # profilers can restrict themselves to the timed steps
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ev, U, rs = step_device()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.nvtx.range_pop()
    barrier()
    t_wall = time.perf_counter() - t_wall0
    clocks = clk.stop()
    launches = (R.launches() - launches0) // max(1, args.steps)
    rs_h = rs.cpu().numpy()
    pairs = int(np.sum(rs_h <= RESID_TOL))
    ms = statistics.mean(times)
    value, ms_max = aggregate(ms, pairs, world, dist, dev)
    st = R.stats()

    # end to end through the public API with host buffers: mesh description
    # in, eigenvalues, eigenvectors and residuals out (pageable host memory)
    h2d = int(sum(np.asarray(mm, dtype=np.int32).nbytes for mm in mesh.mults))
    d2h = 8 * (k + N * k + k)
    e2e_times = []
    for _ in range(0 if args.no_e2e else max(1, min(args.steps, 3))):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        R.assemble(mesh)
        evh, Uh, rsh = R.eigs(k, cfg["sigma"], RESID_TOL, vectors=True, device_out=False)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
    e2e_val = None
    if e2e_times:
        e2e_pairs = int(np.sum(rsh <= RESID_TOL))
        e2e_val = world * e2e_pairs / statistics.mean(e2e_times)

    # roofline: one profiled step (phase timing with CUDA events on the
    # library's stream), dominant phase by device time
    R.profile(True)
    if not args.no_profile_pass:
        step_device()
    prof = R.profile_get()
    R.profile(False)
    roof = roofline(prof, q)
    fronts = fronts_rate(prof, q["flops_fact"], R.stats()["n_fact"], *fp64_front_peak(args.fp64_update))
    phases = {p: {"ms": round(v["ms"], 3), "calls": v["calls"], "launches": v["launches"]} for p, v in prof.items() if v["calls"]}

    # the mixed path (FP32 fronts, FP64 refinement, residuals, Lanczos and
    # inertia) on the same workload, same timing rules
    mixed = None
    if args.precision == "fp64" and not args.no_mixed:
        mprec = riga.RIGA_TF32 if args.mixed_precision == "tf32" else riga.RIGA_FP32
        R.set_eig_options(slice=cfg["slice"], precision=mprec, extra=2, seed=11)
        for _ in range(max(1, args.warmup)):
            step_device()
        mt = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, _, rs_m = step_device()
            e1.record(stream)
            e1.synchronize()
            mt.append(e0.elapsed_time(e1))
        rs_mh = rs_m.cpu().numpy()
        stm = R.stats()
        R.profile(True)
        step_device()
        prof_m = R.profile_get()
        R.profile(False)
        fronts_m = fronts_rate(prof_m, q["flops_fact"], R.stats()["n_fact"],
                               TF32_PEAK_TFLOPS if args.mixed_precision == "tf32" else FP32_PEAK_TFLOPS)
        mixed = {"value": world * int(np.sum(rs_mh <= RESID_TOL)) / (statistics.mean(mt) / 1e3),
                 "unit": "eigenpairs/s", "ms_per_step": statistics.mean(mt), "converged_pairs": int(np.sum(rs_mh <= RESID_TOL)),
                 "max_resid": float(np.max(rs_mh)), "n_fact": stm["n_fact"], "lanczos_steps": stm["lanczos_steps"],
                 "dtype": ("f32 fronts with tf32 tensor-core updates" if args.mixed_precision == "tf32" else "f32 fronts")
                          + ", f64 refinement/Lanczos/inertia", "fronts": fronts_m,
                 "phases_ms_one_step": {p: round(v["ms"], 3) for p, v in prof_m.items() if v["calls"]}}
        R.set_eig_options(slice=cfg["slice"], precision=prec, extra=2, seed=11)

    c3 = None
    if args.c3_steps > 0 and args.mesh in ("riga", "iga") and args.precision == "fp64":
        c3 = run_c3_leg(args, local_rank, flush)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        os.environ.setdefault("OMP_NUM_THREADS", "1")
        v, dt, desc = oracle_sample(cfg)
        cpu = {"value": v, "unit": "eigenpairs/s", "cores": 1, "kind": "oracle", "sample": desc}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "eigenpairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32-fronts/f64",
            "data": "synthetic (deterministic mesh; seeded Lanczos start vectors)",
            "config": config_dict(args, cfg, {"N": N, "nnz": q["nnz"], "nnzL": q["nnzL"],
                                              "flops_fact": q["flops_fact"]}),
            "converged_pairs": pairs, "max_resid": float(np.max(rs_h)),
            "e2e": {"value": e2e_val, "unit": "eigenpairs/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches),
            "roofline": roof,
            "fronts": fronts,
            "autotune": tuned,
            "assembly_ms": statistics.median(asm_ms),
            "mixed_path": mixed,
            "c3": c3,
            "phases_ms_one_step": phases,
            "counts_per_step": {"n_fact": st["n_fact"], "n_solve": st["n_solve"], "n_matvec": st["n_matvec"],
                                "lanczos_steps": st["lanczos_steps"]},
            "clocks": clocks,
            "wall_s_timed": t_wall,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    R.close()
    if dist is not None:
        dist.destroy_process_group()


def run_c3_leg(args, local_rank, flush):
    """The 3D workload (64^3 elements, p=2, C0 planes every 8 elements,
    N = 357,911, 50 pairs, Lanczos blocks of 2) on its own context, three
    ways: FP64 fronts with the Schur updates as exact BF16 digit-slice
    products on the tensor cores ("fp64", the default update), FP64 fronts
    with FP64 FMA updates on the CUDA cores ("fp64_fma", the plain FP64
    path), and FP32 fronts with TF32 tensor-core updates plus FP64
    refinement, residuals, Lanczos and inertia ("mixed").  Each with one
    untimed warm-up step and args.c3_steps timed steps (CUDA events, L2
    flushed before each step), the same metric as the headline."""
    import numpy as np
    import torch
    from paper_2009_08167_gb300 import riga
    from paper_2009_08167_gb300.inputs import config_c3
    cfg = config_c3()
    stream = torch.cuda.current_stream()
    R = riga.Riga(local_rank, stream)
    R.set_fp64_update(1 if args.fp64_update == "tc" else 0)
    R.set_eig_block(2)
    t0 = time.perf_counter()
    R.assemble(cfg["mesh"])
    setup_s = time.perf_counter() - t0
    q = R.query()
    out = {"workload": "laplace3d_p2_64x64x64_riga_bs8_k50", "N": q["N"], "nnz": q["nnz"], "nnzL": q["nnzL"],
           "flops_fact": q["flops_fact"], "pairs": cfg["k"], "lanczos_block": 2, "setup_s": setup_s,
           "l2": "flushed between timed steps (512 MiB write)"}
    for name, prec, upd in (("fp64", riga.RIGA_FP64, 1), ("fp64_fma", riga.RIGA_FP64, 0), ("mixed", riga.RIGA_TF32, 1)):
        R.set_fp64_update(upd)
        R.set_eig_options(slice=cfg["k"], precision=prec, extra=2, seed=11)
        R.eigs(cfg["k"], 0.0, RESID_TOL, vectors=True, device_out=True)
        times, rs = [], None
        for _ in range(args.c3_steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, _, rs = R.eigs(cfg["k"], 0.0, RESID_TOL, vectors=True, device_out=True)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        rs_h = rs.cpu().numpy()
        ok = int(np.sum(rs_h <= RESID_TOL))
        st = R.stats()
        out[name] = {"value": ok / (statistics.mean(times) / 1e3), "unit": "eigenpairs/s",
                     "ms_per_step": statistics.mean(times), "steps": len(times), "converged_pairs": ok,
                     "max_resid": float(np.max(rs_h)), "n_fact": st["n_fact"], "lanczos_steps": st["lanczos_steps"],
                     "dtype": ("f64 fronts, updates as exact bf16 digit-slice products on the tensor cores"
                               if upd else "f64 fronts, f64 fma updates") if prec == riga.RIGA_FP64 else
                              "f32 fronts with tf32 tensor-core updates, f64 refinement/Lanczos/inertia"}
    R.set_fp64_update(1 if args.fp64_update == "tc" else 0)
    out["mixed_over_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    out["fp64_over_fp64_fma"] = out["fp64"]["value"] / out["fp64_fma"]["value"]
    out["mixed_over_fp64_fma"] = out["mixed"]["value"] / out["fp64_fma"]["value"]
    R.close()
    return out


def bs_sweep(dim, ne, p, pairs, steps=5, device=0, slice_=None):
    """Time per factorization, per f/b solve (one right-hand side) and per
    M mat-vec, and eigenpairs/s of a full eigensolve, against the rIGA
    blocksize (Sec. 7, Figs. 6 and 9: the paper sweeps bs = 2^0 .. n_e on one
    CPU core and finds 16 best; bs = n_e is IGA).  FP64 fronts, Lanczos
    blocks of 2, CUDA events on the library's stream, each call averaged
    over `steps`.  Returns one row per blocksize."""
    import numpy as np
    import torch
    from paper_2009_08167_gb300 import riga
    from paper_2009_08167_gb300.inputs import Mesh
    stream = torch.cuda.current_stream()
    rows = []
    bs_list = [1 << i for i in range(int(np.log2(ne)) + 1)]
    for bs in bs_list:
        mesh = Mesh(dim, ne, p, None if bs == ne else bs)
        R = riga.Riga(device, stream)
        R.set_eig_block(2)
        R.set_eig_options(slice=slice_ or pairs, precision=riga.RIGA_FP64, extra=2, seed=3)
        R.assemble(mesh)
        q = R.query()
        N = q["N"]

        def timed(fn, n):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(n):
                fn()
            e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1) / n

        R.factor(0.0, riga.RIGA_FP64)
        t_fact = timed(lambda: R.factor(0.0, riga.RIGA_FP64), steps)
        b = torch.randn(N, dtype=torch.float64, device="cuda")
        x = torch.empty_like(b)
        R.solve(b, out=x)
        t_fb = timed(lambda: R.solve(b, out=x), 4 * steps)
        t_mv = timed(lambda: R.spmv(0, b), 4 * steps)  # y = M x, global numbering (two permutations included)
        R.eigs(pairs, 0.0, RESID_TOL, vectors=False, device_out=True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ev, _, rs = R.eigs(pairs, 0.0, RESID_TOL, vectors=False, device_out=True)
        e1.record(stream)
        e1.synchronize()
        t_eigs = e0.elapsed_time(e1)
        ok = int((rs <= RESID_TOL).sum().item())
        rows.append({"bs": bs, "iga": bs == ne, "N": N, "nnz": q["nnz"], "nnzL": q["nnzL"],
                     "flops_fact": q["flops_fact"], "fact_ms": t_fact, "fb_ms": t_fb, "mv_ms": t_mv,
                     "eigs_ms": t_eigs, "pairs": ok, "pairs_per_s": ok / (t_eigs / 1e3),
                     "evals": ev.cpu().numpy().tolist()})
        R.close()
    return rows


def run_bs_sweep(args, local_rank):
    torch_dev = local_rank
    import torch
    torch.cuda.set_device(torch_dev)
    if args.sweep_dim == 3:
        dim, ne, p = 3, 32, 2
    else:
        dim, ne, p = 2, 256, 3
    rows = bs_sweep(dim, ne, p, args.sweep_pairs, steps=max(1, args.steps), device=local_rank)
    for r in rows:
        r.pop("evals")
    best = {key: min(rows, key=lambda r: r[key])["bs"] for key in ("fact_ms", "fb_ms", "mv_ms", "eigs_ms")}
    print(json.dumps({"mode": "bs-sweep", "dim": dim, "elements_per_side": ne, "degree": p,
                      "pairs": args.sweep_pairs, "rows": rows, "best_bs": best}), flush=True)


def run_interval(args, local_rank):
    """Every eigenpair in [0, hi) of the workload's mesh by dynamic spectrum
    slicing with thick-restart Lanczos (riga_eigs_interval), the paper's
    large-N0 setting (N0 = 4096 in 2D, 1024 in 3D).  hi comes from Weyl's
    law for the unit square / cube (N(lambda) ~ lambda / (4 pi) in 2D,
    lambda^{3/2} / (6 pi^2) in 3D) at 5 % above --interval-pairs; the exact
    count is the inertia difference.  One untimed warm-up, then --steps timed
    runs (CUDA events, L2 flushed)."""
    import math
    import numpy as np
    import torch
    from paper_2009_08167_gb300 import riga
    torch.cuda.set_device(local_rank)
    stream = torch.cuda.current_stream()
    prec = {"fp64": riga.RIGA_FP64, "fp32": riga.RIGA_FP32, "tf32": riga.RIGA_TF32, "bf16": riga.RIGA_BF16}[args.precision]
    cfg = workload(args.mesh)
    mesh = cfg["mesh"]
    target = 1.05 * args.interval_pairs
    hi = 4.0 * math.pi * target * 1.0137 if mesh.dim == 2 else (6.0 * math.pi ** 2 * target) ** (2.0 / 3.0) * 1.0137
    R = riga.Riga(local_rank, stream)
    R.set_fp64_update(1 if args.fp64_update == "tc" else 0)
    R.set_eig_options(slice=50, precision=prec, extra=2, seed=11)
    R.assemble(mesh)
    kmax = int(2 * args.interval_pairs + 64)
    ev, U, rs, basis = R.eigs_interval(0.0, hi, kmax, RESID_TOL)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    times = []
    for _ in range(max(1, args.steps)):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ev, U, rs, basis = R.eigs_interval(0.0, hi, kmax, RESID_TOL)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    st = R.stats()
    n = int(ev.size)
    ok = int(np.sum(rs <= RESID_TOL))
    print(json.dumps({"mode": "interval", "workload": config_dict(args, cfg)["workload"], "hi": hi, "count": n,
                      "converged_pairs": ok, "max_resid": float(np.max(rs)) if n else None,
                      "ms": statistics.mean(times), "pairs_per_s": ok / (statistics.mean(times) / 1e3),
                      "basis_cols": basis, "basis_bytes": 2 * 8 * basis * R.query()["N"],
                      "eigenvector_bytes": 8 * n * R.query()["N"], "n_fact": st["n_fact"],
                      "lanczos_steps": st["lanczos_steps"], "precision": args.precision}), flush=True)
    R.close()


def run_kernel_mode(args, local_rank):
    """Short program for profilers: the benchmark's mesh, one numeric
    assembly, then --steps factorizations (mode factor) or one factorization
    and --steps solves (mode solve) through the C ABI; prints one JSON line
    with device times."""
    import numpy as np
    import torch
    from paper_2009_08167_gb300 import riga
    torch.cuda.set_device(local_rank)
    stream = torch.cuda.current_stream()
    prec = {"fp64": riga.RIGA_FP64, "fp32": riga.RIGA_FP32, "tf32": riga.RIGA_TF32, "bf16": riga.RIGA_BF16}[args.precision]
    cfg = workload(args.mesh)
    R = riga.Riga(local_rank, stream)
    R.set_fp64_update(1 if args.fp64_update == "tc" else 0)
    if cfg.get("batch"):
        R.assemble_batch(cfg["meshes"], cfg["coefK"])
    else:
        R.assemble(cfg["mesh"])
    N = R.query()["N"]
    b = torch.randn(N, dtype=torch.float64, device="cuda")
    x = torch.empty_like(b)
    if args.mode == "trace":
        R.factor(0.0, prec)
        for _ in range(3):
            R.solve(b, out=x)
        tr, order = R.trace_solve(b.cpu().numpy())
        sym = R.get_symbolic()
        np.savez(args.trace_out, trace=tr, order=order, parent=sym["parent"],
                 node_ptr=sym["node_ptr"], front_ptr=sym["front_ptr"])
        t0 = tr[:, 1].min()
        print(json.dumps({"mode": "trace", "items": int(tr.shape[0]), "span_us": float((tr[:, 3].max() - t0) / 1e3)}))
        R.close()
        return
    R.profile(True)
    R.factor(0.0, prec)
    for _ in range(args.steps):
        if args.mode == "factor":
            R.factor(0.0, prec)
        else:
            R.solve(b, out=x)
    prof = R.profile_get()
    R.profile(False)
    q = R.query()
    print(json.dumps({"mode": args.mode, "steps": args.steps, "N": N, "nnzL": q["nnzL"], "flops_fact": q["flops_fact"],
                      "phases": prof}), flush=True)
    R.close()


def main():
    args = parse()
    if args.mode == "bs-sweep":
        run_bs_sweep(args, int(os.environ.get("LOCAL_RANK", "0")))
        return
    if args.mode == "interval":
        run_interval(args, int(os.environ.get("LOCAL_RANK", "0")))
        return
    if args.mode != "eigs":
        run_kernel_mode(args, int(os.environ.get("LOCAL_RANK", "0")))
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_riga(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
