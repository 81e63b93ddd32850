#!/usr/bin/env python
"""Benchmark of the GB300 H(curl) AMG: time to a 1e-8 relative residual (setup + PCG solve) on a
synthetic coefficient-jump workload, the achieved HBM bandwidth of the dominant V-cycle kernel,
and the CPU oracle beside it.  Prints one JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference] [--precision f64|f32|bf16]

A step is one pass of the whole path on one system: amgh_setup (graph steps, local harmonic-
extension solves, Galerkin products, smoother blocks) and amgh_pcg_solve to ||r|| <= 1e-8 ||r0||,
with A, G and f already in device memory.  Under torchrun every rank solves its own copy
(replicas: the path has no data exchange between independent systems).
"""
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

METRIC = "time to 1e-8 rel residual; V-cycle HBM GB/s vs 8 TB/s; FP64 vs mixed/learned"
WORKLOAD = "hex64_checker"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="f64", choices=["f64", "f32", "bf16"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--dense-tail", type=int, default=None,
                    help="rows at or below which the V-cycle tail is one dense operator (library default if unset)")
    ap.add_argument("--fuse-restrict", type=int, default=None, choices=[-1, 0, 1],
                    help="fused residual + restriction: -1 tuned per level, 0 off, 1 on (library default if unset)")
    ap.add_argument("--interp", default="local", choices=["local", "constrained"],
                    help="interior extension: the paper's local harmonic extension, or the same corrected to "
                         "commute with a nodal interpolation")
    ap.add_argument("--variants", default="hex128_spheres",
                    help="workload of the FP64 / FP32 / BF16 comparison reported in the line ('none' to skip)")
    ap.add_argument("--variant-steps", type=int, default=1)
    ap.add_argument("--learned-meshes", type=int, default=40,
                    help="training meshes of the learned-interpolation comparison reported in the line (0 to skip)")
    ap.add_argument("--profile-setup", action="store_true",
                    help="set up once, then once more between cudaProfilerStart/Stop and exit (for ncu "
                         "--profile-from-start off); prints no bench line")
    ap.add_argument("--profile-mlp-epoch", action="store_true",
                    help="learned interpolation: build the samples of 20 seeded 24^3 meshes, train one epoch, "
                         "then one more between cudaProfilerStart/Stop and exit; prints the epoch time")
    ap.add_argument("--profile-vcycles", type=int, default=0,
                    help="set up once, then run this many V-cycles between cudaProfilerStart/Stop and exit "
                         "(for ncu --profile-from-start off); prints no bench line")
    ap.add_argument("--profile-level", type=int, default=-1,
                    help="set up once, then run one pre-smoothing step of this level between "
                         "cudaProfilerStart/Stop and exit (for ncu --profile-from-start off); prints no bench line")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# GB300 dense FP64 rate (nominal), used only when the live measurement below fails
FP64_NOMINAL_TFLOPS = 1.25


def fp64_peak_tflops(dev):
    """FP64 rate measured live: the best of five cuBLAS FP64 GEMMs (4096^3, 2 n^3 flops), the same
    kind of library figure as the measured bf16 peak; the nominal rate if it cannot run."""
    import torch
    try:
        n = 4096
        a = torch.rand(n, n, dtype=torch.float64, device=dev)
        b = torch.rand(n, n, dtype=torch.float64, device=dev)
        torch.matmul(a, b)
        best = 1e30
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1000.0)
        del a, b
        return 2.0 * n ** 3 / best / 1e12, "measured (cuBLAS FP64 GEMM 4096^3, best of 5)"
    except Exception as e:   # noqa: BLE001
        return FP64_NOMINAL_TFLOPS, "nominal (%s)" % type(e).__name__


def level_profile(amgh, h, A0, G0, hbm_peak, fp64_peak, nvc=10):
    """Per level of a built hierarchy: the Schwarz sweep's time (CUDA events on the handle's
    stream around each of its launches over `nvc` V-cycles), its colour steps, algorithmic bytes
    and FP64 work (counted like the library counts bytes), and the fraction of the HBM and FP64
    peaks; a sweep far below both is bound by the latency of its sequential colour steps."""
    import numpy as np
    import torch
    info = amgh.amgh_info(h)
    n0 = info["n"][0]
    r = torch.tensor(np.linspace(-1.0, 1.0, n0), device="cuda")
    z = torch.zeros_like(r)
    last = info["dense_tail"] if info["dense_tail"] >= 0 else info["levels"] - 1
    out, total = [], 0.0
    for l in range(last):
        amgh.amgh_profile(h, 1, "schwarz", l)
        for _ in range(nvc):
            amgh.amgh_vcycle(h, r, z)
        ks = amgh.amgh_kernel_stats(h)
        amgh.amgh_profile(h, 0, "schwarz", l)
        A = A0 if l == 0 else amgh.amgh_level_matrix(h, l, 0)
        G = G0 if l == 0 else amgh.amgh_level_matrix(h, l, 2)
        colour = amgh.amgh_level_structure(h, l)["colour"]
        vb = 8 if info["precision"][l] == 0 else (4 if info["precision"][l] == 1 else 2)
        tb = 8 if info["precision"][l] == 0 else 4
        by, fl = finest_sweep_work(A, G, colour, vb, tb)
        sweeps = 2 * nvc
        ms = ks["total_ms"] / sweeps if sweeps else 0.0
        steps = 2 * info["ncolours"][l] - 1
        gbs = by / (ms / 1000.0) / 1e9 if ms > 0 else 0.0
        tfl = fl / (ms / 1000.0) / 1e12 if ms > 0 else 0.0
        fh, ff = gbs / hbm_peak, tfl / fp64_peak if info["precision"][l] == 0 else None
        bound = "hbm" if fh >= 0.3 else ("alu" if ff is not None and ff >= 0.3 else "latency")
        total += ms
        out.append({"level": l, "rows": info["n"][l], "nnz": info["nnz"][l], "mode": info["fused"][l],
                    "lanes": info["lanes"][l], "steps_per_sweep": steps, "ms_per_sweep": ms,
                    "us_per_step": 1000.0 * ms / steps, "bytes_per_sweep": by, "GBps": gbs, "hbm_frac": fh,
                    "fp64_TFLOPs": tfl if info["precision"][l] == 0 else None, "fp64_frac": ff,
                    "bound": bound, "launches": ks["launches"]})
    for o in out:
        o["share_of_sweeps"] = o["ms_per_sweep"] / total if total > 0 else None
    return out


def time_variant(amgh, prob, dev_inputs, precision, steps, warmup, **kw):
    """Setup + (flexible) CG to 1e-8 on a workload with a requested storage precision (and other
    setup parameters): wall time of whole steps (synchronised) after warm-up ones, with the level
    storages the handle chose."""
    import numpy as np
    import torch
    A, f = prob["A"], prob["f"]
    Ad, Gd, fd = dev_inputs
    xd = torch.zeros_like(fd)
    code = {"f64": amgh.AMGH_F64, "f32": amgh.AMGH_F32, "bf16": amgh.AMGH_BF16}[precision]
    res = []
    for i in range(warmup + steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = amgh.amgh_setup(Ad, Gd, precision=code, **kw)
        t1 = time.perf_counter()
        xd.zero_()
        it, rel, ok = amgh.amgh_pcg_solve(h, fd, xd, 1e-8, 5000)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        info = amgh.amgh_info(h)
        amgh.amgh_destroy(h)
        if i >= warmup:
            res.append((t2 - t0, t1 - t0, t2 - t1, it, rel, ok, info))
    xs = xd.cpu().numpy()
    true_rel = float(np.linalg.norm(f - A @ xs) / np.linalg.norm(f))
    names = {0: "f64", 1: "f32", 2: "bf16"}
    info = res[-1][6]
    return {"workload": prob["name"], "precision": precision,
            "s_per_step": statistics.mean(r[0] for r in res), "setup_s": statistics.mean(r[1] for r in res),
            "solve_s": statistics.mean(r[2] for r in res), "pcg_iters": res[-1][3], "relres": res[-1][4],
            "converged": res[-1][5], "true_relres": true_rel,
            "level_precision": [names[q] for q in info["precision"]],
            "block_kappa": info["block_kappa"], "levels": info["n"], "op_complexity": round(info["op_complexity"], 4),
            "interp_used": info["interp_used"], "rho": info["rho"], "rho_exact": info["rho_exact"],
            "steps": steps, "warmup": warmup}


def learned_comparison(amgh, prob, dev_inputs, meshes, epochs=8):
    """The learned interpolation on this workload: a network trained on the exact local solves of
    `meshes` seeded 24^3 meshes with alpha = 10^U(-4,4) per element (FP32 and BF16 storage), its
    setup with the convergence-factor test (the exact factor measured once, then passed as the
    stored reference), against the exact local solves; whole steps (setup + CG to 1e-8)."""
    import workloads as W
    from workloads import fields
    t0 = time.perf_counter()
    nets = {"fp32": amgh.amgh_mlp_create(0), "bf16": amgh.amgh_mlp_create(0)}
    amgh.amgh_mlp_set_precision(nets["bf16"], amgh.AMGH_BF16)
    old = os.environ.get("AMGH_TUNE")
    os.environ["AMGH_TUNE"] = "0"   # the samples need the finest P only
    try:
        for s in range(meshes):
            pt = W.hex_problem(24, fields.log_uniform(24, 700 + s), 1.0)
            h = amgh.amgh_setup(pt["A"], pt["G"])
            for m in nets.values():
                amgh.amgh_mlp_add_samples(m, h)
            amgh.amgh_destroy(h)
    finally:
        if old is None:
            del os.environ["AMGH_TUNE"]
        else:
            os.environ["AMGH_TUNE"] = old
    t_data = time.perf_counter() - t0
    out = {"train": {"meshes": meshes, "mesh": "24^3, alpha = 10^U(-4,4) per element, beta = 1",
                     "samples": amgh.amgh_mlp_num_samples(nets["fp32"]), "data_s": t_data, "epochs": epochs}}
    for label, m in nets.items():
        t0 = time.perf_counter()
        losses = [amgh.amgh_mlp_train(m, 1, 512, 1e-3, 20000 + e) for e in range(epochs)]
        out["train"][label] = {"train_s": time.perf_counter() - t0, "loss_first": losses[0], "loss_last": losses[-1]}
    Ad, Gd, fd = dev_inputs
    h = amgh.amgh_setup(Ad, Gd, interp=amgh.AMGH_INTERP_LEARNED, mlp=nets["fp32"])
    rho_ref = amgh.amgh_info(h)["rho_exact"]
    amgh.amgh_destroy(h)
    keys = ("s_per_step", "setup_s", "solve_s", "pcg_iters", "converged", "levels", "interp_used", "rho", "rho_exact")
    ex = time_variant(amgh, prob, dev_inputs, "f64", 2, 1)
    out["exact"] = {k: ex[k] for k in keys if k not in ("interp_used", "rho", "rho_exact")}
    out["rho_exact"] = rho_ref
    for label, m in nets.items():
        v = time_variant(amgh, prob, dev_inputs, "f64", 2, 1, interp=amgh.AMGH_INTERP_LEARNED, mlp=m, rho_ref=rho_ref)
        v = {k: v[k] for k in keys}
        v["kept"] = v.pop("interp_used") == amgh.AMGH_INTERP_LEARNED
        out[label] = v
    return out


def last_colour(res):
    return res[-1].get("colour0") if res else None


def launches_per_sweep(res):
    """launches of one finest-level sweep: one per colour step in the per-colour modes, else one"""
    info = res[-1]["info"]
    return 2 * info["ncolours"][0] - 1 if info["fused"][0] in (0, 4, 6) else 1


def finest_sweep_work(A, G, colour, vbytes, tbytes):
    """(bytes, flops) of one symmetric colour sweep of the finest level, counted per colour step as
    the library counts its algorithmic bytes: each row of each star of the colour moves its entries
    (value + column), its star's block-inverse row and three vector values (vbytes: stored value,
    tbytes: vector value), and does two flops per entry and per inverse entry and two additions."""
    import numpy as np
    Gc = G.tocsc()
    b = np.diff(Gc.indptr)
    rowlen = np.diff(A.indptr)
    star_of = np.repeat(np.arange(Gc.shape[1]), b)
    nz = np.bincount(star_of, weights=rowlen[Gc.indices], minlength=Gc.shape[1])
    C = int(colour.max()) + 1
    cn = np.bincount(colour, weights=nz, minlength=C)
    ci = np.bincount(colour, weights=b.astype(np.float64) ** 2, minlength=C)
    cr = np.bincount(colour, weights=b.astype(np.float64), minlength=C)
    seq = list(range(C)) + list(range(C - 2, -1, -1))
    by = sum(cn[c] * (vbytes + 4) + ci[c] * vbytes + 3 * tbytes * cr[c] for c in seq)
    fl = sum(2 * cn[c] + 2 * ci[c] + 2 * cr[c] for c in seq)
    return float(by), float(fl)


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


def traffic_for(kernel, workload, mode):
    """dram bytes per launch from the committed ncu summary, if the kernel source and its launch
    mode are the ones that were captured."""
    import hashlib
    src = open(os.path.join(ROOT, "paper_2602_23613_gb300", "csrc", "schwarz_chunk.cuh"), "rb").read()
    sha = hashlib.sha256(src).hexdigest()[:16]
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        kv = dict(x.split("=", 1) for x in line.split() if "=" in x)
        if (kv.get("kernel") == kernel and kv.get("workload") == workload and kv.get("sha") == sha
                and kv.get("mode") == mode):
            return float(kv["dram_bytes_per_launch"])
    return None


# ----------------------------------------------------------------------------------------------
# CPU oracle leg (cpu_baseline and --impl reference)
# ----------------------------------------------------------------------------------------------
def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), with the architecture."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return "%s (%s)" % (line.split(":", 1)[1].strip(), platform.machine())
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return "%s (%s)" % (line.split(":", 1)[1].strip(), platform.machine())
    except OSError:
        pass
    return platform.machine()


def scaling_exponents():
    """Growth exponents of the oracle's setup time and per-iteration PCG time with the DoFs,
    from its measured 24^3 and 64^3 runs (tests/golden/oracle_scaling.json); 1 when absent."""
    try:
        rows = {r["n"]: r for r in json.load(open(os.path.join(ROOT, "tests", "golden", "oracle_scaling.json")))["rows"]}
        import math
        a, b = rows[24], rows[64]
        lr = math.log(b["ndof"] / a["ndof"])
        return (math.log(b["setup_s"] / a["setup_s"]) / lr,
                math.log((b["pcg_s"] / b["iters"]) / (a["pcg_s"] / a["iters"])) / lr, "measured 24^3 -> 64^3")
    except (OSError, ValueError, KeyError, ZeroDivisionError):
        return 1.0, 1.0, "linear (no measured exponents)"


def full_iterations(workload):
    """The oracle's own PCG iteration count on the full workload (stored by the oracle-only golden
    script), or None."""
    try:
        return json.load(open(os.path.join(ROOT, "tests", "golden", workload + ".json")))["pcg"]["iterations"]
    except (OSError, ValueError, KeyError):
        return None


def oracle_sample(workload=WORKLOAD, sample=None, pool=None, cores=1):
    """The oracle (setup, then PCG to 1e-8) on a smaller member of the workload family, extrapolated
    to the full workload by one rule that both CPU legs use: setup time x (N/n)^a plus time per
    PCG iteration x (N/n)^b x the full workload's iteration count, with a and b the oracle's measured
    growth exponents and the iteration count the oracle's own at full size (the sample's when that
    is unknown).  pool: a process pool whose map spreads the setup's independent local solves and
    star inverses (the PCG stays on one core)."""
    import workloads as W
    from oracle import amg as O
    sample = sample or W.describe(workload)[1]
    s = W.make_config(sample)
    nfull = W.CONFIGS[workload]["n"]
    full_n = 3 * nfull * (nfull - 1) ** 2
    kw = {} if pool is None else {"pmap": pool.map, "nchunks": 8 * cores}
    t0 = time.perf_counter()
    H = O.setup(s["A"], s["G"], coarse_size=100, **kw)
    t1 = time.perf_counter()
    _, it, _ = O.pcg(H, s["f"], tol=1e-8, maxit=1000)
    t2 = time.perf_counter()
    a, b, src = scaling_exponents()
    r = full_n / s["ndof"]
    it_full = full_iterations(workload) or it
    value = (t1 - t0) * r ** a + (t2 - t1) / max(it, 1) * r ** b * it_full
    return {"value": value, "unit": "s", "cores": cores, "kind": "oracle",
            "sample": "%s (%d DoFs): oracle setup %.2f s%s + PCG %.2f s in %d iterations; extrapolated to %d DoFs "
                      "as setup x (N/n)^%.2f + s/iteration x (N/n)^%.2f x %d iterations (%s exponents; the "
                      "oracle's own full-size iteration count)" % (
                          sample, s["ndof"], t1 - t0, " on %d processes" % cores if pool else "", t2 - t1, it,
                          full_n, a, b, it_full, src),
            "sample_seconds": t2 - t0, "sample_iters": it, "cpu": cpu_model(), "nproc": os.cpu_count()}


def oracle_all_cores(workload=WORKLOAD):
    """The same sample with the setup's independent loops over a pool of all host cores (spawned
    processes: the GPU context of this process must not be forked)."""
    import multiprocessing as mp
    n = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(n) as pool:
        pool.map(abs, range(n))                    # workers started before the timed region
        return oracle_sample(workload=workload, pool=pool, cores=n)


def max_over_ranks(value, device):
    """The largest of every rank's value (the job's time is its slowest replica's); the value
    itself without a process group or with one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import workloads as W
    for _ in range(args.warmup):
        oracle_sample(workload=args.workload, sample="hex8_unit")   # loads the modules only
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(oracle_sample(workload=args.workload))
    wall = time.perf_counter() - t0
    v = statistics.mean(x["value"] for x in vals)
    cb = dict(vals[-1])
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * wall / args.steps,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "desc": W.describe(args.workload)[0],
                                            "sample": W.describe(args.workload)[1]},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------------------------
def run_gpu(args, rank, world, local_rank):
    import numpy as np
    import torch

    import workloads as W
    from paper_2602_23613_gb300 import build, amgh

    torch.cuda.set_device(local_rank)
    build.build()
    amgh.load()
    prec = {"f64": amgh.AMGH_F64, "f32": amgh.AMGH_F32, "bf16": amgh.AMGH_BF16}[args.precision]
    prob = W.make_config(args.workload)
    A, G, f = prob["A"], prob["G"], prob["f"]
    n = prob["ndof"]
    dev = torch.device("cuda", local_rank)

    def dcsr(M):
        return (torch.tensor(M.indptr.astype(np.int32), device=dev), torch.tensor(M.indices.astype(np.int32), device=dev),
                torch.tensor(M.data.astype(np.float64), device=dev), M.shape)

    Ad, Gd = dcsr(A), dcsr(G)
    fd = torch.tensor(f, device=dev)
    xd = torch.zeros(n, dtype=torch.float64, device=dev)
    extra = {} if args.dense_tail is None else {"dense_tail": args.dense_tail}
    if args.fuse_restrict is not None:
        extra["fuse_restrict"] = args.fuse_restrict
    if args.interp == "constrained":
        extra["interp"] = amgh.AMGH_INTERP_CONSTRAINED

    if args.profile_mlp_epoch:
        from workloads import fields
        m = amgh.amgh_mlp_create(0)
        old = os.environ.get("AMGH_TUNE")
        os.environ["AMGH_TUNE"] = "0"   # the samples need the finest P only
        for sd in range(20):
            pt = W.hex_problem(24, fields.log_uniform(24, 500 + sd), 1.0)
            ht = amgh.amgh_setup(pt["A"], pt["G"])
            amgh.amgh_mlp_add_samples(m, ht)
            amgh.amgh_destroy(ht)
        if old is None:
            del os.environ["AMGH_TUNE"]
        else:
            os.environ["AMGH_TUNE"] = old
        amgh.amgh_mlp_train(m, 1, 512, 1e-3, 1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        amgh.amgh_mlp_train(m, 2, 512, 1e-3, 2)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / 2
        torch.cuda.profiler.start()
        amgh.amgh_mlp_train(m, 1, 512, 1e-3, 3)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print("profiled one training epoch of %d samples (batch 512); epoch %.1f ms without the profiler"
              % (amgh.amgh_mlp_num_samples(m), 1000 * dt), flush=True)
        return 0

    if args.profile_setup:
        h = amgh.amgh_setup(Ad, Gd, precision=prec, **extra)
        amgh.amgh_destroy(h)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        h = amgh.amgh_setup(Ad, Gd, precision=prec, **extra)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print("profiled one setup of %s (%d DoFs)" % (args.workload, n), flush=True)
        return 0

    if args.profile_vcycles > 0:
        h = amgh.amgh_setup(Ad, Gd, precision=prec, **extra)
        amgh.amgh_vcycle(h, fd, xd)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        for _ in range(args.profile_vcycles):
            amgh.amgh_vcycle(h, fd, xd)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print("profiled %d V-cycles of %s (%d DoFs)" % (args.profile_vcycles, args.workload, n), flush=True)
        return 0

    if args.profile_level >= 0:
        h = amgh.amgh_setup(Ad, Gd, precision=prec, **extra)
        info = amgh.amgh_info(h)
        lv = args.profile_level
        if lv >= info["levels"] - 1:
            raise SystemExit("level %d has no smoother (%d levels)" % (lv, info["levels"]))
        nl = info["n"][lv]
        fl = torch.tensor(W.uniform("probe", 1, nl), device=dev)
        xl = torch.tensor(W.uniform("probe", 2, nl), device=dev)
        yl = torch.zeros_like(fl)
        amgh.amgh_level_apply(h, lv, 2, fl, xl, yl)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        amgh.amgh_level_apply(h, lv, 2, fl, xl, yl)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print("profiled one pre-smoothing step of level %d of %s (%d rows, %d nonzeros, launch mode %d, %d lanes)"
              % (lv, args.workload, nl, info["nnz"][lv], info["fused"][lv], info["lanes"][lv]), flush=True)
        return 0

    def step(profile):
        h = amgh.amgh_setup(Ad, Gd, precision=prec, **extra)
        if profile:
            amgh.amgh_profile(h, 1, "schwarz", 0)
        xd.zero_()
        t0 = time.perf_counter()
        it, rel, ok = amgh.amgh_pcg_solve(h, fd, xd, 1e-8, 2000)
        solve_s = time.perf_counter() - t0
        info = amgh.amgh_info(h)
        ks = amgh.amgh_kernel_stats(h) if profile else None
        colour0 = amgh.amgh_level_structure(h, 0)["colour"] if profile else None
        amgh.amgh_destroy(h)
        return dict(iters=it, relres=rel, ok=ok, solve_s=solve_s, info=info, ks=ks, colour0=colour0)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step(False)
    barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    lib = amgh.load()
    l0 = lib.amgh_launch_count(None)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    t0 = time.perf_counter()
    # the production path (device-resident PCG) on every timed step; the last one also records
    # CUDA events around the finest Schwarz colour steps (host-driven PCG, a little slower)
    res = [step(i == args.steps - 1) for i in range(args.steps)]
    ev1.record()
    barrier()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    gpu_launches = lib.amgh_launch_count(None) - l0
    dev_ms = ev0.elapsed_time(ev1)
    t_step = max(dev_ms / 1000.0, wall) / args.steps
    t_step = max_over_ranks(t_step, dev)
    ks_launch = sum(r["ks"]["launches"] for r in res if r["ks"])
    ks_ms = sum(r["ks"]["total_ms"] for r in res if r["ks"])
    ks_bytes = sum(r["ks"]["algorithmic_bytes"] for r in res if r["ks"])
    achieved = ks_bytes / (ks_ms / 1000.0) / 1e9 if ks_ms > 0 else None
    pk = peaks()
    peak = pk["hbm_gbs"] if pk else 6800.0
    # the same launches' FP64 work: counted like the library counts their bytes (per colour step:
    # every row of every star of the colour with its entries, its star's block-inverse row and two
    # additions), summed over one sweep (colours 0..C-1, C-2..0)
    fp64_peak, fp64_src = fp64_peak_tflops(dev)
    fp64 = None
    if achieved and last_colour(res) is not None and res[-1]["info"]["precision"][0] == amgh.AMGH_F64:
        sw_bytes, sw_flops = finest_sweep_work(A, G, last_colour(res), 8, 8)
        fl_rate = achieved * 1e9 * (sw_flops / sw_bytes) / 1e12
        fp64 = {"achieved": fl_rate, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": fl_rate / fp64_peak, "peak_source": fp64_src,
                "flops_per_byte": sw_flops / sw_bytes,
                "sweep_bytes_vs_library": sw_bytes / (ks_bytes / ks_launch * launches_per_sweep(res)) if ks_launch else None}
    modes = {0: "colour", 1: "fused", 2: "persistent", 3: "staged", 4: "stream"}
    traffic = traffic_for("schwarz", args.workload, modes.get(res[-1]["info"]["fused"][0]))
    last = res[-1]

    # end to end through the same API with host buffers in page-locked memory (copies inside the
    # timed region)
    def pinned(a):
        return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()

    def pinned_csr(M):
        return (pinned(M.indptr.astype(np.int32)), pinned(M.indices.astype(np.int32)),
                pinned(M.data.astype(np.float64)), M.shape)

    Ah, Gh = pinned_csr(A), pinned_csr(G)
    fh = pinned(np.asarray(f, dtype=np.float64))
    xh = torch.zeros(n, dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        h = amgh.amgh_setup(Ah, Gh, precision=prec, **extra)
        xh.zero_()
        amgh.amgh_pcg_solve(h, fh, xh, 1e-8, 2000)
        amgh.amgh_destroy(h)
    barrier()
    e2e = (time.perf_counter() - t0) / e2e_steps
    csr_bytes = lambda M: 4 * (M.shape[0] + 1) + 12 * M.nnz
    h2d = csr_bytes(A) + csr_bytes(G) + 8 * n + 8 * n
    d2h = 8 * n

    # per-level sweep profile on one more hierarchy (outside the timed region)
    hl = amgh.amgh_setup(Ad, Gd, precision=prec, **extra)
    levels = level_profile(amgh, hl, A, G, peak, fp64_peak)
    amgh.amgh_destroy(hl)
    # the paper's three interpolations on this workload (Sec. 5's comparison): the algebraic one
    # timed above ("Alg"), the refinement-based one ("Ref") and geometric Nedelec ("Geo")
    # and the local extension corrected to commute (P G_c = 2 G P_n), with either coarse variables
    comparison = None
    if world == 1 and W.CONFIGS[args.workload]["n"] % 4 == 0:
        mesh_n = W.CONFIGS[args.workload]["n"]
        din = (Ad, Gd, fd)
        comparison = {}
        ref = dict(coarsening=amgh.AMGH_COARSEN_REFINEMENT, mesh_n=mesh_n)
        for label, kw in (("Ref", ref), ("Geo", dict(ref, interp=amgh.AMGH_INTERP_GEOMETRIC)),
                          ("Alg+C", dict(interp=amgh.AMGH_INTERP_CONSTRAINED)),
                          ("Ref+C", dict(ref, interp=amgh.AMGH_INTERP_CONSTRAINED))):
            v = time_variant(amgh, prob, din, args.precision, 3, 1, **kw)
            comparison[label] = {k: v[k] for k in ("s_per_step", "setup_s", "solve_s", "pcg_iters", "relres",
                                                   "converged", "levels", "op_complexity")}
        comparison["Alg"] = {"s_per_step": t_step, "pcg_iters": last["iters"], "levels": last["info"]["n"],
                             "op_complexity": round(last["info"]["op_complexity"], 4)}
    variants = None
    if args.variants != "none" and world == 1:
        vp = W.make_config(args.variants)
        vin = (dcsr(vp["A"]), dcsr(vp["G"]), torch.tensor(vp["f"], device=dev))
        variants = [time_variant(amgh, vp, vin, pr, args.variant_steps, 1) for pr in ("f64", "f32", "bf16")]
        del vin, vp
        base = variants[0]["s_per_step"]
        for v in variants:
            v["speedup_vs_f64"] = base / v["s_per_step"]

    learned = None
    if args.learned_meshes > 0 and world == 1:
        learned = learned_comparison(amgh, prob, (Ad, Gd, fd), args.learned_meshes)

    if rank != 0:
        return 0
    cpu = oracle_sample(workload=args.workload)
    cpu_all = oracle_all_cores(workload=args.workload)
    info = last["info"]
    line = {
        "metric": METRIC, "value": t_step, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * t_step, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {"workload": args.workload, "desc": W.describe(args.workload)[0], "n_dofs": n, "nnz": int(A.nnz),
                   "precision": args.precision, "tol": 1e-8, "interp": args.interp,
                   "l2": "inputs larger than L2 (A alone %.0f MB > 129 MB)" % (12 * A.nnz / 1e6),
                   "levels": info["n"], "op_complexity": round(info["op_complexity"], 4),
                   "level_precision": [{0: "f64", 1: "f32", 2: "bf16"}[q] for q in info["precision"]],
                   "fused_restrict": info["fused_rr"],
                   "smoother_lanes": info["lanes"], "smoother_fused": info["fused"],
                   "dense_tail_level": info["dense_tail"]},
        "pcg_iters": last["iters"], "relres": last["relres"], "converged": last["ok"],
        "solve_ms": 1000 * statistics.mean(r["solve_s"] for r in res),
        "setup_host_ms": info["setup_host_ms"], "setup_device_ms": info["setup_device_ms"],
        "vcycles_per_s": last["iters"] / statistics.mean(r["solve_s"] for r in res),
        "roofline": {"bound": "hbm", "kernel": "schwarz colour sweep, finest level", "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": (achieved / peak) if achieved else None,
                     "peak_source": "measured" if pk else "fallback",
                     "traffic": traffic, "launches": ks_launch,
                     "algorithmic_bytes_per_launch": ks_bytes / ks_launch if ks_launch else None,
                     "ms_per_launch": ks_ms / ks_launch if ks_launch else None,
                     "timed_on": "CUDA events on the handle's stream, last timed step",
                     "fp64": fp64},
        "cpu_baseline": {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample", "cpu", "nproc")},
        "cpu_baseline_all_cores": {k: cpu_all[k] for k in ("value", "unit", "cores", "kind", "sample", "cpu", "nproc")},
        "e2e": {"value": e2e, "unit": "s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(gpu_launches), "clocks": clk,
    }
    line["roofline"]["levels"] = levels
    if comparison is not None:
        line["comparison"] = comparison
    if variants is not None:
        line["variants"] = variants
    if learned is not None:
        line["learned"] = learned
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "reference":
            dist.init_process_group("gloo")
        else:
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl")
    try:
        if args.impl == "reference":
            return run_reference(args, rank, world)
        return run_gpu(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
