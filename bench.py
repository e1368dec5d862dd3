"""Benchmark of the FFM hot path on one or more GB300s (one process per GPU).

A step is one whole FFM product through the C ABI, ffm_plan + ffm_apply + ffm_destroy
(bounding cubes, Morton sort, box tables, descent, per-level operators, far field of every
level, near field, accumulation), on inputs already resident in HBM.  The default workload
is the Laplace kernel on 1e8 + 1e8 independent float32 points drawn from a mixture of 8
Gaussians (sigma 0.05, centres uniform in the unit cube), u ~ U(-1, 1) float32, w = 1/N,
eps = 1e-3 (laplace_clustered_1e8).

Prints one JSON line (rank 0).  `value` is FFM products per second over all ranks;
`e2e` is the same metric through the same API with host buffers (copies included);
`roofline` is the dominant kernel against its pipe's peak; `cpu_baseline` is the FP64 CPU
oracle (direct sum) timed on this host on a bounded sample of targets, which also gives
the rel-L2 error of the GPU result on those targets.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ffm|reference]
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SM_COUNT = 152
MUFU_PER_SM_CLK = 16          # special-function unit results per SM per clock
FP32_PER_SM_CLK = 128         # FP32 FMA lanes per SM per clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ffm", choices=["ffm", "reference"])
    ap.add_argument("--workload", default="laplace_clustered",
                    choices=["helmholtz_sphere_1M", "laplace_sphere_20k", "helmholtz_cube_200k_64rhs",
                             "laplace_clustered", "laplace_double_layer_sphere_1M", "laplace_gradient_sphere_1M"])
    ap.add_argument("--n", type=int, default=0, help="points per set (0: the workload's own size)")
    ap.add_argument("--serving", action="store_true",
                    help="serving stream: Poisson arrivals of mixed requests, p50/p99 latency and throughput")
    ap.add_argument("--requests", type=int, default=500)
    ap.add_argument("--scenes", type=int, default=0,
                    help="serving: requests share this many scenes (point sets, kernel, k, eps); 0: all distinct")
    ap.add_argument("--err-requests", type=int, default=12, help="serving: requests whose error is measured")
    ap.add_argument("--err-targets", type=int, default=256, help="serving: sampled targets per measured request")
    ap.add_argument("--bem", type=int, default=0, metavar="LEVEL",
                    help="boundary-element solve on an icosphere of this refinement level (GMRES over FFM products)")
    ap.add_argument("--workers", type=int, default=4)
    ap.add_argument("--cpu-targets", type=int, default=0,
                    help="targets of the FP64 direct-sum check (0: as many as fill --cpu-seconds, 256..4096)")
    ap.add_argument("--cpu-seconds", type=float, default=45.0,
                    help="time budget of the all-core direct-sum leg when --cpu-targets is 0")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--pw-transform", default="auto", choices=["auto", "direct", "nufft", "tc"],
                    help="plane-wave F steps: chosen per level, direct sums on the CUDA cores, the NUFFT "
                         "where possible, or direct sums with tensor-core products for several RHS")
    ap.add_argument("--eps", type=float, default=0.0, help="accuracy eps (0: the workload's own)")
    ap.add_argument("--aca", type=float, default=0.0, metavar="EPS_T",
                    help="Laplace workloads: transfer matrices as ACA factors to this tolerance (eq. 11)")
    ap.add_argument("--lagrange-transfer", default="default", choices=["default", "cuda", "tc", "ts"],
                    help="Laplace Lagrange transfer: the default / autotuned pick, or forced (CUDA cores, tcgen05 "
                         "per translation, tcgen05 target-stationary)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="default kernel variants instead of ffm_autotune's picks")
    return ap.parse_args()


def make_problem(name, seed, n=0):
    """The named workload; n > 0 overrides its point count (same generator, k kept at 10
    points per wavelength), for profiling runs on smaller cases."""
    from paper_1909_05600_gb300 import workloads as W
    if name == "helmholtz_sphere_1M":
        return W.helmholtz_sphere(n or 1_000_000, seed=seed)
    if name == "helmholtz_cube_200k_64rhs":
        return W.helmholtz_cube_multirhs(n or 200_000, nrhs=64, seed=seed, eps=1e-4)
    if name == "laplace_clustered":
        return W.laplace_clustered(n or 100_000_000, seed=seed)
    if name == "laplace_double_layer_sphere_1M":
        return W.laplace_double_layer_sphere(n or 1_000_000, seed=seed)
    if name == "laplace_gradient_sphere_1M":
        return W.laplace_gradient_sphere(n or 1_000_000, seed=seed)
    return W.laplace_sphere(n or 20000, seed=seed)


def workload_name(args, prob):
    """The workload as named in the JSON line: its name, with the point count when it is not
    the workload's own (1e8 written as 1e8)."""
    n = int(prob.X.shape[0])
    lg = math.log10(n) if n > 0 else 0.0
    label = "1e%d" % round(lg) if abs(lg - round(lg)) < 1e-12 else str(n)
    if args.workload == "laplace_clustered":
        return "laplace_clustered_%s" % label
    return args.workload if args.n == 0 else "%s_n%s" % (args.workload, label)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def rejected(clk):
    bad = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}
    if bad & set(clk.get("reasons", [])):
        return True
    if clk.get("sm_mhz") and clk.get("sm_max_mhz") and clk["sm_mhz"] < 0.5 * clk["sm_max_mhz"] \
            and "sw_power_cap" not in clk.get("reasons", []):
        return True
    return False


def cpu_direct_sample(prob, ntargets, seed=12345):
    """The FP64 CPU oracle's direct sum (eq. 3) for a seeded subset of targets."""
    from oracle import oracle as O
    from paper_1909_05600_gb300 import workloads as W
    t = W.sample_targets(prob.X.shape[0], ntargets, seed)
    u = prob.u.astype(np.complex128) if np.iscomplexobj(prob.u) else prob.u.astype(np.float64)
    t0 = time.perf_counter()
    if "normals" in prob.meta:  # the double layer
        ref = O.direct_dl(prob.X, prob.Y, prob.meta["normals"], u, w=prob.w, targets=t)
    elif prob.kind == W.LAPLACE_GRAD:  # (targets, nrhs, 3) -> (targets, 3 nrhs)
        ref = O.direct_grad(prob.X, prob.Y, u, w=prob.w, targets=t).reshape(len(t), -1)
    else:
        ref = O.direct(prob.X, prob.Y, u, prob.kind, prob.k, w=prob.w, targets=t)  # (targets, nrhs)
    dt = time.perf_counter() - t0
    return t, ref, dt, O.nthreads()


def reference_targets(prob):
    """Targets per timed oracle step: about 1.2e9 target-source pairs, at least 16, at most
    all targets."""
    return int(min(prob.X.shape[0], max(16, 1.2e9 // prob.Y.shape[0])))


def as_f64(prob):
    """The problem's coordinates and weights as FP64 arrays, converted once (the oracle
    computes in FP64; float32 inputs are promoted exactly)."""
    prob.X = np.ascontiguousarray(prob.X, dtype=np.float64)
    prob.Y = np.ascontiguousarray(prob.Y, dtype=np.float64)
    prob.w = np.ascontiguousarray(prob.w, dtype=np.float64)
    return prob


def cpu_legs(prob, args, vg):
    """The oracle beside the GPU result vg (first right-hand side; (nx,) or (nx, 3) for the
    gradient), on this host's cores:
      - O1 (FP64 direct sum) on a seeded subset of targets with all cores: the rel-L2 error of
        the GPU result there, and the baseline rate scaled to the full product; with
        --cpu-targets 0 the subset is as large as fills --cpu-seconds (256..4096 targets,
        sized from a 16-target probe);
      - O1 with one core on a smaller subset (about a quarter of that time), scaled;
      - O2 (the plain CPU FFM, plan + apply) on the 20,000-point Laplace sphere (the smallest
        workload), with all cores and with one core."""
    from oracle import oracle as O
    from paper_1909_05600_gb300 import workloads as W
    nx = prob.X.shape[0]
    cores = O.nthreads()
    ntg = args.cpu_targets
    if ntg <= 0:
        cpu_direct_sample(prob, 1, seed=778)  # loads the library and starts its threads
        _, _, dtp, _ = cpu_direct_sample(prob, 16, seed=777)
        ntg = int(min(4096, max(256, 16 * args.cpu_seconds / max(dtp, 1e-6))))
    ntg = min(ntg, nx)
    t, ref, dt, _ = cpu_direct_sample(prob, ntg)
    if prob.kind == W.LAPLACE_GRAD:
        vg = vg.T  # (nx, 3)
        ref = ref[:, :3]
    else:
        ref = ref[:, 0]
    err = float(np.linalg.norm(vg[t] - ref) / np.linalg.norm(ref))
    nrhs = 1 if prob.u.ndim == 1 else prob.u.shape[1]
    cpu = {"value": 1.0 / (dt * nx / len(t)), "unit": "applies/s", "cores": cores, "kind": "oracle",
           "sample": "O1, FP64 direct sum over all %d sources for %d seeded targets and all %d right-hand sides "
                     "(%.1f s), scaled to %d targets" % (prob.Y.shape[0], len(t), nrhs, dt, nx)}
    # one core, a smaller seeded subset
    n1 = max(4, int(len(t) * 0.25 / cores))
    O.set_threads(1)
    try:
        _, _, dt1, _ = cpu_direct_sample(prob, n1, seed=4242)
    finally:
        O.set_threads(cores)
    cpu["one_core"] = {"value": 1.0 / (dt1 * nx / n1), "unit": "applies/s", "cores": 1,
                       "sample": "O1 for %d seeded targets (%.1f s), scaled to %d targets" % (n1, dt1, nx)}
    # O2 on the smallest workload (plan + apply; FP64 per-pair operators)
    small = as_f64(W.laplace_sphere(20000, seed=1))
    o2 = {}
    for nthr in (cores, 1):
        O.set_threads(nthr)
        try:
            t0 = time.perf_counter()
            O.ffm(small.X, small.Y, small.u, O.LAPLACE, 0.0, small.eps, w=small.w)
            o2["cores_%d" % nthr] = {"value": 1.0 / (time.perf_counter() - t0), "unit": "applies/s",
                                     "cores": nthr}
        finally:
            O.set_threads(cores)
    cpu["o2_cpu_ffm"] = dict(o2, workload="laplace_sphere_20k", eps=small.eps,
                             note="the plain CPU FFM (plan + apply) of the oracle; the headline workload is "
                                  "far beyond its reach")
    return err, len(t), cpu


def repeat_applies(ffm, torch, prob, X, Y, w, u, flush, stream, reps, tune_cache=None, kw=None):
    """Repeated products with one resident plan (an iterative solver's use): eager
    ffm_apply calls against launches of the same apply captured as a CUDA graph.  Device
    time per product with an L2 flush before each one (outside its events)."""
    with ffm.Plan(X, Y, prob.kind, prob.k, prob.eps, weights=w, autotune_cache=tune_cache, **(kw or {})) as p:
        out = p.apply(u)  # the output buffer (its shape depends on the kernel)

        def run(fn):
            fn()
            torch.cuda.synchronize()
            tot = 0.0
            for _ in range(reps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                e1.synchronize()
                tot += e0.elapsed_time(e1)
            return reps / (tot * 1e-3)
        eager = run(lambda: p.apply(u, out=out))
        with p.graph(u, out) as g:
            graph = run(lambda: g.launch())
            kernels = g.kernels
    return {"eager_applies_per_s": eager, "graph_applies_per_s": graph, "kernels_per_apply": kernels,
            "reps": reps, "note": "plan built once; ffm_apply vs one CUDA graph launch per product"}


def run_reference(args, rank):
    """The oracle as it stands, timed on this host's cores: each step is the FP64 direct
    sum over all sources for a bounded sample of targets, scaled to the full product."""
    if rank != 0:
        return
    prob = as_f64(make_problem(args.workload, 1, args.n))
    if args.eps > 0:
        prob.eps = args.eps
    n = prob.X.shape[0]
    ns = reference_targets(prob)
    for _ in range(args.warmup):
        cpu_direct_sample(prob, ns)
    dts = []
    cores = 0
    for _ in range(args.steps):
        _, _, dt, cores = cpu_direct_sample(prob, ns)
        dts.append(dt * n / ns)
    tot = sum(dts)
    value = args.steps / tot
    line = {"impl": "reference", "metric": "FFM applies/s", "value": value, "unit": "applies/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args, prob), "n": n, "k": prob.k, "eps": prob.eps},
            "cpu_baseline": {"value": value, "unit": "applies/s", "cores": cores, "kind": "oracle",
                             "sample": "FP64 direct sum over all %d sources for %d seeded targets per step, "
                                       "scaled to %d targets" % (n, ns, n)},
            "e2e": {"value": value, "unit": "applies/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def measured_traffic(kernel):
    """DRAM bytes per algorithmic unit of `kernel` (the unit of its roofline family) from the
    committed ncu summary profiles/traffic.txt, or None when there is none or the kernel's
    source file has changed since the counters were taken.  Each line:
    kernel  capture_workload  bytes_per_unit  unit  source_file  source_sha256[:16]."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    for line in lines:
        f = line.split()
        if len(f) != 6 or line.startswith("#") or f[0] != kernel:
            continue
        src = os.path.join(ROOT, "paper_1909_05600_gb300", "csrc", f[4])
        try:
            h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        except OSError:
            return None
        return {"bytes_per_unit": float(f[2]), "unit": f[3], "captured_on": f[1]} if h == f[5] else None
    return None


def roofline(prof, info, steps, clk, pk, pk_kind, workload, nrhs=1):
    """Dominant kernel of the timed region against the pipe that bounds it.
    - Plane-wave transforms and the Helmholtz near field: the special-function (MUFU)
      pipe.  A point-direction pair of a transform costs one MUFU op (one sin and one cos
      serve a direction and its antipode, eq. 17's quadrature being symmetric); a Helmholtz
      near pair costs three (rsqrt, sin, cos).
    - Laplace near field: instruction issue, at one rsqrt and about nine FP32 operations
      per pair (10 issue slots).  Double-layer near field: the same pipe at 64 slots per
      pair (hi+lo difference, rsqrt, cube, and the compensated dot product n.(x - y)).
      Gradient near field: 20 slots (hi+lo difference, rsqrt, cube, three multiply-adds).
    - Gegenbauer transfer tables: FP32 issue, 72 instructions per recurrence step (double-float),
      19 on FP32 levels.
    - NUFFT grid kernels: the FP32 pipe, 4 FLOP per complex x real multiply-add of a W^3
      kernel window (per direction and box, or per point).
    - Lagrange transfer: tensor cores, 2 r r_K FLOP per admissible pair (r_K = r, or 3 r for
      the double layer's stacked component kernels; the single-precision GEMM; the TF32 hi/lo split triples the MMA work but not the algorithmic work), against
      the measured BF16 peak times the nominal TF32/BF16 ratio (1.1 / 2.25).
    - Plane-wave transforms of several right-hand sides on the tensor cores: 8 FLOP per
      (point, direction pair, right-hand side) (the real GEMMs P and Q over 2 columns per
      right-hand side), against the same TF32 peak.
    - Plane-wave transfer, and the double-float transforms of several right-hand sides: FP32
      issue, per (admissible pair or point, direction, right-hand side) a complex
      multiply-add: 4 instructions in FP32, 16 compensated (TwoSum), 72 in double-float
      arithmetic (4 multiplies of 7 instructions and 4 additions of 11)."""
    # the dominant kernel of this library (library calls such as cuFFT are listed, not ranked)
    name, (nl, ms) = max(((k, v) for k, v in prof.items() if "(library)" not in k), key=lambda kv: kv[1][1])
    mhz = pk.get("sm_max_mhz", 2070.0)
    clk_hz = mhz * 1e6
    helm = any(m == 2 for m in info["mode"])
    dl = workload.startswith("laplace_double_layer")
    grad = workload.startswith("laplace_gradient")
    kfac = 3 if dl or grad else 1
    out = {"kernel": name, "launches_per_step": nl / steps, "ms_per_step": ms / steps, "traffic": None}
    per_s = lambda units: units * steps / (ms * 1e-3)
    basis = "%d SMs x %%s x %.0f MHz (max SM clock, %s peaks file)" % (SM_COUNT, mhz, pk_kind)
    tag = name[name.find("<") + 1:name.find(">")] if "<" in name else ""
    prec_of = {"f32": 1, "f32c": 2, "f64": 3, "f32x2": 4}
    nufft = info.get("nufft", [0] * 22)
    levels = [l for l in range(22) if info["mode"][l] == 2 and not nufft[l] and info["pw_prec"][l] == prec_of.get(tag, -1)]
    if ("k_pw_forward_tc" in name or "k_pw_backward_tc" in name) and tag in prec_of:
        key = "src_points" if "forward" in name else "tgt_points"
        units = 8.0 * nrhs * sum(info[key][l] * info["nQ"][l] / 2 for l in levels)
        peak = pk.get("bf16_tflops", 1900.0) * 1e12 * (1.1 / 2.25)
        out.update({"bound": "tensor", "pipe": "TF32", "unit": "TFLOP/s", "units_per_step": units,
                    "peak_basis": "measured BF16 %.1f TFLOP/s x 1.1/2.25 (%s peaks file)"
                                  % (pk.get("bf16_tflops", 1900.0), pk_kind)})
    elif ("k_pw_transfer" in name or (nrhs > 1 and tag in ("f32x2", "f32c") and
                                      ("k_pw_forward_mr" in name or "k_pw_backward_mr" in name))) and tag != "f64":
        per = {"f32": 4.0, "f32c": 16.0, "f32x2": 72.0}.get(tag, 4.0)
        if "k_pw_transfer" in name:
            units = per * nrhs * sum(info["n_adm"][l] * info["nQ"][l] for l in levels)
        else:
            key = "src_points" if "forward" in name else "tgt_points"
            units = per * nrhs * sum(info[key][l] * info["nQ"][l] / 2 for l in levels)
        peak = SM_COUNT * 128 * clk_hz
        out.update({"bound": "alu", "pipe": "FP32 issue (%g instructions per complex multiply-add)" % per,
                    "unit": "Tops/s", "units_per_step": units, "peak_basis": basis % "128 lanes/clk"})
    elif "k_pw_forward" in name or "k_pw_backward" in name:
        key = "src_points" if "forward" in name else "tgt_points"
        units = 1.0 * sum(info[key][l] * info["nQ"][l] for l in range(22) if info["mode"][l] == 2)
        peak = SM_COUNT * MUFU_PER_SM_CLK * clk_hz
        out.update({"bound": "alu", "pipe": "MUFU", "unit": "Tops/s", "units_per_step": units,
                    "peak_basis": basis % ("%d MUFU results/clk" % MUFU_PER_SM_CLK)})
    elif "k_p2p" in name and helm:
        units = 3.0 * info["p2p_pairs"]
        peak = SM_COUNT * MUFU_PER_SM_CLK * clk_hz
        out.update({"bound": "alu", "pipe": "MUFU", "unit": "Tops/s", "units_per_step": units,
                    "peak_basis": basis % ("%d MUFU results/clk" % MUFU_PER_SM_CLK)})
    elif "k_p2p" in name:
        slots = 64 if dl else 20 if grad else 10
        units = 1.0 * info["p2p_pairs"]
        peak = SM_COUNT * 128 * clk_hz / slots
        out.update({"bound": "alu", "pipe": "FP32 issue (%d slots per pair)" % slots, "unit": "Tpairs/s",
                    "units_per_step": units, "peak_basis": basis % ("128 lanes/clk / %d" % slots)})
    elif "k_pw_table" in name:
        # Gegenbauer transfer tables: per recurrence (translation pair, direction pair) and
        # degree, a Legendre step and the even / odd partial sums: in double-float arithmetic
        # 4 multiplies (7 FP32 instructions) and 4 adds (11) = 72 FP32 instructions; on FP32
        # levels (k_pw_table_f32) a 3-instruction step and two compensated products (8) = 19
        f32 = "f32" in name
        units = (19.0 if f32 else 72.0) * sum(info["pw_recurrences"][l] * info["L"][l] for l in range(22)
                                              if info["mode"][l] == 2
                                              and (info["pw_prec"][l] == 1 and info["cancel"][l] <= 250.0) == f32)
        peak = SM_COUNT * 128 * clk_hz
        out.update({"bound": "alu", "pipe": "FP32 issue" + ("" if f32 else " (double-float)"), "unit": "Tops/s", "units_per_step": units,
                    "peak_basis": basis % "128 lanes/clk"})
    elif "k_nu_" in name:
        # NUFFT grid kernels: complex x real multiply-adds (4 FLOP) of the W^3 kernel windows,
        # per direction and box (interpolation at the directions, spread of v~) or per point
        # (spread of the charges, interpolation at the targets), on the FP32 pipe
        lv = [l for l in range(22) if info["nufft"][l]]
        w3 = lambda l: float(info["nufft_w"][l]) ** 3
        if "k_nu_interp" in name:
            macs = sum(info["nQ"][l] * info["n_src_boxes"][l] * w3(l) for l in lv)
        elif "k_nu_bspread" in name:
            macs = sum(info["nQ"][l] * info["n_tgt_boxes"][l] * w3(l) for l in lv)
        elif "k_nu_spread" in name:
            macs = sum(info["src_points"][l] * w3(l) for l in lv)
        else:
            macs = sum(info["tgt_points"][l] * w3(l) for l in lv)
        units = 4.0 * macs
        peak = SM_COUNT * 128 * 2 * clk_hz
        out.update({"bound": "alu", "pipe": "FP32 (FMA)", "unit": "TFLOP/s", "units_per_step": units,
                    "peak_basis": basis % "128 FMA lanes/clk x 2 FLOP"})
    elif "k_lag_gemm" in name:
        variant = 2 if "_ts" in name else 1 if "_tc" in name else 0

        def lag_units(l):
            # (flops, transfer variant) of a Lagrange level: a dense r x r (x kfac) GEMM per
            # pair, or with ACA factors two r x rank GEMMs per pair (rank: the level's largest)
            r, rk = info["r1"][l] ** 3, info["aca_rank"][l]
            if rk > 0:
                return 4.0 * r * info["aca_pair_terms"][l], info["tune_tc"][l]
            return 2.0 * kfac * r * r * info["n_adm"][l], info["tune_tc"][l]

        units = sum(u for l in range(22) if info["mode"][l] == 1 for u, v in [lag_units(l)] if v == variant)
        peak = pk.get("bf16_tflops", 1900.0) * 1e12 * (1.1 / 2.25)
        out.update({"bound": "tensor", "pipe": "TF32", "unit": "TFLOP/s", "units_per_step": units,
                    "peak_basis": "measured BF16 %.1f TFLOP/s x 1.1/2.25 (%s peaks file)"
                                  % (pk.get("bf16_tflops", 1900.0), pk_kind)})
    elif name == "k_lag_aca":
        # ACA of the transfer matrices: per term, the rank-one update of the r x r residual
        # with its squared norm (3 FP64 operations per entry), plus filling the matrix
        units = sum(3.0 * (info["r1"][l] ** 3) ** 2 * (info["aca_terms"][l] + info["n_trans"][l])
                    for l in range(22) if info["aca_rank"][l] > 0)
        peak = 1.25e12
        out.update({"bound": "alu", "pipe": "FP64", "unit": "TFLOP/s", "units_per_step": units,
                    "peak_basis": "nominal FP64 1.25 TFLOP/s (no measured FP64 peak)"})
    else:
        out.update({"bound": "alu", "achieved": None, "peak": None, "unit": None, "frac": None})
        return out
    achieved = per_s(units) / 1e12
    out.update({"achieved": achieved, "peak": peak / 1e12, "frac": achieved / (peak / 1e12)})
    # DRAM bytes per launch: the per-unit figure of a one-launch ncu capture on a smaller case
    # of the same workload, times this step's units per launch
    tr = measured_traffic(name)
    if tr is not None:
        out["traffic"] = tr["bytes_per_unit"] * units / max(nl / steps, 1e-9)
        out["traffic_basis"] = ("dram__bytes_read.sum + dram__bytes_write.sum per %s from one ncu capture on %s, "
                                "scaled to this step's units per launch" % (tr["unit"], tr["captured_on"]))
    return out


def run_serving(args):
    """Serving stream: requests with N log-uniform in [1e4, 2e6], Laplace or Helmholtz,
    three geometries, eps in {1e-3, 1e-4}; with --scenes S > 0 the requests share S scenes
    (point sets, kernel, k, eps) and differ in their densities, so plans are reused and
    same-scene requests merge into multi-RHS applies.  Inputs resident in HBM.  Passes over
    the same requests:
      - plain FP32: one stream, ffm_plan + ffm_apply + ffm_destroy in turn, with FP32 forced
        on every plane-wave level, direct plane-wave sums and the CUDA-core transfer;
      - single stream: the same loop with the default (mixed-precision, tensor-core, NUFFT)
        kernels; its throughput is the capacity the arrival rates refer to;
      - served, saturated: every request queued at once (continuous batching, plan cache,
        multi-RHS merging, one stream per worker);
      - served at Poisson arrival rates 0.5, 0.8 and 1.0 x capacity: p50 / p99 latency.
    Device overlap = summed per-batch device time (CUDA events on each worker stream) over
    the wall time of the pass.  Accuracy: rel-L2 vs the FP64 direct sum on sampled targets
    of the first requests, for the plain FP32 and the served results."""
    import torch
    from oracle import oracle as O
    from paper_1909_05600_gb300 import build, ffm, workloads as W
    from paper_1909_05600_gb300.serving import Request, Server, latency_stats
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    descs = W.serving_stream(args.requests, scenes=args.scenes)
    t0 = time.perf_counter()
    reqs, scene_pts, probs = [], {}, {}
    for d in descs:
        if d["scene"] not in scene_pts:
            pts = W.serving_points(d)
            t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
            scene_pts[d["scene"]] = (pts, t(pts[0]), t(pts[1]))
        pts, tX, tY = scene_pts[d["scene"]]
        pr = W.serving_problem(d, points=pts)
        if len(probs) < args.err_requests:
            probs[d["id"]] = pr
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
        reqs.append(dict(rid=d["id"], key=(d["scene"], pr.kind, pr.k, pr.eps), nx=pr.X.shape[0], ny=pr.Y.shape[0],
                         kind=pr.kind, k=pr.k, eps=pr.eps, X=tX, Y=tY, w=t(pr.w), u=t(pr.u)))
    t_gen = time.perf_counter() - t0
    n_pts = sum(r["nx"] for r in reqs)
    stream = torch.cuda.current_stream(dev)
    l0 = ffm.launch_count()
    plain_kw = dict(precision=ffm.PREC_F32, pw_transform=ffm.PW_DIRECT, lagrange_transfer=ffm.LAG_CUDA_CORES)

    def one_stream(kw):
        """Requests in arrival order on one stream; device-timed throughput, per-request
        latency (plan + apply + destroy, synchronised), and the results of the first ones."""
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        lat, res = [], {}
        for r in reqs:
            tq = time.perf_counter()
            with ffm.Plan(r["X"], r["Y"], r["kind"], r["k"], r["eps"], weights=r["w"], **kw) as p:
                v = p.apply(r["u"])
            torch.cuda.synchronize()
            lat.append(1e3 * (time.perf_counter() - tq))
            if r["rid"] in probs:
                res[r["rid"]] = v.cpu().numpy()
        ev1.record(stream)
        torch.cuda.synchronize()
        t = ev0.elapsed_time(ev1) * 1e-3
        return {"throughput_rps": len(reqs) / t, "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99))}, res

    st_plain, res_plain = one_stream(plain_kw)
    st_single, _ = one_stream({})
    cap = st_single["throughput_rps"]

    def serve(rate):
        rng = np.random.default_rng(7)
        arrivals = np.zeros(len(reqs)) if rate is None else np.cumsum(rng.exponential(1.0 / rate, len(reqs)))
        objs = [Request(**r) for r in reqs]
        srv = Server(device=0, workers=args.workers)
        try:
            t_start = time.perf_counter()
            for o, ta in zip(objs, arrivals):
                while time.perf_counter() - t_start < ta:
                    time.sleep(0.0005)
                o.t_arrival = time.perf_counter()
                srv.submit(o)
            srv.drain(len(objs), timeout=1800)
        finally:
            srv.close()
        st = latency_stats(objs)
        st.update({"device_overlap": srv.device_ms * 1e-3 / st["wall_s"] if st.get("wall_s") else None,
                   "batches": srv.batches, "plan_cache_hits": srv.cache.hits, "plan_cache_misses": srv.cache.misses})
        if rate is not None:
            st["rate_rps"] = rate
        return st, objs

    st_sat, objs_sat = serve(None)
    at = {}
    for f in (0.5, 0.8, 1.0):
        at["%.1f" % f], _ = serve(f * cap)
    launches = ffm.launch_count() - l0

    def err(res_of):
        e = []
        for rid, pr in probs.items():
            t = W.sample_targets(pr.X.shape[0], args.err_targets, seed=rid)
            u = pr.u.astype(np.complex128) if np.iscomplexobj(pr.u) else pr.u.astype(np.float64)
            ref = O.direct(pr.X, pr.Y, u, pr.kind, pr.k, w=pr.w, targets=t)[:, 0]
            v = res_of(rid)
            e.append({"rid": rid, "n": int(pr.X.shape[0]), "kernel": int(pr.kind), "eps": pr.eps,
                      "err": float(np.linalg.norm(v[t] - ref) / np.linalg.norm(ref))})
        return e

    by_id = {o.rid: o for o in objs_sat}
    err_plain = err(lambda rid: res_plain[rid])
    err_served = err(lambda rid: by_id[rid].result.cpu().numpy())
    line = {"metric": "serving requests/s", "value": st_sat["throughput_rps"], "unit": "requests/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "serving_stream", "requests": len(reqs), "scenes": args.scenes,
                       "n_points_total": n_pts, "workers": args.workers, "generation_s": t_gen},
            "plain_fp32": dict(st_plain, path="one stream, plan + apply + destroy per request; FP32 forced on "
                                              "plane-wave levels, direct plane-wave sums, CUDA-core transfer"),
            "single_stream": dict(st_single, path="one stream, plan + apply + destroy per request, default kernels"),
            "served_saturated": st_sat, "served_at_capacity_fraction": at,
            "speedup_vs_plain_fp32": st_sat["throughput_rps"] / st_plain["throughput_rps"],
            "speedup_vs_single_stream": st_sat["throughput_rps"] / cap,
            "err_vs_fp64_direct": {"targets_per_request": args.err_targets, "plain_fp32": err_plain,
                                   "served": err_served,
                                   "max_err_over_eps": {"plain_fp32": max(x["err"] / x["eps"] for x in err_plain),
                                                        "served": max(x["err"] / x["eps"] for x in err_served)}},
            "gpu_launches": launches, "failed": [o.error for o in objs_sat if o.error][:3]}
    print(json.dumps(line), flush=True)


def run_bem(args):
    """Boundary-element solve: the Laplace single layer's Galerkin system on the unit sphere
    (P1, icosphere of level args.bem) with the Galerkin right-hand side of the constant 1, whose
    solution is the unit density.  A step is ffm_bem_create + ffm_bem_solve + ffm_bem_destroy,
    timed with CUDA events; the density's deviation from 1 is the accuracy."""
    import torch
    from paper_1909_05600_gb300 import build, ffm, workloads as W
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    V, F = W.icosphere(args.bem)
    P = V[F]
    area = 0.5 * np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1)
    rhs = np.zeros(len(V))
    np.add.at(rhs, F.ravel(), np.repeat(area / 3.0, 3))  # integral of each hat function
    tV, tF, trhs = (torch.as_tensor(a, device=dev) for a in (V, F, rhs))
    stream = torch.cuda.current_stream(dev)
    eps, tol = 1e-4, 1e-5

    def step():
        with ffm.Bem(tV, tF, eps=eps) as bem:
            x, it, rr = bem.solve(trhs, tol=tol, restart=100, maxit=1000)
            return x, it, rr, bem.products()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(0)
    clocks.start()
    l0 = ffm.launch_count()
    ev0.record(stream)
    for _ in range(args.steps):
        x, it, rr, prods = step()
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = ffm.launch_count() - l0
    t = ev0.elapsed_time(ev1) * 1e-3
    xs = x.cpu().numpy()
    line = {"metric": "BEM GMRES solves/s", "value": args.steps / t, "unit": "solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "bem_laplace_single_layer_icosphere_%d" % args.bem, "vertices": len(V),
                       "triangles": len(F), "quadrature_nodes": 3 * len(F), "eps": eps, "gmres_tol": tol,
                       "step": "ffm_bem_create + ffm_bem_solve + ffm_bem_destroy"},
            "gmres_iterations": it, "ffm_products_per_solve": prods, "relres": rr,
            "ffm_products_per_s": prods * args.steps / t,
            "density_error": {"mean_minus_1": float(xs.mean() - 1), "max_abs_minus_1": float(np.max(np.abs(xs - 1)))},
            "clocks": clk, "gpu_launches": launches}
    print(json.dumps(line), flush=True)


def max_over_ranks(vals, dist):
    """Element-wise maximum of per-rank timings (ms) over all ranks (the slowest replica sets
    the job's time); the values themselves with one rank."""
    if not dist:
        return list(vals)
    import torch
    import torch.distributed as tdist
    tt = torch.tensor(list(vals), dtype=torch.float64)
    tdist.all_reduce(tt, op=tdist.ReduceOp.MAX)
    return tt.tolist()


def whole_job_rate(steps, world, t_ms):
    """Products per second of the whole job: every rank runs `steps` products (weak scaling,
    one independent replica per GPU) in at most t_ms."""
    return steps * world / (t_ms * 1e-3)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo", rank=rank, world_size=world)
    if args.bem and args.impl == "ffm":
        if rank == 0:
            run_bem(args)
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return
    if args.serving and args.impl == "ffm":
        if rank == 0:
            run_serving(args)
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return
    if args.impl == "reference":
        run_reference(args, rank)
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    import torch
    from paper_1909_05600_gb300 import build, ffm, workloads as W

    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prob = make_problem(args.workload, 1 + rank, args.n)
    if args.eps > 0:
        prob.eps = args.eps
    n = max(prob.X.shape[0], prob.Y.shape[0])
    X = torch.as_tensor(prob.X, device=dev)
    Y = torch.as_tensor(prob.Y, device=dev)
    w = torch.as_tensor(prob.w, device=dev)
    u_host = np.ascontiguousarray(prob.u.T) if prob.u.ndim == 2 else prob.u  # (nrhs, n) for several RHS
    nrhs = 1 if prob.u.ndim == 1 else prob.u.shape[1]
    u = torch.as_tensor(u_host, device=dev)
    # extra plan arguments: the source normals of the double layer
    kw = {"normals": torch.as_tensor(prob.meta["normals"], device=dev)} if "normals" in prob.meta else {}
    kw["pw_transform"] = {"auto": ffm.PW_AUTO, "direct": ffm.PW_DIRECT, "nufft": ffm.PW_NUFFT,
                          "tc": ffm.PW_DIRECT_TC}[args.pw_transform]
    if args.aca > 0:
        kw["aca_eps"] = args.aca
    if args.lagrange_transfer != "default":
        kw["lagrange_transfer"] = {"cuda": ffm.LAG_CUDA_CORES, "tc": ffm.LAG_TC_TRANSLATION,
                                   "ts": ffm.LAG_TC_TARGET}[args.lagrange_transfer]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    # kernel variants: ffm_autotune times them once on a plan of this workload, before the
    # timed region; every plan below takes the picks from the cache file (no timing)
    tune_cache, tune = None, None
    if not args.no_autotune:
        import tempfile
        fd, tune_cache = tempfile.mkstemp(prefix="ffm_tune_", suffix=".txt")
        os.close(fd)
        t0 = time.perf_counter()
        with ffm.Plan(X, Y, prob.kind, prob.k, prob.eps, weights=w, **kw) as pt:
            ti = pt.autotune(nrhs=nrhs, cache_path=tune_cache)
        tune = {"seconds": time.perf_counter() - t0, "p2p_tchunk": ti["p2p_tchunk"], "p2p_smax": ti["p2p_smax"],
                "tune_tc": [ti["tune_tc"][l] for l in range(ti["l_stop"] + 1)],
                "tune_pw": [ti["tune_pw"][l] for l in range(ti["l_stop"] + 1)],
                "note": "picked once before the timed region; each timed plan reads them from the cache"}

    def step(events=None):
        if events:
            events[0].record(stream)
        p = ffm.Plan(X, Y, prob.kind, prob.k, prob.eps, weights=w, autotune_cache=tune_cache, **kw)
        if events:
            events[1].record(stream)
        v = p.apply(u)
        if events:
            events[2].record(stream)
        p.close()
        return v, p

    info = None
    for _ in range(args.warmup):
        flush.zero_()
        v, _ = step()
    torch.cuda.synchronize()
    with ffm.Plan(X, Y, prob.kind, prob.k, prob.eps, weights=w, autotune_cache=tune_cache, **kw) as p0:
        info = p0.info()

    def timed(profiled, nsteps):
        """nsteps steps between a barrier and synchronisations.  The unprofiled pass (K steps)
        gives the throughput; the profiled pass (the library brackets every kernel with two
        events) gives each kernel's device time for the roofline.  Event records cost host
        time per launch, which shows up as gaps between the many small kernels of a plan."""
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(nsteps)]
        clocks = Clocks(local)
        ffm.profile_reset()
        l0 = ffm.launch_count()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        clocks.start()
        vlast = None
        for i in range(nsteps):
            flush.zero_()  # L2 flush between steps, outside the step's events
            ffm.profile_enable(profiled)
            vlast, _ = step(ev[i])
            ffm.profile_enable(False)
        torch.cuda.synchronize()
        clk = clocks.stop()
        if dist:
            dist.barrier()
        launches = ffm.launch_count() - l0
        t_plan = sum(e[0].elapsed_time(e[1]) for e in ev)
        t_apply = sum(e[1].elapsed_time(e[2]) for e in ev)
        return vlast, t_plan, t_apply, clk, launches, (ffm.profile_read() if profiled else None)

    vlast, t_plan, t_apply, clk, launches, _ = timed(False, args.steps)
    # the profiled pass and the repeated applies take at most about 10 s each on large
    # workloads (at least one step, at most K)
    step_s = (t_plan + t_apply) * 1e-3 / args.steps
    apply_s = t_apply * 1e-3 / args.steps
    k_prof = max(1, min(args.steps, math.ceil(10.0 / max(step_s, 1e-9))))
    _, tp_plan, tp_apply, _, _, prof = timed(True, k_prof)
    reps = max(3, min(args.steps, math.ceil(5.0 / max(apply_s, 1e-9))))
    rep = repeat_applies(ffm, torch, prob, X, Y, w, u, flush, stream, reps, tune_cache, kw)
    note = None
    if rejected(clk):
        note = "first timed run rejected (clock reasons %s); re-measured" % clk.get("reasons")
        vlast, t_plan, t_apply, clk, launches, _ = timed(False, args.steps)
    t_step, t_plan, t_apply = max_over_ranks([t_plan + t_apply, t_plan, t_apply], dist)
    value = whole_job_rate(args.steps, world, t_step)
    pk, pk_kind = peaks()

    e2e = None
    if not args.no_e2e:
        Xh = torch.as_tensor(prob.X).pin_memory()
        Yh = torch.as_tensor(prob.Y).pin_memory()
        wh = torch.as_tensor(prob.w).pin_memory()
        uh = torch.as_tensor(u_host).pin_memory()
        kwh = {k: torch.as_tensor(prob.meta[k]).pin_memory() for k in kw if k in prob.meta}
        kwh["pw_transform"] = kw["pw_transform"]
        for key in ("aca_eps", "lagrange_transfer"):
            if key in kw:
                kwh[key] = kw[key]
        vshape = tuple(uh.shape[:-1]) + ((3,) if prob.kind == W.LAPLACE_GRAD else ()) + (prob.X.shape[0],)
        vh = torch.empty(vshape, dtype=uh.dtype).pin_memory()
        ke = max(2, min(args.steps // 2, math.ceil(15.0 / max(step_s, 1e-9))))
        ts = []
        for i in range(ke + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with ffm.Plan(Xh, Yh, prob.kind, prob.k, prob.eps, weights=wh, stream=stream,
                          autotune_cache=tune_cache, **kwh) as ph:
                ph.apply(uh, out=vh, stream=stream)
            torch.cuda.synchronize()
            if i:
                ts.append(time.perf_counter() - t0)
        h2d = Xh.numel() * Xh.element_size() + Yh.numel() * Yh.element_size() + wh.numel() * wh.element_size() \
            + uh.numel() * uh.element_size() + sum(t.numel() * t.element_size() for t in kwh.values()
                                                   if hasattr(t, "numel"))
        e2e = {"value": world * len(ts) / sum(ts), "unit": "applies/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": vh.numel() * vh.element_size(), "steps": len(ts),
               "api": "ffm_plan(host X, Y, w) + ffm_apply(host u -> host v) + ffm_destroy"}

    cpu = None
    err = None
    err_targets = None
    if rank == 0 and not args.no_cpu_baseline:
        vg = vlast.cpu().numpy()
        if prob.kind == W.LAPLACE_GRAD:
            vg = vg if vg.ndim == 2 else vg[0]  # (3, nx) of the first right-hand side
        else:
            vg = vg if vg.ndim == 1 else vg[0]
        err, err_targets, cpu = cpu_legs(as_f64(prob), args, vg)

    if rank == 0:
        rl = roofline(prof, info, k_prof, clk, pk, pk_kind, args.workload, nrhs)
        kernels = {k: {"launches_per_step": v[0] / k_prof, "ms_per_step": v[1] / k_prof}
                   for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}
        line = {
            "metric": "FFM applies/s", "value": value, "unit": "applies/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(args, prob), "n_x": int(prob.X.shape[0]),
                       "n_y": int(prob.Y.shape[0]),
                       "kernel": {0: "laplace", 1: "helmholtz", 2: "laplace_double_layer",
                                  3: "laplace_gradient"}[prob.kind],
                       "k": prob.k, "eps": prob.eps,
                       "u_dtype": str(prob.u.dtype), "step": "ffm_plan + ffm_apply + ffm_destroy",
                       "l2": "flushed between steps (512 MiB write, outside the step events)",
                       "replicas": world, "nrhs": nrhs, "pw_transform": args.pw_transform,
                       "lagrange_transfer": args.lagrange_transfer,
                       **({"aca_eps": args.aca} if args.aca > 0 else {})},
            "mpoints_per_s": n * value / 1e6, "rhs_per_s": value * nrhs,
            "t_plan_ms": t_plan / args.steps, "t_apply_ms": t_apply / args.steps,
            "apply_only_per_s": args.steps * world / (t_apply * 1e-3),
            "repeat_apply": rep, "autotune": tune,
            "profiled_pass_ms_per_step": (tp_plan + tp_apply) / k_prof, "profiled_pass_steps": k_prof,
            "err_vs_fp64_direct": err, "err_targets": err_targets,
            "roofline": rl, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "gpu_launches": launches,
            "kernels": kernels,
            "plan": {"l_stop": info["l_stop"], "mode": info["mode"][:info["l_stop"] + 1],
                     "L": info["L"][:info["l_stop"] + 1], "nQ": info["nQ"][:info["l_stop"] + 1],
                     "n_adm": info["n_adm"][:info["l_stop"] + 1], "p2p_pairs": info["p2p_pairs"],
                     "nufft": info["nufft"][:info["l_stop"] + 1], "nufft_n2": info["nufft_n2"][:info["l_stop"] + 1],
                     "pw_prec": info["pw_prec"][:info["l_stop"] + 1], "cancel": info["cancel"][:info["l_stop"] + 1],
                     "tune_tc": info["tune_tc"][:info["l_stop"] + 1],
                     **({"aca_rank": info["aca_rank"][:info["l_stop"] + 1]} if args.aca > 0 else {})},
        }
        if note:
            line["note"] = note
        print(json.dumps(line), flush=True)
    if tune_cache:
        os.remove(tune_cache)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
