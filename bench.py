#!/usr/bin/env python
"""Benchmark: forward + adjoint reduced gradient of the tumor
reaction-diffusion model at 256^3 (nt = 32, 125 Gaussians), in cell-updates/s.

One step = one ``rd_gradient`` call: Gaussian synthesis, the Strang/CN
forward solve with PCG, the misfit, the discrete adjoint sweep and the
gradient assembly (p, k_f, rho_f).  cell-updates/s = n^3 * nt / step time.

Inputs are seeded synthetic brain-like fields (``synth.calibration_problem``)
resident in HBM before the timed region for ``value``; ``e2e`` repeats the
step through the C ABI from pinned host buffers (tissue maps and data copied
in, gradient copied out, every step).  Every field is 64 MiB (FP32) or more,
so the working set (> 2 GiB) is far larger than L2.

``--impl reference`` times the FP64 CPU oracle on the host instead (a
bounded sample: one operator application and one preconditioner
application at the same grid, scaled by the oracle's own PCG work for this
gradient, which a full oracle run stored under tests/golden/; labelled
"extrapolated").  The CPU baseline of the main line adds complete oracle
gradients at 64^3 timed on one core and on all host cores.
Multi-GPU runs (torchrun) execute independent replicas, one per rank.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+adjoint gradient cell-updates/s at 256^3 (FP32-mixed vs FP64, same GB300), %HBM peak"
UNIT = "cell-updates/s"
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0   # GB300 HBM3e data-sheet bandwidth (context only)
GOLDEN = os.path.join(ROOT, "tests", "golden")


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(x, dist=None, device="cuda"):
    """The largest value of x over all ranks (the slowest rank's time); x
    itself on a single process."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, ms_max):
    """Whole-job throughput of independent replicas (weak scaling): the
    units every rank processed, divided by the slowest rank's time."""
    return world * units_per_rank / (ms_max / 1e3)


def problem(n, nt):
    from paper_1907_07774_gb300 import synth
    return synth.calibration_problem(n=n, nt=nt, m=round(GRADIENT_GAUSSIANS ** (1 / 3)))


GRADIENT_GAUSSIANS = 125   # 5^3 Gaussians of the calibration recipe at the benchmark grid


def gradient_config(n, nt, np_, ckpt_stride, world):
    """The workload both arms measure: one reduced gradient (forward solve,
    adjoint solve, gradient) of the calibration problem, PCG rtol 1e-6.  The
    arithmetic each arm uses is in its dtype and its own keys, not here."""
    return {"workload": f"rd_gradient {n}^3 nt={nt} np={np_} pcg_rtol=1e-6", "grid": n, "nt": nt, "np": np_,
            "ckpt_stride": ckpt_stride,
            "l2": f"inputs larger than L2 (fields {n ** 3 * 4 / 2 ** 20:.0f} MiB in FP32, working set "
                  f"{n ** 3 * 4 * (nt + 18) / 2 ** 30:.1f} GiB)",
            "parallelism": "replicas" if world > 1 else "single"}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


FP64_RTOL = 1e-10   # PCG tolerance of the FP64 arm (the plain FP64 solve of the 64^3 workload)

def csrc_hash():
    """Hash of the CUDA sources of the tumor solver (the registration and the
    allocation-free entry point are other translation units and do not
    change the tumor kernels)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1907_07774_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.startswith("rd_reg") or f == "rd_noalloc.cu":
            continue
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(cls, n):
    """Per-launch DRAM bytes of a kernel class from the committed ncu
    summary, if it was taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
    except Exception:
        return None
    if d.get("csrc_hash") != csrc_hash():
        return None
    ent = d.get("classes", {}).get(cls)
    if not ent:
        return None
    return float(ent["bytes_per_launch"]) * (n ** 3) / float(ent.get("cells", n ** 3))


def ncu_dram_weighted(prof, n, peak):
    """Time-weighted DRAM throughput of the FFT/operator kernels from ncu's
    DRAM counters: the committed per-launch DRAM bytes of each class (one
    ncu capture on the current sources, profiles/ncu_traffic.json) times the
    launches of this step, over the classes' live CUDA-event time.  ncu
    replays each launch with cold caches, so its bytes bound the live ones
    from above; None when the capture predates the sources."""
    tot_b, tot_ms, used = 0.0, 0.0, []
    for cls, (ms, cnt) in prof.items():
        if not cnt:
            continue
        b = ncu_traffic(cls, n)
        if b is None:
            continue
        tot_b += b * cnt
        tot_ms += ms
        used.append(cls)
    if not used or tot_ms <= 0:
        return None
    gbs = tot_b / (tot_ms / 1e3) / 1e9
    return {"gbs": gbs, "frac": gbs / peak, "classes": used,
            "source": "profiles/ncu_traffic.json (dram__bytes_read.sum + dram__bytes_write.sum per launch)"}


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        try:
            for line in open(self.f.name):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.f.name)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]),
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_median": statistics.median(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


# algorithmic fields moved per launch of each kernel class, over the whole grid
# (the CG update reads r and q and writes r and H_2 r; x += alpha p rides on
# the next iteration's direction kernel)
FIELDS_PER_LAUNCH = {"op_axis01": 4, "op_axis2": 3, "pcg_opx": 5, "dht_plain": 2, "dht_sym": 2,
                     "dht_setup": 2, "dht_update": 4, "grad": 4}


def fields_per_launch(active, iters=0, solves=0):
    """Fields each class must move per launch once the tiles where kappa
    vanishes are skipped (rd_active_tiles): the strided operator passes move
    u, kappa, q in and q out only on active tiles (axes 0 and 1 alternate);
    the direction kernel reads kappa only on active row tiles; the k_f
    gradient passes (axes 2, 1, 0) skip inactive strided tiles.  From the
    second iteration of a solve on, the direction kernel also reads and
    writes x (the deferred x += alpha p)."""
    f0 = active["axis0"][0] / max(1, active["axis0"][1])
    f1 = active["axis1"][0] / max(1, active["axis1"][1])
    fr = active["rows"][0] / max(1, active["rows"][1])
    out = dict(FIELDS_PER_LAUNCH)
    out["op_axis01"] = 4 * 0.5 * (f0 + f1)
    out["pcg_opx"] = 4 + fr
    out["grad"] = 4 * (1 + f0 + f1) / 3
    if iters > 0:
        out["pcg_opx"] += 2 * max(0, iters - solves) / iters
    return out, {"axis0": f0, "axis1": f1, "rows": fr}


def oracle_case(n, nt):
    """The stored FP64 oracle run of this workload (tests/golden/, written by
    make_golden_full.py from the oracle alone): its scalars and its labels,
    or None.  The run at PCG rtol 1e-12 is preferred; the run at the
    benchmark's own rtol 1e-6 (same labels recipe) stands in otherwise."""
    import numpy as np
    for name in (f"grad{n}_nt{nt}", f"work{n}_nt{nt}_rtol1e-6"):
        js = os.path.join(GOLDEN, f"oracle_full_{name}.json")
        nz = os.path.join(GOLDEN, f"oracle_full_{name}.npz")
        if os.path.exists(js) and os.path.exists(nz):
            break
    else:
        return None
    want = json.load(open(js))
    bits = np.load(nz)["labels_bits"]
    labels = np.unpackbits(bits)[: n ** 3].reshape(n, n, n).astype(np.float64)
    return want, labels


def oracle_work(n, nt):
    """The oracle's own PCG work for the benchmark gradient (iterations,
    solves), stored by a full oracle run (tests/golden/make_golden_full.py,
    PCG rtol 1e-6 as in the benchmark), or None when no run is stored."""
    path = os.path.join(GOLDEN, f"oracle_full_work{n}_nt{nt}_rtol1e-6.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    its = d["pcg_iters_forward"] + d["pcg_iters_adjoint"]
    return {"iters": int(sum(its)), "solves": len(its), "source": os.path.relpath(path, ROOT),
            "seconds_x86": d.get("seconds_gradient")}


def cpu_oracle_sample(n, nt, k_f):
    """Time one FP64 oracle operator application and one preconditioner
    application on the host at grid n (the work of one PCG iteration)."""
    import numpy as np
    from oracle import rd as orc
    prob = problem(n, nt)
    M = orc.model_from_problem(prob, kind="numpy")
    u = np.random.default_rng(0).standard_normal(prob.n)
    t0 = time.perf_counter()
    M.A(u, k_f)
    t1 = time.perf_counter()
    M.sp.precond(u, M.s * k_f * orc.kbar_positive(M.kappa1))
    t2 = time.perf_counter()
    return t1 - t0, t2 - t1


def cpu_cells_per_s(n, nt, t_apply, t_prec, iters, solves):
    # per PCG iteration: one operator + one preconditioner; per solve: one
    # right-hand-side operator and one preconditioner; per adjoint step: the
    # k_f integrand (six transforms, ~3/4 of an operator)
    t = iters * (t_apply + t_prec) + solves * (t_apply + t_prec) + nt * 0.75 * t_apply
    return n ** 3 * nt / t, t


def fft_flops_per_gradient(n, nt, iters, solves):
    """Estimated floating-point operations of one gradient on the GPU path:
    every pencil transform of length L costs 5 L log2 L flops per packed pair
    of real pencils, i.e. 2.5 log2 L per real value; a PCG iteration makes 18
    transforms per cell (Hartley passes 1 + 2 + 1 + 1, direction kernel 5, two
    operator passes 4 each), a solve's set-up and right-hand side 13, an
    adjoint step's k_f integrand 12.  Pointwise work is left out (a few per
    cent)."""
    per_transform = 2.5 * math.log2(n)
    transforms = iters * 18 + solves * 13 + nt * 12
    return transforms * per_transform * n ** 3


def cpu_model():
    """CPU model name of this host (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


_FULL = {"n": 64, "nt": 16, "m": 4}


def _full_gradient_worker(args):
    """One complete oracle gradient (single-threaded child process)."""
    n, nt, m, d = args
    from oracle import rd as orc
    from paper_1907_07774_gb300 import synth
    prob = synth.calibration_problem(n=n, nt=nt, m=m)
    M = orc.model_from_problem(prob, rtol=1e-6, maxit=5000, kind="numpy")
    t0 = time.perf_counter()
    M.gradient(prob.p, prob.k_f, prob.rho_f, d)
    return time.perf_counter() - t0, int(sum(M.iters))


def cpu_full_gradients():
    """Complete oracle gradients of the calibration recipe at 64^3, nt = 16
    (PCG rtol 1e-6), timed on one core and on every host core at once (one
    single-threaded process per core, independent problems), in
    cell-updates/s; the data are made once by the oracle and not timed."""
    import multiprocessing as mp
    from oracle import rd as orc
    from paper_1907_07774_gb300 import synth
    n, nt, m = _FULL["n"], _FULL["nt"], _FULL["m"]
    prob = synth.calibration_problem(n=n, nt=nt, m=m)
    M = orc.model_from_problem(prob, rtol=1e-6, maxit=5000, kind="numpy")
    c_true, _ = M.forward(prob.p_true, prob.k_f_true, prob.rho_f_true)
    d = synth.labels(c_true, synth.ellipsoid_mask(prob.n), prob.seed + 7)
    cores = os.cpu_count() or 1
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    ctx = mp.get_context("spawn")
    with ctx.Pool(1) as pool:
        t1, its = pool.map(_full_gradient_worker, [(n, nt, m, d)])[0]
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_full_gradient_worker, [(n, nt, m, d)] * cores)
    tall = time.perf_counter() - t0
    cells = n ** 3 * nt
    return {"workload": f"oracle gradient {n}^3 nt={nt} np={m ** 3} pcg_rtol=1e-6 (numpy FFT, FP64)",
            "pcg_iters": its, "one_core": {"seconds": t1, "value": cells / t1, "cores": 1},
            "all_cores": {"seconds_wall": tall, "value": cores * cells / tall, "cores": cores,
                          "note": "one single-threaded oracle gradient per core, run at once; wall time "
                                  "includes process start-up"},
            "unit": UNIT}


def cpu_extrapolated(n, nt, k_f):
    """The oracle on the benchmark workload itself: one operator and one
    preconditioner application timed at n^3, scaled by the oracle's own PCG
    work for the whole gradient."""
    ta, tp = cpu_oracle_sample(n, nt, k_f)
    w = oracle_work(n, nt)
    if w is None:
        return None, ta, tp
    v, tgrad = cpu_cells_per_s(n, nt, ta, tp, w["iters"], w["solves"])
    return {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"extrapolated: one FP64 operator application ({ta:.2f} s) and one preconditioner "
                      f"application ({tp:.2f} s) of the oracle (numpy FFT) at {n}^3, scaled by the oracle's own "
                      f"PCG work for this gradient ({w['iters']} iterations in {w['solves']} solves at rtol 1e-6, "
                      f"from {w['source']}): {tgrad:.0f} s per gradient",
            "seconds_per_gradient": tgrad}, ta, tp


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    n, nt = args.n, args.nt
    w = oracle_work(n, nt)
    if w is None:
        print(json.dumps({"impl": "reference", "unavailable": f"no stored oracle PCG work for {n}^3 nt={nt}"}))
        return 0
    steps = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        ta, tp = cpu_oracle_sample(n, nt, 0.02)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            steps.append((dt, ta, tp))
    ta = statistics.median(s[1] for s in steps)
    tp = statistics.median(s[2] for s in steps)
    value, tgrad = cpu_cells_per_s(n, nt, ta, tp, w["iters"], w["solves"])
    ms_step = 1e3 * statistics.mean(s[0] for s in steps)
    sample = (f"extrapolated: each step times one FP64 operator application ({ta:.2f} s) and one preconditioner "
              f"application ({tp:.2f} s) of the oracle (numpy FFT) at {n}^3 on one core; value = the gradient's "
              f"cell-updates over the oracle's own PCG work for it ({w['iters']} iterations in {w['solves']} "
              f"solves at rtol 1e-6, {w['source']}): {tgrad:.0f} s per gradient")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": gradient_config(n, nt, GRADIENT_GAUSSIANS, args.ckpt_stride, world),
            "arithmetic": "the FP64 CPU oracle (numpy FFT), one core",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             "nproc": os.cpu_count(), "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, rank, world, local):
    import numpy as np
    import torch

    from paper_1907_07774_gb300 import build as _build
    from paper_1907_07774_gb300 import rd as R
    from paper_1907_07774_gb300 import synth

    _build.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    n, nt = args.n, args.nt
    prob = problem(n, nt)
    gkw = {} if args.guess_restart is None else {"guess_restart": args.guess_restart}
    ctx = R.context_for(prob, prec="mixed", pcg_rtol=1e-6, pcg_maxit=500, ckpt_stride=args.ckpt_stride, **gkw)
    gold = oracle_case(n, nt)
    if gold is not None:
        # the labels of the stored oracle run (thresholded oracle c_true(1))
        d_host = gold[1]
        data_src = "labels of the stored FP64 oracle run (tests/golden)"
    else:
        c_true = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
        ctx.rd_forward(prob.p_true, prob.k_f_true, prob.rho_f_true, c_true)
        d_host = synth.labels(c_true.cpu().numpy(), synth.ellipsoid_mask(prob.n), prob.seed + 7)
        del c_true
        data_src = "labels of the GPU mixed c_true(1)"
    d_dev = torch.from_numpy(d_host).cuda()
    m_dev = [torch.from_numpy(x).cuda() for x in (prob.m_wm, prob.m_gm, prob.m_csf)]
    ctx.rd_set_tissue(*m_dev)
    ctx.rd_set_data(d_dev)
    p, k_f, rho_f = prob.p, prob.k_f, prob.rho_f
    stream = torch.cuda.current_stream()
    tuned = ctx.rd_autotune(reps=3) if args.autotune else None

    for _ in range(args.warmup):
        J, g = ctx.rd_gradient(p, k_f, rho_f)
    iters, solves = ctx.rd_last_pcg_iters(), ctx.rd_last_pcg_solves()
    graph_solves = ctx.rd_last_graph_solves()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timed region (PCG solves run as CUDA graphs)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            J, g = ctx.rd_gradient(p, k_f, rho_f)
        e1.record(stream)
        barrier()
    ms = max_over_ranks(e0.elapsed_time(e1), dist)
    clocks = clk.summary()
    cells = n ** 3 * nt
    value = job_rate(cells * args.steps, world, ms)

    # ---- one more step of the same workload with every launch bracketed by
    # CUDA events on the solver's stream (host-driven PCG loop, same kernels)
    R.rd_profile_enable(True)
    barrier()
    ctx.rd_gradient(p, k_f, rho_f)
    barrier()
    prof = R.rd_profile_read()
    R.rd_profile_enable(False)
    launches_per_step = int(sum(c for _, c in prof.values()))

    # ---- roofline of the dominant kernel class
    esz = 4
    fpl, act_frac = fields_per_launch(ctx.rd_active_tiles(), iters, solves)
    dom = max((k for k in prof if k in fpl), key=lambda k: prof[k][0])
    dms, dcount = prof[dom]
    alg_bytes = fpl[dom] * n ** 3 * esz
    achieved = alg_bytes / (dms / dcount / 1e3) / 1e9
    peak, peak_kind = measured_peaks()
    pcg_classes = [k for k in fpl if k in prof and prof[k][1]]
    tot_bytes = sum(fpl[k] * n ** 3 * esz * prof[k][1] for k in pcg_classes)
    tot_ms = sum(prof[k][0] for k in pcg_classes)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind,
                "frac_of_nominal": achieved / NOMINAL_HBM_GBS, "nominal_gbs": NOMINAL_HBM_GBS,
                "traffic": ncu_traffic(dom, n), "alg_bytes_per_launch": alg_bytes,
                "avg_launch_us": 1e3 * dms / dcount, "launches_per_step": dcount,
                "share_of_step": dms / (ms / args.steps),
                "fft_operator_kernels_time_weighted_gbs": tot_bytes / (tot_ms / 1e3) / 1e9,
                "fft_operator_kernels_frac": tot_bytes / (tot_ms / 1e3) / 1e9 / peak,
                "ncu_dram": ncu_dram_weighted(prof, n, peak),
                "timing": "per-launch CUDA events in one profiled step after the timed region (host-driven "
                          "PCG loop: its class times sum to a little more than the graph-run step)",
                "active_tile_fraction": act_frac,
                "alg_fields_per_launch": {k: fpl[k] for k in pcg_classes}}
    per_class = {k: {"ms_per_step": v[0], "launches_per_step": v[1]} for k, v in prof.items() if v[1]}

    # ---- end to end through the C ABI from pinned host buffers
    host_m = [torch.from_numpy(x).pin_memory() for x in (prob.m_wm, prob.m_gm, prob.m_csf)]
    host_d = torch.from_numpy(d_host).pin_memory()
    barrier()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for _ in range(args.steps):
        ctx.rd_set_tissue(*host_m)
        ctx.rd_set_data(host_d)
        Je, ge = ctx.rd_gradient(p, k_f, rho_f)
    e3.record(stream)
    barrier()
    ms_e2e = max_over_ranks(e2.elapsed_time(e3), dist)
    e2e = {"value": job_rate(cells * args.steps, world, ms_e2e), "unit": UNIT,
           "h2d_bytes_per_step": 4 * n ** 3 * 8 + len(p) * 8,
           "d2h_bytes_per_step": (len(p) + 2) * 8 + 8}

    # ---- the same gradient with sqrt(nt) checkpoints (the adjoint recomputes
    # the states of each segment), and the batched uneven workload
    ckpt = None
    batch = None
    if rank == 0 and not args.no_extras:
        s_ck = int(math.ceil(math.sqrt(nt)))
        cck = R.context_for(prob, prec="mixed", pcg_rtol=1e-6, pcg_maxit=500, ckpt_stride=s_ck)
        cck.rd_set_data(d_dev)
        for _ in range(2):
            Jc, gc = cck.rd_gradient(p, k_f, rho_f)
        torch.cuda.synchronize()
        e4, e5 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e4.record(stream)
        for _ in range(3):
            Jc, gc = cck.rd_gradient(p, k_f, rho_f)
        e5.record(stream)
        torch.cuda.synchronize()
        ms_ck = e4.elapsed_time(e5) / 3
        del cck
        # the state solves' guesses restart at every segment start: a
        # store-all run restarting them at the same period gives the same bits
        csa = R.context_for(prob, prec="mixed", pcg_rtol=1e-6, pcg_maxit=500, guess_restart=s_ck)
        csa.rd_set_data(d_dev)
        Js, gs = csa.rd_gradient(p, k_f, rho_f)
        del csa
        ckpt = {"ckpt_stride": s_ck, "value": cells / (ms_ck / 1e3), "unit": UNIT, "ms_per_step": ms_ck,
                "steps": 3, "stored_states": (nt + s_ck - 1) // s_ck + s_ck,
                "grad_bitwise_equal_to_store_all_same_restarts": bool(Jc == Js and np.array_equal(gc, gs)),
                "grad_rel_diff_vs_headline_run": float(np.linalg.norm(gc - g) / np.linalg.norm(g))}
        torch.cuda.empty_cache()
        batch = batch_measure(R, synth, torch, 3, 1)

    # ---- FP64 path on the same GPU
    fp64 = None
    if args.fp64_steps > 0 and rank == 0:
        del ctx
        torch.cuda.empty_cache()
        c64 = R.context_for(prob, prec="fp64", pcg_rtol=FP64_RTOL, pcg_maxit=1000, ckpt_stride=args.ckpt_stride,
                            **gkw)
        c64.rd_set_data(d_dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.fp64_steps):
            J64, g64 = c64.rd_gradient(p, k_f, rho_f)
        torch.cuda.synchronize()
        s64 = (time.perf_counter() - t0) / args.fp64_steps
        it64, so64 = c64.rd_last_pcg_iters(), c64.rd_last_pcg_solves()
        flops64 = fft_flops_per_gradient(n, nt, it64, so64)
        fma64 = R.rd_probe_fma_rate("fp64")
        fp64 = {"value": cells / s64, "ms_per_step": 1e3 * s64, "pcg_iters": it64, "pcg_solves": so64,
                "alu_roofline": {"bound": "alu", "fma_peak_tflops_measured": fma64,
                                 "est_tflops_achieved": flops64 / s64 / 1e12,
                                 "frac": flops64 / s64 / 1e12 / fma64,
                                 "est_flops_per_gradient": flops64,
                                 "fp32_fma_peak_tflops_measured": R.rd_probe_fma_rate("mixed"),
                                 "note": "flops estimated from the transform count (bench.fft_flops_per_gradient); "
                                         "peak from rd_probe_fma_rate (register FMA loop)"},
                "mixed_speedup": (cells * args.steps / (ms / 1e3)) / (cells / s64),
                "mixed_grad_rel_err_vs_fp64": float(np.linalg.norm(g - g64) / np.linalg.norm(g64)),
                "mixed_misfit_rel_err_vs_fp64": abs(J - J64) / abs(J64)}
        del c64

    # ---- CPU oracle baseline (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, ta, tp = cpu_extrapolated(n, nt, k_f)
        if cpu is None:
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"no stored oracle PCG work for {n}^3 nt={nt}; one operator application "
                             f"{ta:.2f} s, one preconditioner application {tp:.2f} s"}
        cpu["nproc"] = os.cpu_count()
        cpu["cpu_model"] = cpu_model()
        if not args.no_cpu_full:
            cpu["measured_full_gradients"] = cpu_full_gradients()

    vs_oracle = None
    if gold is not None:
        want = gold[0]
        g_or = np.asarray(want["gradient"])
        vs_oracle = {"grad_rel_l2": float(np.linalg.norm(g - g_or) / np.linalg.norm(g_or)),
                     "misfit_rel": abs(J - want["misfit"]) / abs(want["misfit"]), "tolerance": 2e-4,
                     "oracle_pcg_rtol": want["case"]["rtol"]}
        if fp64 is not None:
            vs_oracle["fp64_grad_rel_l2"] = float(np.linalg.norm(g64 - g_or) / np.linalg.norm(g_or))
            vs_oracle["fp64_pcg_rtol"] = FP64_RTOL
            vs_oracle["fp64_note"] = ("the FP64 arm solves to rtol 1e-10 (the tolerance of the plain FP64 solve); "
                                      "its distance to the rtol-1e-12 oracle run is that tolerance. Solved to 1e-12 "
                                      "the FP64 path is within 1e-10 of this oracle run (tests/test_golden_full.py)")
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": gradient_config(n, nt, len(p), args.ckpt_stride, world),
                "arithmetic": "mixed: FP32 fields, FP64 reductions and PCG scalars",
                "misfit": J, "pcg_iters_per_step": iters, "pcg_solves_per_step": solves,
                "pcg_graph_solves_per_step": graph_solves,
                "data_labels": data_src, "vs_fp64_oracle": vs_oracle,
                "gpu_launches": launches_per_step * args.steps, "clocks": clocks, "roofline": roofline, "e2e": e2e,
                "cpu_baseline": cpu, "fp64": fp64, "checkpointed": ckpt, "batch": batch,
                "kernel_classes": per_class, "autotuned_blocks": tuned}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def _gpu_setup(local):
    import torch
    from paper_1907_07774_gb300 import build as _build
    _build.build()
    torch.cuda.set_device(local)
    return torch


def _calibrated_context(R, synth, torch, prob, prec, **kw):
    ctx = R.context_for(prob, prec=prec, **kw)
    c_true = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    ctx.rd_forward(prob.p_true, prob.k_f_true, prob.rho_f_true, c_true)
    d = synth.labels(c_true.cpu().numpy(), synth.ellipsoid_mask(prob.n), prob.seed + 7)
    ctx.rd_set_data(torch.from_numpy(d).cuda())
    return ctx, d


def batch_measure(R, synth, torch, steps, warmup):
    """48 independent problems of uneven size (16 each at 64^3, 96^3, 128^3,
    nt = 16, mixed), own tissue seeds, k_f ~ U(0.01, 0.1), rho_f ~ U(5, 15),
    all gradients in one CUDA-graph launch per step; the same 48 gradients
    one after another for comparison."""
    import numpy as np
    rng = np.random.default_rng(3)
    ctxs, thetas, cells = [], [], 0
    for i, n in enumerate([64] * 16 + [96] * 16 + [128] * 16):
        prob = synth.calibration_problem(n=n, nt=16, m=4, seed=3000 + i,
                                         k_f_true=float(rng.uniform(0.01, 0.1)),
                                         rho_f_true=float(rng.uniform(5, 15)))
        ctx, _ = _calibrated_context(R, synth, torch, prob, "mixed", pcg_rtol=1e-6, pcg_maxit=500)
        ctxs.append(ctx)
        thetas.append((prob.p, prob.k_f, prob.rho_f))
        cells += n ** 3 * 16
    def timed_batch():
        for _ in range(warmup):
            R.rd_batch_gradient(ctxs, thetas)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            Js, _ = R.rd_batch_gradient(ctxs, thetas)
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / steps, Js

    R.rd_autotune_clear()
    dt_fixed, _ = timed_batch()
    # tile shape and grid size per kernel class, tuned once per grid size on
    # the first instance of that size; the batch graph is captured again
    choices = {}
    for n in (64, 96, 128):
        i = [64, 96, 128].index(n) * 16
        choices[f"{n}^3"] = ctxs[i].rd_autotune(reps=3)
    ctxs = ctxs[1:] + ctxs[:1]          # another list: the next call captures a new graph
    thetas = thetas[1:] + thetas[:1]
    dt, Js = timed_batch()
    t1 = time.perf_counter()
    for c, t in zip(ctxs, thetas):
        c.rd_gradient(*t)
    torch.cuda.synchronize()
    seq = time.perf_counter() - t1
    R.rd_autotune_clear()
    del ctxs
    torch.cuda.empty_cache()
    return {"metric": "batched fwd+adjoint gradient cell-updates/s, 48 uneven instances", "value": cells / dt,
            "unit": UNIT, "steps": steps, "warmup": warmup, "ms_per_step": 1e3 * dt,
            "config": {"workload": "rd_batch_gradient: 16 x 64^3, 16 x 96^3, 16 x 128^3, nt=16, mixed, "
                                   "one graph launch per step, tile shapes and grid sizes autotuned per grid size"},
            "value_untuned": cells / dt_fixed, "autotuned": choices,
            "sequential_ms": 1e3 * seq, "batch_speedup_vs_sequential": seq / dt,
            "misfit_range": [min(Js), max(Js)]}


def run_batch(args, rank, world, local):
    """The batched workload alone (see batch_measure)."""
    torch = _gpu_setup(local)
    from paper_1907_07774_gb300 import rd as R
    from paper_1907_07774_gb300 import synth
    res = batch_measure(R, synth, torch, args.steps, args.warmup)
    line = dict(res, n_gpus=1, higher_is_better=True, dtype="f32", data="synthetic")
    print(json.dumps(line), flush=True)
    return 0


def run_newton(args, rank, world, local):
    """256^3, nt = 32, 125 Gaussians: gradient plus 20 Gauss-Newton
    Hessian-vector products (the CG of one Newton step), mixed, with the
    misfit and gradient compared to the FP64 path of the same GPU."""
    import numpy as np
    torch = _gpu_setup(local)
    from paper_1907_07774_gb300 import gn
    from paper_1907_07774_gb300 import rd as R
    from paper_1907_07774_gb300 import synth
    prob = problem(256, 32)
    ctx, d = _calibrated_context(R, synth, torch, prob, "mixed", pcg_rtol=1e-6, pcg_maxit=500)
    th = (prob.p, prob.k_f, prob.rho_f)
    ctx.rd_gradient(*th)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J, g = ctx.rd_gradient(*th)
    hv_count = [0]

    def hv(v):
        hv_count[0] += 1
        return ctx.rd_hessvec(*th, v)
    step, used = gn.cg(hv, -g, 20, 1e-12)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    ref = R.context_for(prob, prec="fp64", pcg_rtol=1e-10, pcg_maxit=1000)
    ref.rd_set_data(torch.from_numpy(d).cuda())
    J64, g64 = ref.rd_gradient(*th)
    line = {"metric": "gradient + 20 GN Hessian-vector products at 256^3 (s)", "value": dt, "unit": "s",
            "higher_is_better": False, "n_gpus": 1, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "256^3 nt=32 np=125 mixed; CG on rd_hessvec, 20 products"},
            "hessvecs": used, "misfit": J, "misfit_fp64": J64,
            "misfit_rel_err_vs_fp64": abs(J - J64) / J64,
            "grad_rel_err_vs_fp64": float(np.linalg.norm(g - g64) / np.linalg.norm(g64)),
            "newton_step_norm": float(np.linalg.norm(step))}
    print(json.dumps(line), flush=True)
    return 0


class AutogradObjective:
    """The calls the Gauss-Newton loop makes, with every misfit and gradient
    going through torch.autograd: rd_forward builds J = RDSolve.apply(p, k_f,
    rho_f, ctx) and rd_adjoint is J.backward() (the hand-written adjoint);
    Hessian-vector products go to the context."""

    def __init__(self, ctx):
        self.ctx, self.np, self.J, self.leaves = ctx, ctx.np, None, None

    def rd_forward(self, p, k_f, rho_f):
        import torch
        from paper_1907_07774_gb300 import autograd
        self.leaves = [torch.tensor(np_, dtype=torch.float64, requires_grad=True)
                       for np_ in (list(p), k_f, rho_f)]
        self.J = autograd.misfit(*self.leaves, self.ctx)
        return float(self.J.detach())

    def rd_adjoint(self):
        import numpy as np
        self.J.backward()
        pg, kg, rg = (x.grad for x in self.leaves)
        return np.concatenate([pg.numpy(), [float(kg), float(rg)]])

    def rd_gradient(self, p, k_f, rho_f):
        J = self.rd_forward(p, k_f, rho_f)
        return J, self.rd_adjoint()

    def rd_hessvec(self, p, k_f, rho_f, v):
        return self.ctx.rd_hessvec(p, k_f, rho_f, v)


def run_gn(args, rank, world, local):
    """Gauss-Newton calibration at 256^3, nt = 64, sqrt(nt) = 8 checkpoints,
    mixed, every misfit and gradient through torch.autograd.Function.  Runs
    the loop on (p, k_f, rho_f) from k_f = 0.02, rho_f = 6 as specified, and
    with rho_f held at its true value (the paper's protocol); scans the
    misfit along k_f at the true parameters to show where the thresholded
    labels put its minimum; times the FP64 path's gradient, Gauss-Newton
    product and forward solve for its time per iteration."""
    import numpy as np
    torch = _gpu_setup(local)
    from paper_1907_07774_gb300 import gn
    from paper_1907_07774_gb300 import rd as R
    from paper_1907_07774_gb300 import synth
    prob = synth.calibration_problem(n=args.n, nt=64, m=5)
    npar = len(prob.p)
    ctx, d = _calibrated_context(R, synth, torch, prob, "mixed", pcg_rtol=1e-6, pcg_maxit=500, ckpt_stride=8,
                                 beta_p=1e-4)
    obj = AutogradObjective(ctx)
    truth = np.concatenate([prob.p_true, [prob.k_f_true, prob.rho_f_true]])
    err = lambda th: {"p_rel": float(np.linalg.norm(th[:-2] - truth[:-2]) / np.linalg.norm(truth[:-2])),
                      "k_f_rel": abs(th[-2] - truth[-2]) / truth[-2], "rho_f_rel": abs(th[-1] - truth[-1]) / truth[-1],
                      "k_f": float(th[-2]), "rho_f": float(th[-1])}
    runs = {}
    for name, th0, fixed in (("joint", np.concatenate([prob.p, [prob.k_f, prob.rho_f]]), ()),
                             ("rho_fixed_at_truth", np.concatenate([prob.p, [prob.k_f, prob.rho_f_true]]),
                              (npar + 1,))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = gn.gauss_newton(obj, th0, iters=args.gn_iters, cg_maxit=20, forcing=1e-3, fixed=fixed)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        its = max(1, len(res.history))
        runs[name] = {"seconds_per_iteration": dt / its, "iterations": len(res.history),
                      "stopped": "iteration limit" if len(res.history) >= args.gn_iters else
                                 "line search found no decrease",
                      "start_error": err(th0), "final_error": err(res.theta),
                      "misfit_history": [h["misfit"] for h in res.history],
                      "hessvecs": [h["hessvecs"] for h in res.history],
                      "line_search_solves": [h["line_search"] for h in res.history]}
    scan = [(kf, ctx.rd_forward(prob.p_true, kf, prob.rho_f_true)) for kf in (0.0, 0.01, 0.025, 0.05, 0.1)]
    hv_mean = float(np.mean(runs["joint"]["hessvecs"] or [0]))
    ls_mean = float(np.mean(runs["joint"]["line_search_solves"] or [0]))
    ms_mixed = 1e3 * runs["joint"]["seconds_per_iteration"]
    del ctx, obj
    torch.cuda.empty_cache()
    # FP64 path: one gradient, one Gauss-Newton product, one forward solve
    c64 = R.context_for(prob, prec="fp64", pcg_rtol=1e-10, pcg_maxit=2000, ckpt_stride=8, beta_p=1e-4)
    c64.rd_set_data(torch.from_numpy(d).cuda())
    th = (prob.p, prob.k_f, prob.rho_f)
    v = synth.random_directions(1, npar + 2, 5)[0]

    def t(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    t_g = t(lambda: c64.rd_gradient(*th))
    t_h = t(lambda: c64.rd_hessvec(*th, v))
    t_f = t(lambda: c64.rd_forward(*th))
    t_it64 = t_g + hv_mean * t_h + ls_mean * t_f
    line = {"metric": "Gauss-Newton iteration time at 256^3 nt=64 (s)", "value": ms_mixed / 1e3,
            "unit": "s/iteration", "higher_is_better": False, "n_gpus": 1, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.n}^3 nt=64 np=125 mixed ckpt_stride=8 beta_p=1e-4, "
                                   f"{args.gn_iters} GN iterations, CG to 1e-3 with <= 20 Hessian-vector products on "
                                   f"the parameter-scaled system, Armijo backtracking; misfit and gradient through "
                                   f"torch.autograd.Function (RDSolve)"},
            "runs": runs,
            "misfit_along_k_f_at_truth": {"k_f": [x[0] for x in scan], "misfit": [x[1] for x in scan],
                                          "note": "thresholded labels with 1% flips; truth k_f = 0.05"},
            "fp64": {"gradient_s": t_g, "hessvec_s": t_h, "forward_s": t_f,
                     "seconds_per_iteration_extrapolated": t_it64,
                     "note": "FP64 iteration = gradient + mean Hessian-vector products + mean line-search solves "
                             "of the mixed joint run, each timed once on the FP64 path",
                     "mixed_speedup_per_iteration": t_it64 / (ms_mixed / 1e3)}}
    print(json.dumps(line), flush=True)
    return 0


def run_picard(args, rank, world, local):
    """The tumor side of one Picard step at 256^3, nt = 32 (mixed): the
    Moving-Atlas gradient (D_c + D_m, anatomy final condition) with the
    coupling field q(x) accumulated during the adjoint and read back to the
    device, timed next to the plain gradient on the same problem."""
    import numpy as np
    torch = _gpu_setup(local)
    from paper_1907_07774_gb300 import rd as R
    from paper_1907_07774_gb300 import synth
    prob = problem(args.n, args.nt)
    plain, d = _calibrated_context(R, synth, torch, prob, "mixed", pcg_rtol=1e-6, pcg_maxit=500)
    ma = R.context_for(prob, prec="mixed", pcg_rtol=1e-6, pcg_maxit=500, moving_atlas=True, coupling=True)
    ma.rd_set_data(torch.from_numpy(d).cuda())
    rng = np.random.default_rng(prob.seed + 11)
    md = [np.clip(m + 0.05 * rng.standard_normal(prob.n), 0, 1) * (m > 0)
          for m in (prob.m_wm, prob.m_gm, prob.m_csf)]
    ma.rd_set_anatomy_data(*[torch.from_numpy(x).cuda() for x in md])
    q = [torch.empty(prob.n, dtype=torch.float64, device="cuda") for _ in range(3)]
    th = (prob.p, prob.k_f, prob.rho_f)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / args.steps

    def ma_step():
        ma.rd_gradient(*th)
        ma.rd_coupling_field(*q)

    t_ma = timed(ma_step)
    t_plain = timed(lambda: plain.rd_gradient(*th))
    cells = args.n ** 3 * args.nt
    J, g = ma.rd_gradient(*th)
    line = {"metric": "Moving-Atlas gradient + coupling field cell-updates/s at 256^3", "value": cells / t_ma,
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_ma,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.n}^3 nt={args.nt} np=125 mixed, D_c + D_m objective, q(x) to device"},
            "plain_gradient_ms": 1e3 * t_plain, "overhead_vs_plain": t_ma / t_plain - 1.0,
            "misfit": J, "q_abs_max": [float(x.abs().max()) for x in q]}
    print(json.dumps(line), flush=True)
    return 0


def run_tumor_inv(args, rank, world, local):
    """The paper's tumor optimiser (l1 GIST with the Hoyer beta search, then
    weighted-l2 L-BFGS on (p, k_f)) at 128^3, nt = 16, 4^3 Gaussians, mixed;
    reports wall time and solver counts."""
    import numpy as np
    torch = _gpu_setup(local)
    from paper_1907_07774_gb300 import rd as R
    from paper_1907_07774_gb300 import synth
    from paper_1907_07774_gb300 import tumor_inv as T
    prob = synth.calibration_problem(n=128, nt=16, m=4, sigma=2 * np.pi / 32)
    ctx, _ = _calibrated_context(R, synth, torch, prob, "mixed", pcg_rtol=1e-6, pcg_maxit=500)
    t0 = time.perf_counter()
    out = T.tumor_inversion(ctx, rho_f=prob.rho_f_true, k_f_l2=0.02, beta_steps=5,
                            gist_kw={"maxit": 30, "tau_j": 1e-5}, beta_l2=1e-4, opttol=1e-3, l2_maxit=25)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    evals = sum(t["iters"] for t in out.l1.tried)
    line = {"metric": "tumor inversion (l1 GIST + Hoyer beta search, weighted-l2 L-BFGS) wall time at 128^3 (s)",
            "value": dt, "unit": "s", "higher_is_better": False, "n_gpus": 1, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "128^3 nt=16 np=64 mixed, 5 beta bisection steps (GIST <= 30 iterations), "
                                   "L-BFGS <= 25 iterations on (p, k_f)"},
            "gist_iterations": evals, "lbfgs_iterations": out.l2.iters, "lbfgs_evaluations": out.l2.evals,
            "beta_l1": out.beta_l1, "sparsity": out.sparsity, "nnz_l1": int(np.count_nonzero(out.l1.p)),
            "misfit_final": out.misfit, "k_f_final": out.k_f}
    print(json.dumps(line), flush=True)
    return 0


def run_registration(args, rank, world, local):
    """The registration sub-problem of the Picard step at 128^3, nt = 8
    (mixed): reduced gradient and Gauss-Newton Hessian-vector product
    through the C ABI, and three Gauss-Newton-Krylov iterations from v = 0
    (PCG with at most 5 products, Armijo)."""
    import numpy as np
    torch = _gpu_setup(local)
    from paper_1907_07774_gb300 import reg_gn
    from paper_1907_07774_gb300 import rg as RG
    from paper_1907_07774_gb300 import synth
    n, nt = 128, 8
    prob = synth.registration_problem(n=n, nt=nt, seed=4700, ndir=1)
    ctx = RG.context_for(prob, "mixed")
    dev = lambda xs: [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in xs]
    v, vt = dev(prob.v), dev(prob.directions[0])
    g = [torch.empty(prob.n, dtype=torch.float64, device="cuda") for _ in range(3)]
    hv = [torch.empty(prob.n, dtype=torch.float64, device="cuda") for _ in range(3)]

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / args.steps

    t_g = timed(lambda: ctx.rg_gradient(v, g))
    t_h = timed(lambda: ctx.rg_hessvec(v, vt, hv))
    ref = RG.context_for(prob, "fp64")
    J64, g64 = ref.rg_gradient(prob.v)
    J32, g32 = ctx.rg_gradient(prob.v)
    num = math.sqrt(sum(float(np.sum((a - b) ** 2)) for a, b in zip(g32, g64)))
    den = math.sqrt(sum(float(np.sum(b * b)) for b in g64))
    h3 = (2 * math.pi) ** 3 / n ** 3
    zero = [np.zeros(prob.n) for _ in range(3)]
    J0 = ctx.rg_forward(zero)
    t0 = time.perf_counter()
    res = reg_gn.gauss_newton(ctx, zero, h3, iters=3, cg_maxit=5)
    t_gn = time.perf_counter() - t0
    cells = n ** 3 * nt
    line = {"metric": "registration reduced-gradient cell-updates/s at 128^3 (semi-Lagrangian state + adjoint)",
            "value": cells / t_g, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_g, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"rg_gradient {n}^3 nt={nt} mixed (FP32 fields, FP64 reductions), "
                                   "smooth synthetic anatomy, patient = atlas under a divergence-free displacement"},
            "hessvec_ms": 1e3 * t_h, "grad_rel_err_vs_fp64": num / den, "misfit_rel_err_vs_fp64": abs(J32 - J64) / J64,
            "gn_seconds": t_gn, "gn_objective": [J0] + [h["objective"] for h in res.history],
            "gn_hessvecs": [h["hessvecs"] for h in res.history]}
    print(json.dumps(line), flush=True)
    return 0


def run_picard_loop(args, rank, world, local):
    """The Moving-Atlas Picard iteration at 64^3 (tumor nt = 16, mixed;
    registration nt = 4, mixed): beta_v 1e-1 -> 1e-2 with two final
    iterations, two tumor Gauss-Newton and two registration Gauss-Newton
    iterations per Picard step; the patient is the atlas under a
    divergence-free displacement with a tumor grown in the patient anatomy."""
    import numpy as np
    torch = _gpu_setup(local)
    from paper_1907_07774_gb300 import picard as P
    from paper_1907_07774_gb300 import rd as R
    from paper_1907_07774_gb300 import rg as RG
    from paper_1907_07774_gb300 import synth
    n, nt = (64, 64, 64), 16
    prob = synth.registration_problem(n=n, nt=4, seed=4900, disp_amp=0.25, q_amp=0.0, ndir=0)
    atlas, healthy = prob.m_atlas, prob.m_patient
    sigma = 2 * math.pi / 32
    centers = synth.lattice_centers(4, 1.5 * sigma)
    p_true = synth.two_site_truth(4)
    gen = R.Context(n, nt, len(p_true), prec="fp64")
    gen.rd_set_tissue(*healthy)
    gen.rd_set_basis(centers, sigma)
    c_true = np.zeros(n)
    gen.rd_forward(p_true, 0.05, 10.0, c_true)
    d = synth.labels(c_true, synth.ellipsoid_mask(n), 7)
    m_P = [m * (1.0 - c_true) for m in healthy]
    tumor = R.Context(n, nt, len(p_true), prec="mixed", pcg_rtol=1e-6, moving_atlas=True, coupling=True)
    tumor.rd_set_tissue(*atlas)
    tumor.rd_set_basis(centers, sigma)
    tumor.rd_set_data(d)
    tumor.rd_set_anatomy_data(*m_P)
    theta0 = np.concatenate([0.1 * p_true + 0.05, [0.02, 6.0]])
    make_reg = lambda beta: RG.RegContext(n, 4, prec="mixed", beta_v=beta)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = P.picard(tumor, make_reg, atlas, m_P, theta0, beta_init=1e-1, beta_final=1e-2, final_repeats=2,
                   tumor_iters=2, reg_iters=2)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    line = {"metric": "Moving-Atlas Picard iteration time at 64^3 (s per Picard step)",
            "value": dt / len(res.history), "unit": "s/iteration", "higher_is_better": False, "n_gpus": 1,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "64^3, tumor nt=16 (mixed, 64 Gaussians), registration nt=4 (mixed), "
                                   "beta_v 1e-1 -> 1e-2 (+1), 2 tumor GN + 2 registration GN iterations per step"},
            "history": res.history, "k_f": float(res.theta[-2]), "rho_f": float(res.theta[-1])}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--nt", type=int, default=32)
    ap.add_argument("--ckpt-stride", type=int, default=0)
    ap.add_argument("--guess-restart", type=int, default=None,
                    help="restart period of the state solves' extrapolated guesses (-1: off; default: the library's)")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the checkpointed gradient and the batched workload of the main line")
    ap.add_argument("--no-cpu-full", action="store_true",
                    help="skip the complete 64^3 oracle gradients of the CPU baseline")
    ap.add_argument("--workload", default="gradient",
                    choices=["gradient", "batch", "newton", "gn", "picard", "tumor_inv", "registration",
                             "picard_loop"],
                    help="gradient: the headline 256^3 gradient; batch: 48 uneven instances in one graph; "
                         "newton: gradient + 20 Hessian-vector products; gn: Gauss-Newton calibration; "
                         "picard: Moving-Atlas gradient + coupling field; tumor_inv: l1/l2 tumor optimiser; "
                         "registration: the registration sub-problem (gradient, GN product, GN iterations); "
                         "picard_loop: the Moving-Atlas Picard iteration")
    ap.add_argument("--gn-iters", type=int, default=10)
    ap.add_argument("--autotune", action="store_true", help="tune grid sizes per kernel class first")
    args = ap.parse_args()
    rank, world, local = env_rank()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "batch":
        return run_batch(args, rank, world, local)
    if args.workload == "newton":
        return run_newton(args, rank, world, local)
    if args.workload == "gn":
        return run_gn(args, rank, world, local)
    if args.workload == "picard":
        return run_picard(args, rank, world, local)
    if args.workload == "tumor_inv":
        return run_tumor_inv(args, rank, world, local)
    if args.workload == "registration":
        return run_registration(args, rank, world, local)
    if args.workload == "picard_loop":
        return run_picard_loop(args, rank, world, local)
    return run_ours(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
