#!/usr/bin/env python3
"""Benchmark of the lattice Basic Scheme (Algorithm 1, arXiv 1605.05712) on GB300.

Workload (one "step"): the 2-D two-phase laminate (normal (1,3)/sqrt(10),
volume fraction 1/2, isotropic phases (lam, mu) = (1,1) and (10,10), plane
strain, C0 = mean of the phase extremes) on three lattices of m = 262,144
points -- the tensor grid diag(512,512), the rank-1 lattice [[512,1],[0,512]]
and the sheared rank-2 lattice [[512,16],[0,512]] -- with the three unit
load cases solved one after another to a Cauchy residual of 1e-8, binary64
throughout.  Metric: lattice-point iterations per second
(sum over lattices and load cases of m x iterations / step time).

Legs: device-timed steps with inputs resident in HBM (value), the same through
the C ABI with the phase field copied host->device and the strain field
copied back every step (e2e), per-kernel CUDA-event timing of one iteration
(roofline), and the CPU oracle on a bounded sample (cpu_baseline).
``--impl reference`` times the oracle alone.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

LATS = ["grid512", "rank1_262144", "rank2_262144"]
WORKLOAD = ("2-D laminate n=(1,3), m=262144 on diag(512,512), rank-1 [[512,1],[0,512]] and rank-2 "
            "[[512,16],[0,512]]; 3 unit load cases solved separately; tol 1e-8; FP64")
LAMES = [(1.0, 1.0), (10.0, 10.0)]
N_INT = [1, 3]
TOL = 1e-8
MAXIT = 2000
METRIC = "lattice-point iterations/s"
FP64_PEAK_TFLOPS = 1.25
L2_FLUSH_BYTES = 512 << 20


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def load_cases(n_c=3):
    E = np.zeros((n_c, n_c))
    for a in range(n_c):
        E[a, a] = 1.0 if a < 2 else 0.5     # unit load cases, tensor components (eps_12 = 1/2)
    return E


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, idx):
        self.f = tempfile.NamedTemporaryFile(prefix="clk", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(idx), "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        rows = [l.split(",") for l in open(self.f.name).read().strip().splitlines() if l.strip()]
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for i, nm in enumerate(names):
                if len(r) > 5 + i and "Active" in r[5 + i] and "Not" not in r[5 + i]:
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def row_col_flops(P, n_c=3):
    """Algorithmic flops of one iteration split by kernel (5 N log2 N per complex FFT of N points)."""
    import math
    m, Rh = P["m"], P["Rh"]
    # row pass: inverse + forward half-length complex FFT of every row and component, R2C pre/post
    # processing (~10 flops per complex point each way), polarization (n_c^2 FMA), residual (3 n_c)
    row = n_c * (2 * 5 * (m // 2) * math.log2(Rh) + 2 * 10 * (m // 2)) + m * (2 * n_c * n_c + 3 * n_c)
    col = []
    for G in P["groups"]:
        f = n_c * 2 * 5 * (m // 2 + m // P["R"]) * math.log2(G)
        col.append(f)
    col[0] += (m // 2 + m // P["R"]) * 2 * 45       # Green operator, ~45 flops per real part
    return row, col


def algorithmic_bytes(P, n_c=3, s=8):
    """HBM bytes of one iteration by kernel: row pass reads T + eps + phase, writes eps + T;
    a column pass reads and writes T (half spectrum + Nyquist plane)."""
    m = P["m"]
    spec = n_c * (m // 2 + m // P["R"]) * 2 * s
    row = spec + n_c * m * s + m + n_c * m * s + spec
    col = [2 * spec for _ in P["groups"]]
    return row, col


def setup(dev):
    import torch
    from paper_1605_05712_gb300 import lattice_plan, synth
    out = []
    for name in LATS:
        P = lattice_plan(synth.LATTICES[name])
        ph = synth.laminate_phase(P.points(), P.m, N_INT)
        out.append(dict(name=name, plan=P, phase_host=torch.from_numpy(ph).pin_memory(),
                        phase=torch.from_numpy(ph).to(dev)))
    return out


PLAIN_LAUNCHES = False   # --plain-launches: iterate with plain launches instead of the CUDA-graph loop


C0_EM = (np.sqrt(1.0 * 10.0), np.sqrt(1.0 * 10.0))   # geometric mean of the laminate's extremes


def run_step(work, stiff, C0, E, ws, eps, mode="fp64_separate", tol=TOL):
    """One pass of the workload.  fp64_separate: each load case its own solve (the configured
    form); *_batched: the three load cases of a lattice in one batched solve; df64 = the binary64-accurate
    double-float kernels."""
    from paper_1605_05712_gb300 import basic_scheme_solve
    tot = 0
    iters = []
    for w in work:
        prec = mode.split("_")[0]                       # fp64, df64 or mixed
        em = mode.endswith("_em")                       # Eyre-Milton at the geometric-mean reference
        if mode.endswith("_cg"):                        # conjugate gradients (boundary frequencies zeroed)
            g = basic_scheme_solve(w["plan"], w["phase"], stiff, C0, E, tol=tol, maxit=MAXIT, workspace=ws,
                                   eps_out=eps, precision=prec, plain_launches=PLAIN_LAUNCHES, scheme="cg",
                                   boundary="zero")
            its = [int(x) for x in g["iters"]]
        elif em:
            g = basic_scheme_solve(w["plan"], w["phase"], stiff, C0_EM, E, tol=tol, maxit=MAXIT, workspace=ws,
                                   eps_out=eps, precision=prec, plain_launches=PLAIN_LAUNCHES, scheme="eyre_milton")
            its = [int(x) for x in g["iters"]]
        elif mode.endswith("_separate"):
            its = []
            for lc in range(E.shape[0]):
                g = basic_scheme_solve(w["plan"], w["phase"], stiff, C0, E[lc:lc + 1], tol=tol, maxit=MAXIT,
                                       workspace=ws, eps_out=eps[lc:lc + 1], precision=prec,
                                       plain_launches=PLAIN_LAUNCHES)
                its.append(int(g["iters"][0]))
        else:
            g = basic_scheme_solve(w["plan"], w["phase"], stiff, C0, E, tol=tol, maxit=MAXIT, workspace=ws,
                                   eps_out=eps, precision=prec, plain_launches=PLAIN_LAUNCHES)
            its = [int(x) for x in g["iters"]]
        iters.append(its)
        tot += w["plan"].m * int(np.sum(its))
    return tot, iters


def timed(fn, steps, flush, st):
    import torch
    times, units, last = [], 0, None
    for _ in range(steps):
        flush.fill_(1)                                   # L2 flush between timed steps (not timed)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        u, last = fn()
        e1.record(st)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        units += u
    return float(np.mean(times)), units / steps, last


def kernel_sha():
    import hashlib
    h = hashlib.sha1()
    for f in ("kernels.cu", "fft_smem.cuh", "kernels.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1605_05712_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:12]


def profiled_traffic(kernel_tag):
    """DRAM bytes per launch of a kernel from the committed ncu summary, if it was taken on the
    current kernel sources (sha recorded in the summary); else None."""
    import glob
    for f in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        txt = open(f).read()
        if "kernel_tag: " + kernel_tag not in txt:
            continue
        sha = tr = None
        for line in txt.splitlines():
            if line.startswith("kernel_sources_sha: "):
                sha = line.split(": ", 1)[1].strip()
            if line.startswith("dram_bytes_per_launch: "):
                tr = float(line.split(": ", 1)[1])
        if sha == kernel_sha() and tr is not None:
            return tr
    return None


def aggregate_ranks(ms_list, units_list, world, device):
    """Replicas: every rank ran the same workload on its own GPU.  The job's time is the slowest rank's
    (all-reduce MAX of each time), its throughput all ranks' units over that time.  Returns
    (times_ms, values)."""
    import torch
    import torch.distributed as dist
    ms = [float(x) for x in ms_list]
    if world > 1:
        t = torch.tensor(ms, dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = [float(x) for x in t.tolist()]
    return ms, [world * u / (m / 1e3) for u, m in zip(units_list, ms)]


def bench_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_1605_05712_gb300 import lattice_pass_times, synth
    from paper_1605_05712_gb300.api import LAT_WS_CG
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stiff = [synth.iso_voigt(*l) for l in LAMES]
    C0 = synth.c0_mean_extremes([l[0] for l in LAMES], [l[1] for l in LAMES])
    E = load_cases()
    work = setup(dev)
    m = work[0]["plan"].m
    ws = torch.empty(max(w["plan"].workspace_bytes(3, p) for w in work for p in (0, 1, 2, 0 | LAT_WS_CG, 2 | LAT_WS_CG)),
                     dtype=torch.uint8, device=dev)
    eps = torch.empty((3, 3, m), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream()

    for _ in range(args.warmup):
        run_step(work, stiff, C0, E, ws, eps)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = Clocks(local)
    ms_step, units, iters = timed(lambda: run_step(work, stiff, C0, E, ws, eps), args.steps, flush, st)
    # end-to-end: host phase -> device, solves, strain -> host, every step
    eps_host = torch.empty((3, 3, m), dtype=torch.float64).pin_memory()

    def e2e_step():
        for w in work:
            w["phase"].copy_(w["phase_host"], non_blocking=True)
        u, it = run_step(work, stiff, C0, E, ws, eps)
        eps_host.copy_(eps, non_blocking=True)
        return u, it
    ms_e2e, e2e_units, _ = timed(e2e_step, args.steps, flush, st)
    clocks = clk.stop()
    (ms_step, ms_e2e), (value, e2e_value) = aggregate_ranks([ms_step, ms_e2e], [units, e2e_units], world, dev)

    # variants on the same inputs: batched load cases (binary64, mixed) and time to a 1e-6 residual
    variants = {}
    if not args.no_variants:
        for mode in ("df64_separate", "fp64_batched", "df64_batched", "mixed_batched"):
            run_step(work, stiff, C0, E, ws, eps, mode)
            ms_v, u_v, it_v = timed(lambda: run_step(work, stiff, C0, E, ws, eps, mode), args.steps, flush, st)
            variants[mode] = {"value": round(u_v / (ms_v / 1e3), 1), "ms_per_step": round(ms_v, 4), "iterations": it_v}
        ttt = {}
        for mode in ("fp64_separate", "fp64_batched", "df64_batched", "mixed_batched", "fp64_batched_em",
                     "mixed_batched_em", "fp64_batched_cg", "df64_batched_cg"):
            run_step(work, stiff, C0, E, ws, eps, mode, tol=1e-6)
            ms_v, _, it_v = timed(lambda: run_step(work, stiff, C0, E, ws, eps, mode, tol=1e-6), args.steps, flush, st)
            ttt[mode] = {"ms": round(ms_v, 4), "iterations": it_v}
        variants["time_to_resid_1e-6_ms"] = ttt

    # per-kernel timing of one iteration on the rank-2 lattice (dominant kernel -> roofline)
    w = work[2]
    P = w["plan"]
    pt = lattice_pass_times(P, w["phase"], stiff, C0, E[0], n_reps=50)
    pt_df = lattice_pass_times(P, w["phase"], stiff, C0, E[0], precision="df64", n_reps=50)
    model = {"m": P.m, "R": 512, "Rh": 256, "groups": [512]}   # the planner's decomposition of all three lattices
    bytes_row, bytes_col = algorithmic_bytes(model)
    flops_row, flops_col = row_col_flops(model)
    dom = int(np.argmax(pt[:2]))
    ms_dom = pt[dom]
    pk = peaks()
    fl, by = (flops_row, bytes_row) if dom == 0 else (flops_col[0], bytes_col[0])
    tag = ("row_pass" if dom == 0 else "col_pass") + "<double,3>/rank2_262144"
    fp64_peak = FP64_PEAK_TFLOPS
    roof = {"bound": "alu", "achieved": round(fl / (ms_dom * 1e-3) / 1e12, 4), "peak": fp64_peak,
            "unit": "TFLOP/s", "frac": round(fl / (ms_dom * 1e-3) / 1e12 / fp64_peak, 4),
            "traffic": profiled_traffic(tag), "kernel": tag,
            "peak_source": "nominal GB300 binary64 rate 1.25 TFLOP/s (no FP64 entry in the measured peaks; an "
                           "FMA-loop probe measured 1.19)",
            "algorithmic_flops_per_launch": fl, "algorithmic_bytes_per_launch": by,
            "hbm_achieved_gbs": round(by / (ms_dom * 1e-3) / 1e9, 1),
            "hbm_peak_gbs": pk.get("hbm_gbs"), "per_kernel_ms": [round(x, 5) for x in pt],
            "df64_per_kernel_ms": [round(x, 5) for x in pt_df],
            "df64_achieved_fp64_equiv_tflops": round(fl / (pt_df[dom] * 1e-3) / 1e12, 4)}
    gpu_launches = 0
    for it in iters:
        for n in it:   # per solve: fill, prologue (row + column), n loop iterations, effective stress
            gpu_launches += 1 + 2 + 2 * n + 1
    res = {
        "metric": METRIC, "value": round(value, 1), "unit": "point-iterations/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded laminate phases generated on the host)",
        "config": {"workload": WORKLOAD, "lattices": LATS, "load_cases": 3, "tol": TOL, "iterations": iters,
                   "l2": "flushed (512 MiB write) between timed steps", "parallelism": "replicas" if world > 1 else "1 GPU",
                   "launch": "plain launches, host convergence check per iteration" if PLAIN_LAUNCHES
                             else "one CUDA-graph WHILE loop per solve"},
        "roofline": roof,
        "e2e": {"value": round(e2e_value, 1), "unit": "point-iterations/s",
                "h2d_bytes_per_step": int(sum(w_["plan"].m for w_ in work)),
                "d2h_bytes_per_step": int(eps.numel() * 8)},
        "gpu_launches": gpu_launches,
        "clocks": clocks,
        "variants": variants,
    }
    if rank == 0 and world == 1 and not args.no_cpu:
        res["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(res))


def bench_hashin(args):
    """Config-3 workload: the coated-ellipsoid (generalized Hashin) structure at m = 2^21 on the tensor grid,
    the rank-1 and the sheared 3-D lattices; six unit load cases batched in one solve, tol 1e-6, mixed
    precision (binary32 FFT/Gamma0/polarization, binary64 residual, averages and strain), timed against
    the plain binary64 form on the same inputs; C^eff eps0 against the analytic value."""
    import torch
    from paper_1605_05712_gb300 import basic_scheme_solve, lattice_plan, synth
    from paper_1605_05712_gb300.api import LAT_WS_CG
    dev = torch.device("cuda", 0)
    w = synth.hashin_workload()
    E = np.eye(6)
    E[3:, 3:] *= 0.5
    e0 = np.array([w["eps0"][0, 0], w["eps0"][1, 1], w["eps0"][2, 2], 2 * w["eps0"][1, 2], 2 * w["eps0"][0, 2],
                   2 * w["eps0"][0, 1]])
    ce_ref = np.array([w["ceff_eps0"][0, 0], w["ceff_eps0"][1, 1], w["ceff_eps0"][2, 2], w["ceff_eps0"][1, 2],
                       w["ceff_eps0"][0, 2], w["ceff_eps0"][0, 1]])
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream()
    out = {}
    for name in ("grid128", "rank1_2097152", "sheared128"):
        P = lattice_plan(synth.LATTICES[name])
        ph = torch.from_numpy(synth.coated_ellipsoid_phase(P.points(), P.m, w["c"], w["rho_c"], w["rho_e"],
                                                            R=w["R"])).to(dev)
        eps = torch.empty((6, 6, P.m), dtype=torch.float64, device=dev)
        res = {}
        # forms: Algorithm 1 in each precision; the accelerated schemes (Eyre-Milton at the geometric mean
        # of the core and coating moduli, conjugate gradients with the boundary frequencies zeroed)
        g_mean = float(np.sqrt(10.0 * 1.0))
        forms = {"mixed": ("mixed", w["C0"], {}), "df64": ("df64", w["C0"], {}), "fp64": ("fp64", w["C0"], {}),
                 "eyre_milton_mixed": ("mixed", (g_mean, g_mean), {"scheme": "eyre_milton"}),
                 "cg_df64": ("df64", w["C0"], {"scheme": "cg", "boundary": "zero"})}
        for form, (prec, C0f, kw) in forms.items():
            flag = LAT_WS_CG if kw.get("scheme") == "cg" else 0
            ws = torch.empty(P.workspace_bytes(6, {"fp64": 0, "mixed": 1, "df64": 2}[prec] | flag),
                             dtype=torch.uint8, device=dev)
            run = lambda: basic_scheme_solve(P, ph, w["stiffness"], C0f, E, tol=1e-6, maxit=2000,
                                             precision=prec, workspace=ws, eps_out=eps, **kw)
            for _ in range(args.warmup if prec == "mixed" else 1):
                g = run()
            steps = args.steps if form == "mixed" else 1
            last = {}

            def step():
                g = run()
                last["g"] = g
                return P.m * int(np.sum(g["iters"])), None
            ms, units, _ = timed(step, steps, flush, st)
            g = last["g"]
            ce = (g["sigma_bar"].T @ e0)
            res[form] = {"ms": round(ms, 3), "value": round(units / (ms / 1e3), 1),
                         "iterations": [int(x) for x in g["iters"]],
                         "ceff_eps0_rel_err_vs_analytic": float(np.linalg.norm(ce - ce_ref) / np.linalg.norm(ce_ref)),
                         "sigma_bar": g["sigma_bar"].tolist()}
            del ws
        sb_d = np.array(res["fp64"]["sigma_bar"])
        for form in ("mixed", "df64", "eyre_milton_mixed", "cg_df64"):
            res[form + "_vs_fp64_ceff_rel"] = float(np.abs(np.array(res[form]["sigma_bar"]) - sb_d).max()
                                                    / np.abs(sb_d).max())
        for form in forms:
            res[form].pop("sigma_bar")
        out[name] = res
    print(json.dumps({"workload": "hashin3d (config 3): coated ellipsoid c=(0.1,0.15,0.2), fraction 0.25, "
                                  "core/coating/matrix 10/1/1+rank-one, m=2^21, 6 load cases batched, tol 1e-6",
                      "metric": METRIC, "unit": "point-iterations/s", "results": out}))


def bench_warmstart(args):
    """Learned warm start: train the network on the GPU (own kernels) on plain-scheme solutions of random
    ellipsoidal-inclusion microstructures at 64^3 (contrast 10^U(-1,2)), evaluate on held-out seeds at
    128^3: iterations and wall time to a 1e-6 residual for the six unit load cases batched, from the cold
    start, the raw prediction, and both after the two-iteration start filter, in binary64 and in mixed
    precision; every result checked against the plain binary64 cold start (effective stress)."""
    import torch
    from paper_1605_05712_gb300 import basic_scheme_solve, lattice_plan
    from paper_1605_05712_gb300.warmstart import (UNIT_E, WarmStartNet, feature_table, random_microstructure,
                                                  solve_filtered, solve_warm, train)
    dev = torch.device("cuda", 0)
    net = WarmStartNet(dev, seed=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = train(net, args.ws_train_n, args.ws_samples, 2, 3e-4, seed0=5000)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    n = args.ws_eval_n
    P = lattice_plan(np.diag([n, n, n]).tolist())
    E = UNIT_E
    names = ["cold", "warm", "cold_filtered", "warm_filtered"]
    tot = {prec: {k: {"iters": 0, "s": 0.0} for k in names} for prec in ("fp64", "mixed")}
    per_seed, worst_sb = [], 0.0
    for s in range(args.ws_eval):
        ph, stiff, C0 = random_microstructure(900000 + s, n, dev)
        ref = None
        row = {"contrast": float(stiff[1][0, 0] / 3)}
        for prec in ("fp64", "mixed"):
            fns = {"cold": lambda: basic_scheme_solve(P, ph, stiff, C0, E, tol=1e-6, maxit=5000, precision=prec),
                   "warm": lambda: solve_warm(P, net, ph, stiff, C0, E, n, tol=1e-6, precision=prec, filtered=False),
                   "cold_filtered": lambda: solve_filtered(P, ph, stiff, C0, E, tol=1e-6, precision=prec),
                   "warm_filtered": lambda: solve_warm(P, net, ph, stiff, C0, E, n, tol=1e-6, precision=prec)}
            for k in names:
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                r = fns[k]()
                torch.cuda.synchronize()
                dt = time.perf_counter() - t1
                it = int(np.sum(r["iters"]))
                tot[prec][k]["iters"] += it
                tot[prec][k]["s"] += dt
                row["%s_%s" % (prec, k)] = it
                if ref is None:
                    ref = r["sigma_bar"]
                worst_sb = max(worst_sb, float(np.abs(r["sigma_bar"] - ref).max() / np.abs(ref).max()))
        tab = torch.from_numpy(feature_table(stiff, C0[1]).reshape(-1)).to(dev)
        eps0 = net.predict(ph, tab, n, E)
        cold = basic_scheme_solve(P, ph, stiff, C0, E, tol=1e-6, maxit=5000)
        Eb = torch.from_numpy(E).to(dev)[:, :, None]
        row["pred_err2"] = round(float(((eps0 - cold["eps"]) ** 2).sum() / ((cold["eps"] - Eb) ** 2).sum()), 4)
        per_seed.append(row)
    for prec in tot:
        for k in names:
            tot[prec][k]["s"] = round(tot[prec][k]["s"], 3)
    print(json.dumps({"workload": "warmstart (config 5): train %d samples x 2 Adam steps at %d^3, evaluate %d "
                                  "held-out seeds at %d^3, 6 unit load cases batched, tol 1e-6"
                                  % (args.ws_samples, args.ws_train_n, args.ws_eval, n),
                      "train_s": round(t_train, 1), "train_loss_first_last": [float(np.mean(losses[:100])),
                                                                               float(np.mean(losses[-100:]))],
                      "totals": tot, "max_sigma_bar_rel_diff_vs_fp64_cold": worst_sb, "per_seed": per_seed}))


def bench_sweep(args):
    """Uneven serving sweep: 256 seeded independent problems (2-D and 3-D, m = 2^12 .. 2^21, rank-1 /
    rank-2 / diagonal lattices, 1-8 inclusions, contrast 1e-2 .. 1e2, all unit load cases), mixed
    precision to a 1e-6 residual in one basic_scheme_solve_multi call (one CUDA graph, a WHILE loop per
    lattice), against the same problems solved one call each; sampled problems checked against binary64."""
    import torch
    from paper_1605_05712_gb300 import (basic_scheme_solve, basic_scheme_solve_multi, lattice_plan,
                                        multi_workspace_bytes, synth)
    dev = torch.device("cuda", 0)
    t0 = time.perf_counter()
    sweep = synth.serving_sweep()
    probs = []
    for s_ in sweep:
        P = lattice_plan(s_["M"])
        ph = torch.from_numpy(synth.inclusions_phase(P.points(), P.m, s_["incl"])).to(dev)
        probs.append(dict(plan=P, phase=ph, stiffness=s_["stiffness"], C0=s_["C0"], E=s_["E"],
                          eps=torch.empty((len(s_["E"]), P.n_c, P.m), dtype=torch.float64, device=dev)))
    t_setup = time.perf_counter() - t0
    ws = torch.empty(max(multi_workspace_bytes(probs, "mixed"), multi_workspace_bytes(probs, "df64", scheme="cg")),
                     dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    res = {}

    def run_multi():
        return basic_scheme_solve_multi(probs, tol=1e-6, maxit=5000, precision="mixed", workspace=ws)

    def run_each():
        out = []
        for p_ in probs:
            out.append(basic_scheme_solve(p_["plan"], p_["phase"], p_["stiffness"], p_["C0"], p_["E"], tol=1e-6,
                                          maxit=5000, precision="mixed", eps_out=p_["eps"]))
        return out
    probs_em = [dict(p_, C0=(np.sqrt(s_["stiffness"][0][0, 1] * s_["stiffness"][1][0, 1]),) * 2)
                for p_, s_ in zip(probs, sweep)]

    def run_multi_em():
        return basic_scheme_solve_multi(probs_em, tol=1e-6, maxit=5000, precision="mixed", workspace=ws,
                                        scheme="eyre_milton")

    def run_multi_cg():
        return basic_scheme_solve_multi(probs, tol=1e-6, maxit=5000, precision="df64", workspace=ws, scheme="cg",
                                        boundary="zero")

    for name, fn in (("multi", run_multi), ("one_call_each", run_each), ("multi_eyre_milton", run_multi_em),
                     ("multi_cg_df64", run_multi_cg)):
        fn()
        times = []
        for _ in range(max(1, args.steps)):
            flush.fill_(1)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            out = fn()
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t1)
        outs = out[1] if name.startswith("multi") else out
        pit = sum(p_["plan"].m * int(np.sum(o["iters"])) for p_, o in zip(probs, outs))
        its = np.concatenate([np.asarray(o["iters"]) for o in outs])
        res[name] = {"s": round(float(np.median(times)), 3), "point_iterations": pit,
                     "value": round(pit / float(np.median(times)), 1),
                     "iterations_min_median_max": [int(its.min()), int(np.median(its)), int(its.max())]}
    # check a sample against binary64: extremes of contrast and the largest problems
    order = np.argsort([s_["contrast"] for s_ in sweep])
    sizes = np.argsort([s_["m"] for s_ in sweep])
    pick = sorted(set(list(order[:2]) + list(order[-2:]) + list(sizes[-2:])))
    _, outs = run_multi()
    worst = {"strain": 0.0, "sigma_bar": 0.0}
    for i in pick:
        p_, o = probs[i], outs[i]
        ref = basic_scheme_solve(p_["plan"], p_["phase"], p_["stiffness"], p_["C0"], p_["E"], tol=1e-6, maxit=5000)
        worst["strain"] = max(worst["strain"], float((o["eps"] - ref["eps"]).abs().max() / ref["eps"].abs().max()))
        worst["sigma_bar"] = max(worst["sigma_bar"], float(np.abs(o["sigma_bar"] - ref["sigma_bar"]).max()
                                                           / np.abs(ref["sigma_bar"]).max()))
    print(json.dumps({"workload": "sweep (config 4): 256 problems, m = 2^12..2^21 (sum %d points), 2-D and 3-D, "
                                  "rank-1/rank-2/diagonal, contrast 1e-2..1e2, all unit load cases, mixed, tol 1e-6"
                                  % sum(p_["plan"].m for p_ in probs),
                      "metric": METRIC, "unit": "point-iterations/s", "setup_s": round(t_setup, 1), "results": res,
                      "checked_problems": [int(i) for i in pick], "max_rel_err_vs_fp64": worst,
                      "l2": "flushed between timed steps"}))


def bench_gather(args):
    """Subsampling (Sec. 2.1 / 5.2): three binary64 field planes on the 2048 x 2048 grid gathered onto its
    rank-2 subpattern N = [[2048,1024],[0,1024]] (m = 2^21) through lattice_gather; HBM GB/s of the
    gather (algorithmic bytes: the planes read at the mapped points and written, plus the map)."""
    import torch
    from paper_1605_05712_gb300 import gather, gather_map, lattice_plan
    dev = torch.device("cuda", 0)
    src, dst = lattice_plan([[2048, 0], [0, 2048]]), lattice_plan([[2048, 1024], [0, 1024]])
    t0 = time.perf_counter()
    mp = torch.from_numpy(gather_map(src, dst)).to(dev)
    t_map = time.perf_counter() - t0
    x = torch.randn((3, src.m), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream()
    for _ in range(args.warmup):
        gather(x, mp)
    def step():
        gather(x, mp)
        return dst.m, None
    ms, _, _ = timed(step, args.steps, flush, st)
    nbytes = 3 * dst.m * 8 * 2 + dst.m * 4
    pk = peaks()
    print(json.dumps({"workload": "gather: 3 binary64 planes, 2048^2 grid -> subpattern [[2048,1024],[0,1024]] "
                                  "(m = 2^21)", "map_host_s": round(t_map, 3), "ms": round(ms, 4),
                      "algorithmic_bytes": nbytes, "achieved_gbs": round(nbytes / (ms * 1e-3) / 1e9, 1),
                      "hbm_peak_gbs": pk.get("hbm_gbs"),
                      "frac": round(nbytes / (ms * 1e-3) / 1e9 / pk["hbm_gbs"], 3) if pk.get("hbm_gbs") else None}))


def bench_shear_sweep(args):
    """Sec. 5.1 shear sweep: Example 4.1's coated ellipse (one point along x3) on the 393 pattern matrices
    M_{j,k,alpha}, M~_j (m = 2^14 / 2^13), the analytic load case eps0, all in one
    basic_scheme_solve_multi call per precision, tol 1e-8; e_eff of the Table-1 matrices against the
    analytic C^eff eps0."""
    import torch
    from paper_1605_05712_gb300 import basic_scheme_solve_multi, lattice_plan, multi_workspace_bytes, synth
    dev = torch.device("cuda", 0)
    w = synth.hashin2d_workload()
    E = np.array([[w["eps0"][0, 0], w["eps0"][1, 1], w["eps0"][2, 2], w["eps0"][1, 2], w["eps0"][0, 2],
                   w["eps0"][0, 1]]])
    probs = []
    for name, M in synth.shear_sweep_matrices():
        P = lattice_plan(M)
        ph = synth.coated_ellipsoid_phase(P.points(), P.m, w["c"], w["rho_c"], w["rho_e"], R=w["R"])
        probs.append(dict(name=name, plan=P, phase=torch.from_numpy(ph).to(dev), stiffness=w["stiffness"],
                          C0=w["C0"], E=E, eps=torch.empty((1, 6, P.m), dtype=torch.float64, device=dev)))
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream()
    ref = np.linalg.norm(w["ceff_eps0"])
    res = {}
    for prec in ("fp64", "df64", "mixed"):
        ws = torch.empty(multi_workspace_bytes(probs, prec), dtype=torch.uint8, device=dev)
        last = {}

        def step():
            rc, outs = basic_scheme_solve_multi(probs, tol=1e-8, maxit=3000, precision=prec, workspace=ws)
            last["outs"] = outs
            return sum(p_["plan"].m * int(o["iters"][0]) for p_, o in zip(probs, outs)), None
        step()
        ms, units, _ = timed(step, max(1, args.steps), flush, st)
        eff = {}
        for p_, o in zip(probs, last["outs"]):
            sb = o["sigma_bar"][0]
            S = np.array([[sb[0], sb[5], sb[4]], [sb[5], sb[1], sb[3]], [sb[4], sb[3], sb[2]]])
            eff[p_["name"]] = float(np.linalg.norm(S - w["ceff_eps0"]) / ref)
        res[prec] = {"ms": round(ms, 2), "value": round(units / (ms / 1e3), 1),
                     "e_eff_table1": {k: round(eff[k], 5) for k in ("M_7,0,0", "M~_7", "M_8,16,0", "M_9,-496,0",
                                                                   "M_9,16,0", "M_7,272,1")},
                     "e_eff_min": [min(eff, key=eff.get), round(min(eff.values()), 5)]}
        del ws
    print(json.dumps({"workload": "shear sweep (Sec. 5.1): 393 matrices M_{j,k,alpha}, M~_j, coated ellipse of "
                                  "Example 4.1, eps0 load case, tol 1e-8", "metric": METRIC,
                      "unit": "point-iterations/s", "results": res}))


def profile_case(args):
    """Plain launches of the iteration kernels (lattice_pass_times) for ncu: precision and lattice on argv."""
    import torch
    from paper_1605_05712_gb300 import lattice_pass_times, lattice_plan, synth
    prec, M = args.profile_case[0], json.loads(args.profile_case[1])
    P = lattice_plan(M)
    ph = torch.from_numpy(synth.laminate_phase(P.points(), P.m, [1, 3] if P.d == 2 else [1, 3, 2])).cuda()
    st = [synth.iso_voigt(*l) for l in LAMES]
    E = np.zeros(P.n_c)
    E[0] = 1.0
    if args.profile_scheme == "cg":
        # a conjugate-gradient solve with plain launches (ncu sees each kernel): prologue stages
        # FWD_X, FULL0, A, then per iteration B, the column passes, A
        from paper_1605_05712_gb300 import basic_scheme_solve
        t0 = time.perf_counter()
        g = basic_scheme_solve(P, ph, st, (5.5, 5.5), E, tol=0.0, maxit=args.steps, precision=prec, scheme="cg",
                               boundary="zero", plain_launches=True)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": M, "precision": prec, "scheme": "cg", "m": P.m,
                          "iterations": int(g["iters"][0]), "s": round(time.perf_counter() - t0, 3)}))
        return
    ms = lattice_pass_times(P, ph, st, (5.5, 5.5), E, precision=prec, n_reps=args.steps)
    print(json.dumps({"profile_case": M, "precision": prec, "m": P.m, "ms_per_kernel": ms}))


def oracle_sample(seconds, names=("rank2_262144",)):
    """Time the CPU oracle on a bounded sample: a few iterations of the workload's solves."""
    from oracle import elasticity as el
    from oracle.lattice import Lattice
    from oracle.scheme import basic_scheme
    from paper_1605_05712_gb300 import synth
    S = np.array([el.voigt6_to_tensor(synth.iso_voigt(*l), 2) for l in LAMES])
    C0 = synth.c0_mean_extremes([l[0] for l in LAMES], [l[1] for l in LAMES])
    units, t_total, n_it = 0, 0.0, 0
    lats = {}
    for nm in names:
        L = Lattice(synth.LATTICES[nm])
        lats[nm] = (L, synth.laminate_phase(L.p, L.m, N_INT))
    E = el.comps_to_sym(load_cases()[0], 2)
    while t_total < seconds:
        for nm in names:
            L, ph = lats[nm]
            t0 = time.perf_counter()
            r = basic_scheme(L, ph, S, C0, E, tol=0.0, maxit=2)
            t_total += time.perf_counter() - t0
            units += L.m * r["iters"]
            n_it += r["iters"]
    return units / t_total, t_total, n_it


def cpu_baseline(seconds):
    v, t, n = oracle_sample(seconds)
    return {"value": round(v, 1), "unit": "point-iterations/s", "cores": 1, "kind": "oracle",
            "sample": "%d iterations of the oracle (numpy float64, single thread) on the rank-2 m=262144 "
                      "laminate, unit load case 11, %.1f s" % (n, t)}


def bench_reference(args):
    rank = int(os.environ.get("RANK", 0))
    if rank != 0:
        return
    vals = []
    for _ in range(args.warmup):
        oracle_sample(1.0)
    tt = 0
    for _ in range(args.steps):
        v, t, n = oracle_sample(max(2.0, args.cpu_seconds / max(args.steps, 1)))
        vals.append(v)
        tt += t
    v = float(np.mean(vals))
    res = {"impl": "reference", "metric": METRIC, "value": round(v, 1), "unit": "point-iterations/s",
           "n_gpus": 0, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
           "ms_per_step": round(1e3 * tt / max(args.steps, 1), 2), "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "lattices": LATS, "load_cases": 3, "tol": TOL,
                      "sample": "each step a bounded sample of the workload: oracle iterations on the rank-2 "
                                "lattice [[512,16],[0,512]], unit load case 11, point-iterations counted"},
           "cpu_baseline": {"value": round(v, 1), "unit": "point-iterations/s", "cores": 1, "kind": "oracle",
                            "sample": "2-iteration oracle solves repeated for ~%.0f s per step" %
                                      max(2.0, args.cpu_seconds / max(args.steps, 1))},
           "e2e": {"value": round(v, 1), "unit": "point-iterations/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(res))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--profile-case", nargs=2, metavar=("PRECISION", "M_JSON"))
    ap.add_argument("--profile-scheme", default="basic", choices=["basic", "cg"],
                    help="with --profile-case: cg runs a conjugate-gradient solve of --steps iterations")
    ap.add_argument("--plain-launches", action="store_true",
                    help="iterate with plain kernel launches (same results) so that ncu lists every kernel")
    ap.add_argument("--workload", default="laminate2d", choices=["laminate2d", "hashin3d", "warmstart", "sweep", "gather", "shear_sweep"])
    ap.add_argument("--ws-samples", type=int, default=2000)
    ap.add_argument("--ws-train-n", type=int, default=64)
    ap.add_argument("--ws-eval-n", type=int, default=128)
    ap.add_argument("--ws-eval", type=int, default=4)
    args = ap.parse_args()
    global PLAIN_LAUNCHES
    PLAIN_LAUNCHES = args.plain_launches
    if args.profile_case:
        profile_case(args)
    elif args.workload == "hashin3d":
        bench_hashin(args)
    elif args.workload == "warmstart":
        bench_warmstart(args)
    elif args.workload == "sweep":
        bench_sweep(args)
    elif args.workload == "gather":
        bench_gather(args)
    elif args.workload == "shear_sweep":
        bench_shear_sweep(args)
    elif args.impl == "reference":
        bench_reference(args)
    else:
        bench_gpu(args)


if __name__ == "__main__":
    main()
