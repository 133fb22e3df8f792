#!/usr/bin/env python3
"""Benchmark of the lattice Basic Scheme (Algorithm 1, arXiv 1605.05712) on GB300.

Workload (one "step"): the 3-D generalized Hashin structure of Sec. 4.2 -- a coated ellipsoid (core
semi-axes (0.1, 0.15, 0.2), total inclusion fraction 0.25, seeded rotation; core (lam, mu) = (10, 10),
confocal coating (1, 1), matrix (1, 1) plus the rank-one correction that makes the coated inclusion
neutral for eps0) -- on three lattices of m = 2^21 points: the tensor grid diag(128,128,128), the rank-1
lattice [[128,1,0],[0,128,1],[0,0,128]] and the sheared full-rank lattice [[128,16,0],[0,128,16],[0,0,128]].
Per lattice one solve of the six unit load cases batched (one launch set for all six), to a Cauchy
residual of 1e-6, binary64 throughout (the paper's precision).  Metric: lattice-point iterations per
second (sum over lattices and load cases of m x iterations / step time).

Legs: device-timed steps with inputs resident in HBM (value); the same through the C ABI with the phase
fields copied host->device and all six strain fields of every lattice copied back every step (e2e);
per-kernel CUDA-event timing of one batched iteration on each lattice, in binary64 (ALU roofline) and in
mixed precision (HBM roofline); variants (mixed, double-float pairs, Eyre-Milton, conjugate gradients,
time to r < 1e-6 against binary64, and the 2-D m = 262144 laminate); the CPU oracle on a bounded sample
on the host cores (cpu_baseline).  ``--impl reference`` times the oracle alone.
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

LATS = ["grid128", "rank1_2097152", "sheared128"]
WORKLOAD = ("3-D generalized Hashin structure (coated ellipsoid, fraction 0.25, core/coating/matrix 10/1/1 + "
            "rank-one neutrality correction), m=2^21 on diag(128,128,128), rank-1 [[128,1,0],[0,128,1],[0,0,128]] "
            "and sheared [[128,16,0],[0,128,16],[0,0,128]]; 6 unit load cases batched per solve; tol 1e-6; FP64")
TOL = 1e-6
MAXIT = 2000
N_LC = 6
METRIC = "lattice-point iterations/s"
N_SM = 152
FP64_FMA_PER_SM_CLK = 2      # GB300 binary64 pipe: 2 FMA per SM per clock (1.25 TFLOP/s nominal near 2 GHz)
L2_FLUSH_BYTES = 512 << 20
# 2-D laminate of m = 262144 (a variant): normal (1,3), fraction 1/2, phases (1,1) and (10,10)
LATS2 = ["grid512", "rank1_262144", "rank2_262144"]
LAMES = [(1.0, 1.0), (10.0, 10.0)]
N_INT = [1, 3]


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def fp64_peak_tflops(pk):
    """Binary64 ALU peak from unit counts and the maximum SM clock: 152 SMs x 2 FMA x 2 flops x f_max."""
    f = pk.get("sm_max_mhz") or 2070.0
    return N_SM * FP64_FMA_PER_SM_CLK * 2 * f * 1e6 / 1e12


def unit_loads(n_c):
    E = np.eye(n_c)
    d = 3 if n_c == 6 else 2
    E[d:, d:] *= 0.5              # unit load cases in tensor components (eps_ij = eps_ji = 1/2)
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


# ------------------------------------------------------------------ cost model from the plan's decomposition
def tables_orthotropic(stiffness, d):
    """True when every Voigt table couples no normal and shear components and has a diagonal shear block
    (exact zeros): the row pass then polarizes with the normal block and the shear diagonal only."""
    vi = [0, 1, 2, 3, 4, 5] if d == 3 else [0, 1, 5]
    n_c = len(vi)
    for V in stiffness:
        V = np.asarray(V)
        for I in range(n_c):
            for J in range(n_c):
                if I != J and (I >= d or J >= d) and V[vi[I], vi[J]] != 0.0:
                    return False
    return True


def kernel_models(P, n_items, prec, ortho=False):
    """Algorithmic flops and HBM bytes of every kernel of one batched iteration, in launch order (row pass,
    then the column passes: forward groups innermost first, the Green group, inverse groups), from the
    plan's FFT decomposition (lattice_plan_layout).  5 N log2 N flops per complex FFT of N points; ~10 flops
    per complex value for each R2C pre/post-processing; 2 n_c^2 per point for the polarization (orthotropic
    tables: 2 (d^2 + n_c - d), the products that are not structurally zero) and 3 n_c for the update and
    residual; ~90 per complex frequency value for the Green operator; 6 per complex value for each four-step
    twiddle.  Bytes: every HBM-resident word read and written once (spectrum slots of s bytes per complex
    value, the strain as 8-byte words, one phase byte per point)."""
    import math
    lay = P.layout()
    n_c, m = P.n_c, P.m
    n_pol = (P.d * P.d + n_c - P.d) if ortho else n_c * n_c
    ax = lay["ax_len"]
    R = ax[-1]
    Rh = R // 2
    spec = m // 2 + m // R                     # complex values per component: half spectrum + Nyquist plane
    s = 8 if prec == "mixed" else 16
    row_f = n_c * (m // R) * 2 * (5 * Rh * math.log2(max(Rh, 1)) + 10 * Rh) + m * (2 * n_pol + 3 * n_c)
    if len(ax) == 1:
        row_f += 90 * spec
    row_b = 2 * n_c * spec * s + 2 * n_c * m * 8 + m
    out = [dict(kernel="row_pass", flops=n_items * row_f, bytes=n_items * row_b)]
    groups = lay["groups"]
    order = [(k, "gamma" if k == 0 else "fwd") for k in range(len(groups) - 1, -1, -1)] + \
            [(k, "inv") for k in range(1, len(groups))]
    for k, mode in order:
        a0, a1 = groups[k]
        G = int(np.prod(ax[a0:a1]))
        dirs = 2 if mode == "gamma" else 1
        f = n_c * dirs * 5 * spec * math.log2(G)
        if mode == "gamma":
            f += 90 * spec
        if lay["split"]:
            f += n_c * dirs * 6 * spec
        out.append(dict(kernel="col_pass_%s_g%d" % (mode, k), flops=n_items * f, bytes=n_items * 2 * n_c * spec * s))
    return out


def launches_per_solve(P, iters, prec):
    """Kernels one batched solve launches: fill, (pair conversion), prologue, the loop body once per
    iteration of the slowest item, (pair conversion back), effective stress."""
    nk = 1 + max(0, 2 * len(P.layout()["groups"]) - 1)
    return 1 + (2 if prec != "fp64" else 0) + nk + int(max(iters)) * nk + 1


# ------------------------------------------------------------------ workload
def setup(dev, want_host=True):
    import torch
    from paper_1605_05712_gb300 import lattice_plan, synth
    w = synth.hashin_workload()
    out = []
    for name in LATS:
        P = lattice_plan(synth.LATTICES[name])
        ph = synth.coated_ellipsoid_phase(P.points(), P.m, w["c"], w["rho_c"], w["rho_e"], R=w["R"])
        item = dict(name=name, plan=P, phase=torch.from_numpy(ph).to(dev),
                    eps=torch.empty((N_LC, 6, P.m), dtype=torch.float64, device=dev))
        if want_host:
            item["phase_host"] = torch.from_numpy(ph).pin_memory()
            item["eps_host"] = torch.empty((N_LC, 6, P.m), dtype=torch.float64).pin_memory()
        out.append(item)
    return w, out


PLAIN_LAUNCHES = False   # --plain-launches: iterate with plain launches instead of the CUDA-graph loop

FORMS = {
    # name: (precision, scheme options, reference medium: "mean" of the extremes or "geo" geometric mean)
    "fp64": ("fp64", {}, "mean"),
    "mixed": ("mixed", {}, "mean"),
    "df64": ("df64", {}, "mean"),
    "fp64_eyre_milton": ("fp64", {"scheme": "eyre_milton"}, "geo"),
    "mixed_eyre_milton": ("mixed", {"scheme": "eyre_milton"}, "geo"),
    "fp64_cg": ("fp64", {"scheme": "cg", "boundary": "zero"}, "mean"),
    "df64_cg": ("df64", {"scheme": "cg", "boundary": "zero"}, "mean"),
}


def run_step(w, work, ws, form="fp64", tol=TOL, to_host=False):
    """One pass of the workload: per lattice one batched solve of the six unit load cases."""
    from paper_1605_05712_gb300 import basic_scheme_solve
    prec, kw, c0 = FORMS[form]
    C0 = w["C0"] if c0 == "mean" else (float(np.sqrt(10.0)),) * 2   # geometric mean of core and coating
    E = unit_loads(6)
    tot, iters = 0, []
    for it in work:
        if to_host:
            it["phase"].copy_(it["phase_host"], non_blocking=True)
        g = basic_scheme_solve(it["plan"], it["phase"], w["stiffness"], C0, E, tol=tol, maxit=MAXIT, workspace=ws,
                               eps_out=it["eps"], precision=prec, plain_launches=PLAIN_LAUNCHES, **kw)
        if to_host:
            it["eps_host"].copy_(it["eps"], non_blocking=True)
        its = [int(x) for x in g["iters"]]
        iters.append(its)
        tot += it["plan"].m * int(np.sum(its))
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
    for f in ("kernels.cu", "kernels_dev.cuh", "fft_smem.cuh", "kernels.cuh", "kernels_gen.cu", "fft_mixed.cuh"):
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


def roofline_of(w, work, prec, iters, pk, bound):
    """Per-kernel CUDA-event times of one batched iteration (all six load cases, as the solve launches
    them) on every lattice; the dominant kernel is the one with the largest share of the step (time per
    launch x iterations of its lattice); achieved = its algorithmic flops or bytes per launch / its time."""
    from paper_1605_05712_gb300 import lattice_pass_times
    E = unit_loads(6)
    rows, best = [], None
    for it, its in zip(work, iters):
        P = it["plan"]
        ms = lattice_pass_times(P, it["phase"], w["stiffness"], w["C0"], E, precision=prec, n_reps=10)
        models = kernel_models(P, N_LC, prec, ortho=tables_orthotropic(w["stiffness"], P.d))
        for k, (t, mo) in enumerate(zip(ms, models)):
            share = t * max(its)
            rec = dict(lattice=it["name"], kernel=mo["kernel"], ms=round(t, 5), flops=mo["flops"], bytes=mo["bytes"],
                       share_ms_per_step=round(share, 3))
            rows.append(rec)
            if best is None or share > best["share_ms_per_step"]:
                best = rec
    t = best["ms"] * 1e-3
    kname = best["kernel"].split("_")[0] + "_pass"
    real = {"fp64": "double", "mixed": "float", "df64": "dfloat"}[prec]
    tag = "%s<%s,6>/%s/%s" % (kname, real, best["kernel"], best["lattice"])
    if bound == "alu":
        peak = fp64_peak_tflops(pk)
        ach = best["flops"] / t / 1e12
        roof = {"bound": "alu", "achieved": round(ach, 4), "peak": round(peak, 4), "unit": "TFLOP/s",
                "frac": round(ach / peak, 4),
                "peak_source": "derived from unit counts and clocks: 152 SMs x 2 binary64 FMA/clk x 2 flops x "
                               "%.0f MHz (sm_max_mhz of the measured peaks)" % (pk.get("sm_max_mhz") or 2070.0)}
    else:
        peak = pk.get("hbm_gbs")
        ach = best["bytes"] / t / 1e9
        roof = {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                "frac": round(ach / peak, 4) if peak else None,
                "peak_source": "hbm_gbs of MEASURED_PEAKS.json (of measured)" if peak else "no measured peak"}
    roof.update({"traffic": profiled_traffic(tag), "kernel": tag, "algorithmic_flops_per_launch": best["flops"],
                 "algorithmic_bytes_per_launch": best["bytes"], "ms_per_launch": best["ms"],
                 "hbm_achieved_gbs": round(best["bytes"] / t / 1e9, 1),
                 "per_kernel": rows})
    return roof


def bench_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_1605_05712_gb300.api import LAT_WS_CG
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(args.cpu_seconds)     # worker processes spawned before this process uses the GPU
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w, work = setup(dev)
    ws = torch.empty(max(it["plan"].workspace_bytes(N_LC, p) for it in work for p in (0, 1, 2, 0 | LAT_WS_CG, 2 | LAT_WS_CG)),
                     dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream()

    for _ in range(args.warmup):
        run_step(w, work, ws)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = Clocks(local)
    ms_step, units, iters = timed(lambda: run_step(w, work, ws), args.steps, flush, st)
    # end-to-end: host phase fields -> device, solves, all six strain fields of every lattice -> host
    ms_e2e, e2e_units, _ = timed(lambda: run_step(w, work, ws, to_host=True), args.steps, flush, st)
    clocks = clk.stop()
    (ms_step, ms_e2e), (value, e2e_value) = aggregate_ranks([ms_step, ms_e2e], [units, e2e_units], world, dev)
    pk = peaks()
    roof = roofline_of(w, work, "fp64", iters, pk, "alu")

    variants = {}
    if not args.no_variants:
        # a variant that fails is recorded as such; the headline line above it still prints
        def variant(name, fn):
            try:
                variants[name] = fn()
            except Exception as e:          # noqa: BLE001 -- reported in the JSON line, not hidden
                torch.cuda.synchronize()
                variants[name] = {"error": "%s: %s" % (type(e).__name__, e)}

        ttt = {}

        def time_form(form):
            run_step(w, work, ws, form)
            ms_v, u_v, it_v = timed(lambda: run_step(w, work, ws, form), max(1, min(args.steps, 3)), flush, st)
            return {"ms": round(ms_v, 3), "value": round(u_v / (ms_v / 1e3), 1), "iterations": it_v,
                    "speedup_vs_fp64": round(ms_step / ms_v, 2)}

        for form in ("mixed", "df64", "mixed_eyre_milton", "fp64_eyre_milton", "df64_cg", "fp64_cg"):
            try:
                ttt[form] = time_form(form)
            except Exception as e:          # noqa: BLE001
                torch.cuda.synchronize()
                ttt[form] = {"error": "%s: %s" % (type(e).__name__, e)}
        ttt["fp64"] = {"ms": round(ms_step, 3), "value": round(value, 1), "iterations": iters}
        variants["time_to_resid_1e-6_ms"] = ttt
        if "iterations" in ttt["mixed"]:
            def mixed_roof():
                run_step(w, work, ws, "mixed")
                return roofline_of(w, work, "mixed", ttt["mixed"]["iterations"], pk, "hbm")
            variant("mixed_roofline", mixed_roof)
        variant("laminate2d_262144", lambda: bench_laminate2d(dev, args, flush, st))
        variant("laminate4096_latency", lambda: bench_laminate4096(dev, args, flush, st))

    gpu_launches = sum(launches_per_solve(it["plan"], its, "fp64") for it, its in zip(work, iters))
    m_total = sum(it["plan"].m for it in work)
    res = {
        "metric": METRIC, "value": round(value, 1), "unit": "point-iterations/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded coated-ellipsoid phases generated on the host)",
        "config": {"workload": WORKLOAD, "lattices": LATS, "m": work[0]["plan"].m, "load_cases": N_LC, "tol": TOL,
                   "iterations": iters,
                   "l2": "inputs larger than L2 (strain 604 MB per lattice) and a 512 MiB write between timed steps",
                   "parallelism": "replicas" if world > 1 else "1 GPU",
                   "launch": "plain launches, host convergence check per iteration" if PLAIN_LAUNCHES
                             else "one CUDA-graph WHILE loop per solve"},
        "roofline": roof,
        "e2e": {"value": round(e2e_value, 1), "unit": "point-iterations/s",
                "h2d_bytes_per_step": int(m_total),
                "d2h_bytes_per_step": int(sum(it["eps"].numel() * 8 for it in work))},
        "gpu_launches": gpu_launches,
        "clocks": clocks,
        "variants": variants,
    }
    if cpu is not None:
        res["cpu_baseline"] = cpu
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(res))


def bench_laminate2d(dev, args, flush, st):
    """The 2-D laminate at m = 262144 on three lattices, the three unit load cases solved one after another
    to tol 1e-8 in binary64 (and batched, and in the other precisions)."""
    import torch
    from paper_1605_05712_gb300 import basic_scheme_solve, lattice_plan, synth
    stiff = [synth.iso_voigt(*l) for l in LAMES]
    C0 = synth.c0_mean_extremes([l[0] for l in LAMES], [l[1] for l in LAMES])
    E = unit_loads(3)
    work = []
    for name in LATS2:
        P = lattice_plan(synth.LATTICES[name])
        work.append((P, torch.from_numpy(synth.laminate_phase(P.points(), P.m, N_INT)).to(dev)))
    ws = torch.empty(max(P.workspace_bytes(3, p) for P, _ in work for p in (0, 1, 2)), dtype=torch.uint8, device=dev)
    eps = torch.empty((3, 3, work[0][0].m), dtype=torch.float64, device=dev)
    out = {}
    for mode in ("fp64_separate", "fp64_batched", "df64_batched", "mixed_batched"):
        prec = mode.split("_")[0]

        def step():
            tot, its_all = 0, []
            for P, ph in work:
                if mode.endswith("separate"):
                    its = []
                    for lc in range(3):
                        g = basic_scheme_solve(P, ph, stiff, C0, E[lc:lc + 1], tol=1e-8, maxit=MAXIT, workspace=ws,
                                               eps_out=eps[lc:lc + 1], precision=prec)
                        its.append(int(g["iters"][0]))
                else:
                    g = basic_scheme_solve(P, ph, stiff, C0, E, tol=1e-8, maxit=MAXIT, workspace=ws, eps_out=eps,
                                           precision=prec)
                    its = [int(x) for x in g["iters"]]
                its_all.append(its)
                tot += P.m * sum(its)
            return tot, its_all
        step()
        ms, u, its = timed(step, max(1, min(args.steps, 3)), flush, st)
        out[mode] = {"value": round(u / (ms / 1e3), 1), "ms_per_step": round(ms, 3), "iterations": its}
    return out


def bench_laminate4096(dev, args, flush, st):
    """The latency case: the 2-D laminate (layer normal (1,3), phases (1,1) / (10,10), C0 the mean of the
    extremes) at m = 4096, E = (1,0,0), one binary64 solve to tol 1e-8 per lattice: the aligned rank-1
    lattice [[4096,12288],[0,1]], the spread rank-1 lattice [[64,1],[0,64]] and the tensor grid diag(64,64)
    the paper times (94 iterations, 41.2 s in its Matlab code).  Wall time per solve through the C ABI
    (device inputs, results left on the device), median of the timed repeats."""
    import torch
    from paper_1605_05712_gb300 import basic_scheme_solve, lattice_plan, synth
    stiff = [synth.iso_voigt(*l) for l in LAMES]
    C0 = synth.c0_mean_extremes([l[0] for l in LAMES], [l[1] for l in LAMES])
    E = unit_loads(3)[:1]
    out = {}
    for name, M in (("laminate4096_aligned", synth.LATTICES["laminate4096_aligned"]),
                    ("laminate4096_rank1", synth.LATTICES["laminate4096_rank1"]), ("grid64", [[64, 0], [0, 64]])):
        P = lattice_plan(M)
        ph = torch.from_numpy(synth.laminate_phase(P.points(), P.m, N_INT)).to(dev)
        ws = torch.empty(P.workspace_bytes(1, 0), dtype=torch.uint8, device=dev)
        eps = torch.empty((1, 3, P.m), dtype=torch.float64, device=dev)
        solve = lambda: basic_scheme_solve(P, ph, stiff, C0, E, tol=1e-8, maxit=MAXIT, workspace=ws, eps_out=eps)
        for _ in range(3):
            g = solve()
        times = []
        for _ in range(max(5, args.steps)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g = solve()
            times.append((time.perf_counter() - t0) * 1e3)
        ms = float(np.median(times))
        out[name] = {"M": M, "m": P.m, "iterations": int(g["iters"][0]), "ms_per_solve": round(ms, 3),
                     "point_iterations_per_s": round(P.m * int(g["iters"][0]) / (ms / 1e3), 1),
                     "sigma_bar": [float(x) for x in np.asarray(g["sigma_bar"][0])]}
    return out


def bench_hashin(args):
    """The coated-ellipsoid workload: the coated-ellipsoid (generalized Hashin) structure at m = 2^21 on the tensor grid,
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
    print(json.dumps({"workload": "hashin3d: coated ellipsoid c=(0.1,0.15,0.2), fraction 0.25, "
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
    losses = train(net, args.ws_train_n, args.ws_samples, args.ws_steps, args.ws_lr, seed0=5000)
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
    print(json.dumps({"workload": "warmstart: train %d samples x %d Adam steps (lr %g) at %d^3, evaluate "
                                  "%d held-out seeds at %d^3, 6 unit load cases batched, tol 1e-6"
                                  % (args.ws_samples, args.ws_steps, args.ws_lr, args.ws_train_n, args.ws_eval, n),
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
    print(json.dumps({"workload": "sweep: 256 problems, m = 2^12..2^21 (sum %d points), 2-D and 3-D, "
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


def profile_conv(args):
    """Plain launches of the warm-start network for ncu: --steps forward passes at n^3 with seeded
    parameters and a seeded three-phase feature field (the convolutions run on tcgen05 for rows of 16,
    32, 64 and 128 voxels)."""
    import torch
    from paper_1605_05712_gb300.warmstart import WarmStartNet
    dev = torch.device("cuda", 0)
    n = args.profile_conv
    net = WarmStartNet(dev, seed=5)
    rng = np.random.default_rng(5)
    phase = torch.from_numpy(rng.integers(0, 3, size=n ** 3).astype(np.uint8)).to(dev)
    net.features(phase, rng.uniform(0.0, 2.0, size=(3, 21)).astype(np.float32), n)
    for _ in range(max(1, args.steps)):
        net.forward(n)
    torch.cuda.synchronize()


def profile_case(args):
    """Plain launches of one iteration's kernels (lattice_pass_times) for ncu: precision and lattice on argv,
    --profile-loads load cases batched (the bench solves six).  3-D lattices take the coated-ellipsoid
    workload of the bench, 2-D ones the laminate."""
    import torch
    from paper_1605_05712_gb300 import lattice_pass_times, lattice_plan, synth
    prec, M = args.profile_case[0], json.loads(args.profile_case[1])
    P = lattice_plan(M)
    if P.d == 3:
        w = synth.hashin_workload()
        ph = torch.from_numpy(synth.coated_ellipsoid_phase(P.points(), P.m, w["c"], w["rho_c"], w["rho_e"],
                                                           R=w["R"])).cuda()
        st, C0 = w["stiffness"], w["C0"]
    else:
        ph = torch.from_numpy(synth.laminate_phase(P.points(), P.m, [1, 3])).cuda()
        st, C0 = [synth.iso_voigt(*l) for l in LAMES], (5.5, 5.5)
    E = unit_loads(P.n_c)[:max(1, args.profile_loads)]
    if args.profile_scheme == "cg":
        # a conjugate-gradient solve with plain launches (ncu sees each kernel): prologue stages
        # FWD_X, FULL0, A, then per iteration B, the column passes, A
        from paper_1605_05712_gb300 import basic_scheme_solve
        t0 = time.perf_counter()
        g = basic_scheme_solve(P, ph, st, C0, E, tol=0.0, maxit=args.steps, precision=prec, scheme="cg",
                               boundary="zero", plain_launches=True)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": M, "precision": prec, "scheme": "cg", "m": P.m,
                          "iterations": int(g["iters"][0]), "s": round(time.perf_counter() - t0, 3)}))
        return
    ms = lattice_pass_times(P, ph, st, C0, E, precision=prec, n_reps=args.steps)
    print(json.dumps({"profile_case": M, "precision": prec, "m": P.m, "load_cases": len(E), "ms_per_kernel": ms,
                      "layout": P.layout()}))


def _oracle_proc(name, lc, iters, barrier, q):
    """Spawned worker: build the lattice and phases of one coated-ellipsoid problem (m = 2^21), wait for the others at the
    barrier, then run `iters` oracle iterations of unit load case lc (numpy float64, one thread)."""
    sys.path.insert(0, ROOT)
    from oracle import elasticity as el
    from oracle.lattice import Lattice
    from oracle.scheme import basic_scheme
    from paper_1605_05712_gb300 import synth
    w = synth.hashin_workload()
    L = Lattice(synth.LATTICES[name])
    ph = synth.coated_ellipsoid_phase(L.p, L.m, w["c"], w["rho_c"], w["rho_e"], R=w["R"])
    S = np.array([el.voigt6_to_tensor(V, 3) for V in w["stiffness"]])
    E = el.comps_to_sym(unit_loads(6)[lc], 3)
    barrier.wait()
    t0 = time.time()
    r = basic_scheme(L, ph, S, w["C0"], E, tol=0.0, maxit=iters)
    q.put((L.m * r["iters"], t0, time.time()))


def _mem_available():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) * 1024
    except Exception:
        pass
    return 16 << 30


ORACLE_BYTES = 3.5e9     # peak memory of one oracle solve at m = 2^21 (measured ~3.0 GB)


def oracle_sample(n_proc, iters):
    """n_proc spawned processes, each running `iters` oracle iterations of its own (lattice, load case) of
    the coated-ellipsoid workload at the same time; returns (point-iterations/s over the common wall time, wall
    seconds).  Spawned, so no worker inherits a CUDA context."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    barrier, q = ctx.Barrier(n_proc), ctx.Queue()
    procs = [ctx.Process(target=_oracle_proc, args=(LATS[i % 3], i % 6, iters, barrier, q)) for i in range(n_proc)]
    for p_ in procs:
        p_.start()
    res = [q.get() for _ in range(n_proc)]
    for p_ in procs:
        p_.join()
    units = sum(r[0] for r in res)
    wall = max(r[2] for r in res) - min(r[1] for r in res)
    return units / wall, wall


def oracle_procs():
    """Worker count: every host core, capped at 16 and at a quarter of the available memory."""
    ncpu = os.cpu_count() or 1
    return max(1, min(ncpu, 16, int(_mem_available() / 4 / ORACLE_BYTES)))


def cpu_baseline(seconds):
    n = oracle_procs()
    v1, t1 = oracle_sample(1, 1)
    iters = max(1, int(round(seconds / max(t1, 1e-3))))
    vn, tn = oracle_sample(n, iters)
    return {"value": round(vn, 1), "unit": "point-iterations/s", "cores": n, "kind": "oracle",
            "single_process_value": round(v1, 1),
            "host_cpus": os.cpu_count(),
            "sample": "%d processes, each %d oracle iteration(s) (numpy float64, one thread each) of one unit load "
                      "case on one m=2^21 coated-ellipsoid lattice, started together, %.1f s wall; single process: 1 "
                      "iteration in %.1f s" % (n, iters, tn, t1)}


def bench_reference(args):
    rank = int(os.environ.get("RANK", 0))
    if rank != 0:
        return
    n = oracle_procs()
    for _ in range(args.warmup):
        oracle_sample(1, 1)
    vals, tt = [], 0.0
    for _ in range(args.steps):
        v, t = oracle_sample(n, 1)
        vals.append(v)
        tt += t
    v = float(np.mean(vals))
    res = {"impl": "reference", "metric": METRIC, "value": round(v, 1), "unit": "point-iterations/s",
           "n_gpus": 0, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
           "ms_per_step": round(1e3 * tt / max(args.steps, 1), 2), "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "lattices": LATS, "load_cases": N_LC, "tol": TOL,
                      "sample": "each step a bounded sample of the workload: one oracle iteration in each of %d "
                                "processes (lattice i mod 3, unit load case i mod 6), point-iterations counted" % n},
           "cpu_baseline": {"value": round(v, 1), "unit": "point-iterations/s", "cores": n, "kind": "oracle",
                            "host_cpus": os.cpu_count(),
                            "sample": "%d concurrent single-thread oracle processes, 1 iteration each per step" % n},
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
    ap.add_argument("--profile-loads", type=int, default=1, help="with --profile-case: load cases batched")
    ap.add_argument("--profile-conv", type=int, default=0, metavar="N",
                    help="run --steps forward passes of the warm-start network at N^3 (for ncu)")
    ap.add_argument("--profile-scheme", default="basic", choices=["basic", "cg"],
                    help="with --profile-case: cg runs a conjugate-gradient solve of --steps iterations")
    ap.add_argument("--plain-launches", action="store_true",
                    help="iterate with plain kernel launches (same results) so that ncu lists every kernel")
    ap.add_argument("--workload", default="default", choices=["default", "hashin3d", "warmstart", "sweep", "gather",
                                                               "shear_sweep"])
    ap.add_argument("--ws-samples", type=int, default=10000)
    ap.add_argument("--ws-steps", type=int, default=2, help="Adam steps per training sample")
    ap.add_argument("--ws-lr", type=float, default=3e-4)
    ap.add_argument("--ws-train-n", type=int, default=64)
    ap.add_argument("--ws-eval-n", type=int, default=128)
    ap.add_argument("--ws-eval", type=int, default=4)
    args = ap.parse_args()
    global PLAIN_LAUNCHES
    PLAIN_LAUNCHES = args.plain_launches
    if args.profile_case:
        profile_case(args)
    elif args.profile_conv:
        profile_conv(args)
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
