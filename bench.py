"""TDA-risp benchmark: matvecs/s of full FP64 TDA-risp solves on GB300.

One step is one pass of the whole hot path on the 200-atom synthetic molecule
(100 heavy + 100 H, nao = 1900, nocc = 380; range-separated exchange
(0.222 + 0.778 erf(0.2 r))/r, 40 eV window, no aux functions on H):
integrals, metrics, MO transforms (tr_build) and the Davidson solve for 15
states with a block of 30 and residual 1e-5 (tr_solve).  value = Davidson
matvecs per second of the whole step (build included); the step time is the
time to 15 states.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Under torchrun each rank solves its own copy of the molecule (independent
problems, no collective); value sums the ranks' matvecs over the max time.
--impl reference times the CPU oracle on a bounded sample of the same
workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "TDA-risp FP64, 200-atom seeded molecule (100 C/N/O + 100 H), def2-SVP-shaped basis " \
           "(nao 1900), s+p aux on heavy atoms, RSH exchange (0.222 + 0.778 erf(0.2 r))/r, " \
           "40 eV window, 15 states, block 30, tol 1e-5"
METRIC = "TDA-risp matvecs/s (full solve: build + Davidson to 15 states)"
OPTS = dict(cx=1.0, k_alpha=0.222, k_beta=0.778, omega=0.2, window_ev=40.0, nstates=15,
            block=30, tol=1e-5, max_iter=200)


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_over_ranks(ms, units, device):
    """Whole-job figures of a timed region run on every rank: the slowest rank's
    time and the units all ranks processed (value = units / time).  One rank (or
    no process group) returns its own figures."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(units)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t[0]), float(u[0])


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_inputs(case="full"):
    from paper_2603_29257_gb300 import synth
    if case == "small":
        # profiling case of the same shape: 100 atoms (50 heavy + 50 H), nao 950
        return synth.make_molecule(seed=2, n_heavy=50, n_h=50)
    return synth.molecule_200()


# ------------------------------------------------------------------ native arm

def run_native(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_info()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_29257_gb300 import tdarisp

    mol = make_inputs(args.case)
    torch.zeros(1, device="cuda")
    stream = torch.cuda.current_stream()
    C_dev = torch.from_numpy(mol.C).cuda()
    eps_dev = torch.from_numpy(mol.eps).cuda()
    ctx = tdarisp.Context(stream=stream.cuda_stream, **OPTS)
    ctx.set_molecule(mol.Z, mol.xyz, mol.aux_exp, mol.shells)
    ctx.set_orbitals(C_dev, eps_dev, mol.nocc)
    d = ctx.dims()

    def step():
        ctx.build()
        om, X, rs, info = ctx.solve(want_x=True, device=True)
        return info

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
            torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()
    ctx.profile(True)
    launches0 = ctx.launch_count()
    clocks = ClockSampler(local)
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    nmv = 0
    infos = []
    marks = []  # events around each build: the build / solve split of the step
    for _ in range(args.steps):
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        ctx.build()
        b1.record(stream)
        om_last, _, _, info = ctx.solve(want_x=True, device=True)
        marks.append((b0, b1))
        nmv += info.nmatvec
        infos.append(info)
    t1.record(stream)
    barrier()
    clk = clocks.stop()
    om_last = om_last.cpu().numpy()
    ms = t0.elapsed_time(t1)
    launches = ctx.launch_count() - launches0
    prof = ctx.profile_get()
    ctx.profile(False)
    ms_max, nmv_all = reduce_over_ranks(ms, nmv, "cuda")

    # end to end through the C ABI with host buffers (H2D of C, eps; D2H of omega, X)
    e2e = None
    if not args.no_e2e:
        def host_step():
            ctx.set_orbitals(mol.C, mol.eps, mol.nocc)
            ctx.build()
            return ctx.solve(want_x=True, device=False)[3]
        host_step()
        barrier()
        e2e_steps = min(args.steps, E2E_STEPS)
        te0 = time.perf_counter()
        nmv_e = 0
        for _ in range(e2e_steps):
            nmv_e += host_step().nmatvec
        barrier()
        te = time.perf_counter() - te0
        te_max, nmv_e_all = reduce_over_ranks(te, nmv_e, "cuda")
        e2e = {"value": nmv_e_all / te_max, "unit": "matvecs/s",
               "h2d_bytes_per_step": int(mol.C.nbytes + mol.eps.nbytes),
               "d2h_bytes_per_step": int(8 * OPTS["nstates"] * (1 + d.nocc * d.nvir) + 8 * OPTS["nstates"]),
               "steps": e2e_steps}

    # the oracle's roots of this workload (stored by the golden script from the CPU oracle alone)
    gold = oracle_omega_200() if args.case == "full" else None
    # reduced-precision form on the same workload (NEXT: FP32 tensors, 3xTF32 K on tcgen05)
    mixed = fp64tc = None
    if not (args.no_mixed and args.no_fp64tc):
        om64 = fp64_reference_omega(tdarisp, mol, C_dev, eps_dev, stream)
        if not args.no_mixed:
            mixed = run_form(args, tdarisp, mol, C_dev, eps_dev, stream, barrier, 1, om64, gold)
        if not args.no_fp64tc:
            fp64tc = run_form(args, tdarisp, mol, C_dev, eps_dev, stream, barrier, 2, om64, gold)
    # the other configurations of the workload family (rank 0 of a single-GPU run)
    configs = spill = None
    if not args.no_configs and world == 1:
        configs = run_configs(args, tdarisp, stream)
        if args.case == "full":
            spill = spill_figures(tdarisp, mol, C_dev, eps_dev, stream)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    peaks = read_peaks()
    # dominant kernel by device time
    dom = max(prof.items(), key=lambda kv: kv[1]["ms"])
    name, p = dom
    achieved = p["flops"] / (p["ms"] * 1e-3) / 1e12
    fp64_peak = FP64_PEAK_TFLOPS
    traffic = None
    if name == "K_stage1" and p["launches"]:
        # DRAM bytes per launch: the DRAM/algorithmic byte ratio that one ncu capture of this
        # kernel measured on the 100-atom case, times the algorithmic bytes per launch
        traffic = K_STAGE1_TRAFFIC_RATIO * p["bytes"] / p["launches"]
    roof = {"kernel": name, "bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
            "frac": achieved / fp64_peak, "traffic": traffic, "traffic_unit": "bytes per launch",
            "algorithmic_bytes_per_launch": p["bytes"] / max(p["launches"], 1),
            "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz",
            "launches": p["launches"], "avg_launch_ms": p["ms"] / max(p["launches"], 1)}
    kernels = {k: {"ms": round(v["ms"], 3), "launches": v["launches"],
                   "share": round(v["ms"] / sum(x["ms"] for x in prof.values()), 4)}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])[:8]}
    # the oracle on the host cores: rank 0 at N = 1 only (at N > 1 the host cores are shared by the ranks)
    cpu = cpu_baseline(mol, d, nmv / max(args.steps, 1)) if not args.no_cpu and world == 1 else None
    if cpu is not None:
        # the same sample with 4 threads, the thread count of the paper's CPU runs (Sec. 4, Table 2)
        cpu["threads_4"] = cpu_baseline_threads(4, d, nmv / max(args.steps, 1), case=args.case)
    if configs and cpu and "config1_fp64_24atom" in configs:
        # the 24-atom FP64 solve against the oracle's whole solve of it, both measured
        c1, full = configs["config1_fp64_24atom"], cpu["full_24atom_measured"]
        c1["oracle_full_solve_s"] = full["s_to_states"]
        c1["speedup_vs_oracle_full_solve"] = full["s_to_states"] / c1["s_to_states"]
    mv_ms = sum(i.t_matvec_ms for i in infos)
    line = {
        "metric": METRIC, "value": nmv_all / (ms_max * 1e-3), "unit": "matvecs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD if args.case == "full" else "profiling case: 100-atom molecule, same options",
                   "natoms": int(len(mol.Z)), "nao": d.nao, "nocc": d.nocc,
                   "nvir": d.nvir, "naux_j": d.naux_j, "naux_k": d.naux_k, "nocc_k": d.nocc_k,
                   "nvir_k": d.nvir_k, "nstates": OPTS["nstates"], "block": OPTS["block"],
                   "tol": OPTS["tol"], "parallelism": "independent problems per GPU" if world > 1 else "1 GPU",
                   "l2": "working set larger than L2 (B tensors %.2f GB, V/W %.2f GB), no flush"
                         % (8e-9 * d.naux_j * d.nocc * d.nvir, 16e-9 * 300 * d.nocc * d.nvir)},
        "s_to_states": ms_max / args.steps * 1e-3,
        "build_s": sum(b0.elapsed_time(b1) for b0, b1 in marks) / args.steps * 1e-3,
        "matvec_only": {"value": nmv / (mv_ms * 1e-3) if mv_ms else None, "unit": "matvecs/s",
                        "note": "Davidson matvec time only (events around each block product)"},
        "davidson": {"niter": [i.niter for i in infos], "nmatvec": [i.nmatvec for i in infos],
                     "restarts": [i.nrestart for i in infos], "converged": [i.converged for i in infos]},
        "per_state_dOmega_vs_oracle_Ha": per_state_error(om_last, gold),
        "roofline": roof, "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e, "mixed_form": mixed,
        "fp64_tensor_core_form": fp64tc, "configs": configs, "spill": spill,
        "gpu_launches": launches, "clocks": clk,
    }
    for extra in (mixed, fp64tc):
        if extra:
            extra["speedup_vs_fp64_value"] = extra["value"] / line["value"]
            extra["speedup_vs_fp64_s_to_states"] = line["s_to_states"] / extra["s_to_states"]
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


# Peak FP64 arithmetic rate, the roofline denominator of the FP64 form:
# 152 SMs x 2 DFMA per clock per SM x 2 flops x 2.070 GHz (maximum SM clock).
# The per-SM rate of 2 DFMA per clock comes from a register-only FMA loop on
# GB300 (1186 GFLOP/s at 1987 MHz) and agrees with the nominal 1.25 TFLOP/s.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12

# DRAM bytes / algorithmic bytes of K stage 1, from one ncu capture of that kernel
# (737 MB measured for 708 MB algorithmic on the 100-atom profiling case).
K_STAGE1_TRAFFIC_RATIO = 737.0 / 708.0

# nominal dense TF32 / BF16 tensor rates of GB300 (1.1 and 2.25 PFLOP/s)
TF32_OVER_BF16 = 1.1 / 2.25


def fp64_reference_omega(tdarisp, mol, C_dev, eps_dev, stream):
    """Excitation energies of the FP64 form (the comparison for the other forms)."""
    ref = tdarisp.Context(stream=stream.cuda_stream, **OPTS)
    ref.set_molecule(mol.Z, mol.xyz, mol.aux_exp, mol.shells)
    ref.set_orbitals(C_dev, eps_dev, mol.nocc)
    ref.build()
    om64 = ref.solve(want_x=False)[0]
    ref.close()
    return om64


# at most this many steps of the host-buffer end-to-end leg (each repeats a whole step)
E2E_STEPS = 5

GOLDEN = os.path.join(ROOT, "tests", "golden")


def oracle_omega_200():
    """The 15 lowest roots of this workload from the CPU oracle's Davidson at
    residual 1e-7 (written by tests/golden/make_golden.py cfg2, which calls only
    the oracle)."""
    try:
        with open(os.path.join(GOLDEN, "omega_200atom_rsh.json")) as fh:
            return np.array(json.load(fh)["omega"])
    except (OSError, KeyError, ValueError):
        return None


def per_state_error(om, gold):
    """|Omega_k - Omega_k(oracle)| per state, Hartree (None without the oracle's values)."""
    if gold is None or om is None:
        return None
    n = min(len(om), len(gold))
    return [float(x) for x in np.abs(np.asarray(om)[:n] - gold[:n])]


FORMS = {
    1: dict(kind="reduced precision", products=3,
            dtype="f32/tf32x3 (tensor cores) + f64 (integrals, transforms, metrics, Davidson)",
            note="3 tensor products (hi*hi + hi*lo + lo*hi) per useful flop", peak="tf32"),
    2: dict(kind="FP64 on the tensor cores", products=28,
            dtype="f64 results; transforms, J and K as 7-slice Ozaki products on bf16 tensor cores",
            note="28 bf16 slice products (s + t < 7) per useful FP64 flop", peak="bf16"),
}


def run_form(args, tdarisp, mol, C_dev, eps_dev, stream, barrier, precision, om64, gold=None):
    """Same workload in another form (precision 1 or 2); compared with the FP64 form."""
    import torch
    form = FORMS[precision]
    ctx = tdarisp.Context(stream=stream.cuda_stream, precision=precision, **OPTS)
    ctx.set_molecule(mol.Z, mol.xyz, mol.aux_exp, mol.shells)
    ctx.set_orbitals(C_dev, eps_dev, mol.nocc)

    def step():
        ctx.build()
        return ctx.solve(want_x=True, device=True)

    for _ in range(max(args.warmup, 1)):
        step()
    barrier()
    # timed without the library's per-launch events (many short kernels in these forms);
    # one more step with them gives the kernel breakdown
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    nmv, infos, om = 0, [], None
    marks = []  # events after each build: the build / solve split of the step
    for _ in range(args.steps):
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        ctx.build()
        b1.record(stream)
        om, X, rs, info = ctx.solve(want_x=True, device=True)
        marks.append((b0, b1))
        nmv += info.nmatvec
        infos.append(info)
    t1.record(stream)
    barrier()
    ms = t0.elapsed_time(t1)
    build_ms = sum(b0.elapsed_time(b1) for b0, b1 in marks)
    ctx.profile(True)
    step()
    barrier()
    prof = ctx.profile_get()
    ctx.profile(False)
    ctx.close()
    om = om.cpu().numpy()
    peaks = read_peaks()
    bf16 = peaks.get("bf16_tflops") or 1900.0
    peak = bf16 * TF32_OVER_BF16 if form["peak"] == "tf32" else bf16
    peak_src = ("TF32 dense = measured bf16 burst x nominal TF32/BF16 ratio (1.1/2.25)" if form["peak"] == "tf32"
                else "measured bf16 burst (MEASURED_PEAKS.json)")
    name, p = max(((k, v) for k, v in prof.items() if k.endswith("_tc")), key=lambda kv: kv[1]["ms"])
    useful = p["flops"] / (p["ms"] * 1e-3) / 1e12
    mv_ms = sum(i.t_matvec_ms for i in infos)
    return {
        "form": form["kind"],
        "value": nmv / (ms * 1e-3), "unit": "matvecs/s", "s_to_states": ms / args.steps * 1e-3,
        "build_s": build_ms / args.steps * 1e-3, "solve_s": (ms - build_ms) / args.steps * 1e-3,
        "speedup_vs_fp64_value": None, "matvec_only": nmv / (mv_ms * 1e-3) if mv_ms else None,
        "dtype": form["dtype"],
        "max_abs_dOmega_vs_fp64_form_Ha": float(np.abs(om - om64).max()),
        "per_state_dOmega_vs_fp64_form_Ha": [float(x) for x in np.abs(om - om64)],
        "per_state_dOmega_vs_oracle_Ha": per_state_error(om, gold),
        "davidson": {"niter": [i.niter for i in infos], "nmatvec": [i.nmatvec for i in infos],
                     "ms_per_solve": {"matvec": statistics.mean(i.t_matvec_ms for i in infos),
                                      "orthogonalise": statistics.mean(i.t_ortho_ms for i in infos),
                                      "eigh": statistics.mean(i.t_eigh_ms for i in infos),
                                      "other": statistics.mean(i.t_other_ms for i in infos)}},
        "roofline": {"kernel": name, "bound": "tensor", "achieved": form["products"] * useful,
                     "useful_tflops": useful, "peak": peak, "unit": "TFLOP/s",
                     "frac": form["products"] * useful / peak, "peak_source": peak_src, "note": form["note"]},
        "kernels_one_step": {k: {"ms": round(v["ms"], 3), "launches": v["launches"]}
                             for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])[:16]},
    }


# ------------------------------------------------------------------ CPU oracle

def cpu_baseline(mol, d, nmv_per_step, budget_s=25.0, atoms=(1, 2), full_24=True):
    """Oracle on the host cores, bounded sample of the same workload: the oracle
    build for a subset of auxiliary functions (those of `atoms` heavy atoms) and
    its matvec on 2 vectors, both scaled linearly to the full auxiliary counts;
    one step = build + nmv matvecs.  With full_24, also the oracle's whole solve
    of the 24-atom configuration, measured (not extrapolated)."""
    from oracle import tda

    t_start = time.perf_counter()
    heavy = np.nonzero(mol.Z > 1)[0]
    res = []
    for nat in atoms:
        keep = np.zeros(len(mol.Z), dtype=bool)
        keep[heavy[:nat]] = True
        aux = np.where(keep, mol.aux_exp, 0.0)
        t0 = time.perf_counter()
        f = tda.build(mol.Z, mol.xyz, mol.shells, aux, mol.C, mol.eps, mol.nocc, OPTS["cx"],
                      OPTS["k_alpha"], OPTS["k_beta"], OPTS["omega"], OPTS["window_ev"])
        tb = time.perf_counter() - t0
        X = np.random.default_rng(0).normal(size=(2, d.nocc, d.nvir))
        t0 = time.perf_counter()
        tda.matvec(f, X)
        tm = (time.perf_counter() - t0) / 2
        res.append((nat, tb, tm))
        if time.perf_counter() - t_start > budget_s:
            break
    (n1, b1, m1), (n2, b2, m2) = res[0], res[-1]
    full = d.naux_k  # heavy atoms carrying aux functions
    if n2 == n1:
        tb_full, tm_full = b1 * full / n1, m1 * full / n1
    else:
        tb_full = b1 + (b2 - b1) * (full - n1) / (n2 - n1)
        tm_full = m1 + (m2 - m1) * (full - n1) / (n2 - n1)
    t_step = tb_full + nmv_per_step * tm_full
    threads = os.cpu_count()
    out = {"value": nmv_per_step / t_step, "unit": "matvecs/s", "cores": threads, "kind": "oracle",
           "sample": "oracle build and 2-vector matvec with the aux functions of %d and %d of the %d heavy "
                     "atoms, extrapolated linearly to all; one step = build + %d matvecs"
                     % (n1, n2, full, round(nmv_per_step)),
           "s_per_step_extrapolated": t_step, "wall_s": time.perf_counter() - t_start}
    if full_24:
        out["full_24atom_measured"] = oracle_full_24atom()
    return out


def oracle_full_24atom(repeats=5):
    """The oracle's whole TDA-risp solve of the 24-atom configuration (build and
    Davidson to 5 states, residual 1e-6, global hybrid), timed on the host cores:
    a full configuration measured, not extrapolated."""
    from oracle import tda
    from paper_2603_29257_gb300 import synth
    mol = synth.molecule_24()
    tb, ts, res = [], [], None
    for _ in range(repeats):
        t0 = time.perf_counter()
        f = tda.build(mol.Z, mol.xyz, mol.shells, mol.aux_exp, mol.C, mol.eps, mol.nocc, SMALL_OPTS["cx"],
                      SMALL_OPTS["k_alpha"], SMALL_OPTS["k_beta"], SMALL_OPTS["omega"], SMALL_OPTS["window_ev"])
        t1 = time.perf_counter()
        res = tda.solve(f, SMALL_OPTS["nstates"], block=2 * SMALL_OPTS["nstates"], tol=SMALL_OPTS["tol"])
        t2 = time.perf_counter()
        tb.append(t1 - t0)
        ts.append(t2 - t1)
    b, s_ = statistics.median(tb), statistics.median(ts)
    return {"workload": "24-atom molecule, global hybrid c_x 0.25, 40 eV window, 5 states, residual 1e-6",
            "build_s": b, "solve_s": s_, "s_to_states": b + s_, "matvecs_per_s": res.nmatvec / (b + s_),
            "nmatvec": int(res.nmatvec), "niter": int(res.niter), "repeats": repeats, "cores": os.cpu_count()}


def cpu_baseline_threads(nthreads, d, nmv_per_step, budget_s=20.0, timeout_s=240.0, case="full"):
    """cpu_baseline in a child process whose OpenMP and BLAS pools have nthreads
    threads (the pools are sized when the libraries load, hence the child); the
    child rebuilds the molecule of the same case as the parent."""
    env = dict(os.environ, OMP_NUM_THREADS=str(nthreads), OPENBLAS_NUM_THREADS=str(nthreads),
               MKL_NUM_THREADS=str(nthreads))
    code = ("import json, sys; from types import SimpleNamespace; sys.path.insert(0, %r); import bench; "
            "d = SimpleNamespace(**json.loads(sys.argv[1])); "
            "r = bench.cpu_baseline(bench.make_inputs(sys.argv[4]), d, float(sys.argv[2]), budget_s=float(sys.argv[3])); "
            "print(json.dumps(r))") % os.path.dirname(os.path.abspath(__file__))
    dims = json.dumps({"nocc": d.nocc, "nvir": d.nvir, "naux_k": d.naux_k})
    try:
        out = subprocess.run([sys.executable, "-c", code, dims, str(nmv_per_step), str(budget_s), case], env=env,
                             capture_output=True, text=True, timeout=timeout_s)
        r = json.loads(out.stdout.strip().splitlines()[-1])
        r["cores"] = nthreads
        return r
    except Exception as e:  # the headline line never depends on this context figure
        return {"unavailable": "%s: %s" % (type(e).__name__, str(e)[:200])}


def run_reference(args):
    rank, world, local = dist_info()
    if rank != 0:
        return
    import __graft_entry__
    from oracle import build as ob
    ob.build()
    mol = make_inputs()
    from paper_2603_29257_gb300 import synth  # noqa: F401

    class D:
        pass
    d = D()
    d.nocc, d.nvir = mol.nocc, mol.nvir
    d.naux_k = int(np.sum(mol.Z > 1))
    nmv = 259  # matvecs of one GPU solve of this workload (18 Davidson iterations; the count is method-determined)
    vals, walls = [], []
    for _ in range(args.warmup):
        cpu_baseline(mol, d, nmv, budget_s=60.0, full_24=False)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ts = time.perf_counter()
        vals.append(cpu_baseline(mol, d, nmv, budget_s=60.0, full_24=False))
        walls.append(time.perf_counter() - ts)
    wall = time.perf_counter() - t0
    v = statistics.median([x["value"] for x in vals])
    cb = dict(vals[-1])
    cb["value"] = v
    cb["full_24atom_measured"] = oracle_full_24atom()
    # a step of this arm is the bounded sample: ms_per_step is its measured wall
    # time; value is the sample's extrapolation to the whole 200-atom step
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "matvecs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(walls),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "step": cb["sample"]}, "cpu_baseline": cb,
            "s_per_full_step_extrapolated": statistics.median([x["s_per_step_extrapolated"] for x in vals]),
            "e2e": {"value": v, "unit": "matvecs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line))


def batched_molecules(count=64, seed0=1000, lo=20, hi=150):
    """64 seeded molecules with atom counts log-uniform in [20, 150]."""
    from paper_2603_29257_gb300 import synth
    out = []
    for s in range(seed0, seed0 + count):
        rng = np.random.default_rng(s)
        natoms = int(round(np.exp(rng.uniform(np.log(lo), np.log(hi)))))
        out.append(synth.molecule_by_atoms(s, natoms))
    return out


BATCH_OPTS = dict(cx=0.25, k_alpha=1.0, k_beta=0.0, omega=0.0, window_ev=40.0, nstates=10, tol=1e-5,
                  max_iter=200)


def run_matvec(args):
    """Block products alone (throughput of A X and the profiling case of the
    integral and diagonal kernels): tr_build once in the chosen form, then W
    untimed and K timed products of one block of `--block` resident seeded
    vectors.  value = block x K / event time; per kernel kind the library's
    CUDA-event time, algorithmic bytes and flops."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_29257_gb300 import tdarisp
    mol = make_inputs(args.case)
    torch.zeros(1, device="cuda")
    stream = torch.cuda.current_stream()
    C_dev = torch.from_numpy(mol.C).cuda()
    eps_dev = torch.from_numpy(mol.eps).cuda()
    ctx = tdarisp.Context(stream=stream.cuda_stream, **dict(OPTS, precision=args.precision, j_ao=args.j_ao))
    ctx.set_molecule(mol.Z, mol.xyz, mol.aux_exp, mol.shells)
    ctx.set_orbitals(C_dev, eps_dev, mol.nocc)
    ctx.profile(True)
    ctx.build()
    torch.cuda.synchronize()
    build_prof = ctx.profile_get()
    ctx.profile(False)
    d = ctx.dims()
    g = torch.Generator(device="cpu").manual_seed(17)
    X = torch.randn((args.block, d.nocc, d.nvir), generator=g, dtype=torch.float64).cuda()
    AX = torch.empty_like(X)
    for _ in range(max(args.warmup, 1)):
        ctx.matvec(X, out=AX)
    torch.cuda.synchronize()
    ctx.profile(True)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        ctx.matvec(X, out=AX)
    t1.record(stream)
    torch.cuda.synchronize()
    prof = ctx.profile_get()
    ctx.profile(False)
    ms = t0.elapsed_time(t1)

    def table(pr):
        return {k: {"ms": round(v["ms"], 3), "launches": v["launches"],
                    "gbs": round(v["bytes"] / (v["ms"] * 1e-3) / 1e9, 1) if v["ms"] and v["bytes"] else None,
                    "tflops": round(v["flops"] / (v["ms"] * 1e-3) / 1e12, 3) if v["ms"] and v["flops"] else None}
                for k, v in sorted(pr.items(), key=lambda kv: -kv[1]["ms"])[:12]}
    line = {"metric": "TDA-risp matvecs/s (block products alone)", "value": args.block * args.steps / (ms * 1e-3),
            "unit": "matvecs/s", "n_gpus": 1, "steps": args.steps, "warmup": max(args.warmup, 1),
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {0: "f64", 1: "f32/tf32x3 + f64", 2: "f64 (7-slice bf16 tensor-core products)"}[args.precision],
            "data": "synthetic",
            "config": {"workload": (WORKLOAD if args.case == "full" else "100-atom molecule, same options")
                       + "; one block of %d seeded vectors" % args.block,
                       "precision": args.precision, "j_ao": args.j_ao, "nao": d.nao, "nocc": d.nocc, "nvir": d.nvir,
                       "block": args.block,
                       "l2": "X and AX %.0f MB each" % (8e-6 * args.block * d.nocc * d.nvir)},
            "kernels": table(prof), "build_kernels": table(build_prof),
            "device_bytes": dict(zip(("held", "peak", "estimated_peak"), ctx.memory()))}
    print(json.dumps(line))


def run_tddft(args):
    """Full TDDFT-risp (tddft = 1, Sec. 2, Eqs. tddft and hessian) on the same
    molecule and options, in the form --precision (0 FP64 pipe, 2 FP64 on the
    tensor cores): tr_build (with T_ia^P' on the window), W untimed and
    K timed (A + B, A - B) products of one block of `--block` resident seeded
    vectors, then one Davidson solve to 15 states, and the TDA solve of the same
    context options for comparison.  value = vectors x K / event time of the
    block products (each vector gets both products)."""
    if args.precision == 1:
        sys.exit("tddft workload: full TDDFT-risp runs in the FP64 forms only (--precision 0 or 2)")
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_29257_gb300 import tdarisp
    mol = make_inputs(args.case)
    torch.zeros(1, device="cuda")
    stream = torch.cuda.current_stream()
    C_dev = torch.from_numpy(mol.C).cuda()
    eps_dev = torch.from_numpy(mol.eps).cuda()

    def context(tddft):
        c = tdarisp.Context(stream=stream.cuda_stream, **dict(OPTS, tddft=tddft, precision=args.precision))
        c.set_molecule(mol.Z, mol.xyz, mol.aux_exp, mol.shells)
        c.set_orbitals(C_dev, eps_dev, mol.nocc)
        return c
    ctx = context(1)
    torch.cuda.synchronize()
    tb = time.perf_counter()
    ctx.build()
    torch.cuda.synchronize()
    build_s = time.perf_counter() - tb
    d = ctx.dims()
    g = torch.Generator(device="cpu").manual_seed(17)
    X = torch.randn((args.block, d.nocc, d.nvir), generator=g, dtype=torch.float64).cuda()
    for _ in range(max(args.warmup, 1)):
        ctx.matvec_tddft(X)
    torch.cuda.synchronize()
    ctx.profile(True)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        ctx.matvec_tddft(X)
    t1.record(stream)
    torch.cuda.synchronize()
    prof = ctx.profile_get()
    ctx.profile(False)
    ms = t0.elapsed_time(t1)
    del X
    ts = time.perf_counter()
    om, _, _, rs, info = ctx.solve_tddft()
    solve_s = time.perf_counter() - ts
    mem = ctx.memory()
    del ctx
    tda_ctx = context(0)
    tda_ctx.build()
    ts = time.perf_counter()
    om_tda, _, _, info_tda = tda_ctx.solve(want_x=False)
    tda_s = time.perf_counter() - ts
    ev = 27.211386245988
    kern = {k: {"ms": round(v["ms"], 3), "launches": v["launches"],
                "tflops": round(v["flops"] / (v["ms"] * 1e-3) / 1e12, 3) if v["ms"] and v["flops"] else None,
                "gbs": round(v["bytes"] / (v["ms"] * 1e-3) / 1e9, 1) if v["ms"] and v["bytes"] else None}
            for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])[:10]}
    line = {"metric": "full TDDFT-risp (A+B, A-B) products/s (block products alone)",
            "value": args.block * args.steps / (ms * 1e-3), "unit": "vectors/s", "n_gpus": 1,
            "steps": args.steps, "warmup": max(args.warmup, 1), "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {0: "f64", 2: "f64 (7-slice bf16 tensor-core products)"}[args.precision], "data": "synthetic",
            "config": {"workload": (WORKLOAD if args.case == "full" else "100-atom molecule, same options")
                       .replace("TDA-risp", "full TDDFT-risp") + "; one block of %d seeded vectors" % args.block,
                       "precision": args.precision,
                       "nao": d.nao, "nocc": d.nocc, "nvir": d.nvir, "naux_k": d.naux_k, "nocc_k": d.nocc_k,
                       "nvir_k": d.nvir_k, "block": args.block,
                       "l2": "X and products %.0f MB each" % (8e-6 * args.block * d.nocc * d.nvir)},
            "kernels": kern,
            "solve": {"build_s": round(build_s, 3), "solve_s": round(solve_s, 3), "niter": info.niter,
                      "nmatvec": info.nmatvec, "nrestart": info.nrestart, "converged": info.converged,
                      "max_resid": float(np.max(rs)), "t_matvec_ms": round(info.t_matvec_ms, 1),
                      "omega_ev": [round(float(w) * ev, 6) for w in om[:5]]},
            "tda_solve": {"solve_s": round(tda_s, 3), "niter": info_tda.niter, "nmatvec": info_tda.nmatvec,
                          "omega_ev": [round(float(w) * ev, 6) for w in om_tda[:5]]},
            "device_bytes": dict(zip(("held", "peak", "estimated_peak"), mem))}
    print(json.dumps(line))


def batched_figures(tdarisp, stream, steps, warmup):
    """Batched form: 64 molecules (20-150 atoms, 10 states each) in the reduced-precision
    form, all Davidson solves advanced in lockstep with one graph launch of all
    products per step; against 64 sequential reduced-precision and 64 sequential
    plain FP64 solves.  Host wall clock with the device synchronised."""
    import torch
    t0 = time.perf_counter()
    mols = batched_molecules()
    gen_s = time.perf_counter() - t0

    def make(precision):
        cs = []
        for m in mols:
            c = tdarisp.Context(stream=stream.cuda_stream, precision=precision, **BATCH_OPTS)
            c.set_molecule_from(m)
            cs.append(c)
        return cs

    cs = make(1)
    for _ in range(max(warmup, 1)):
        tdarisp.build_batch(cs)
        tdarisp.solve_batch(cs, autotune=True)
    torch.cuda.synchronize()
    times, nmv_b, res_b, tb = [], 0, None, []
    for _ in range(max(steps, 1)):
        torch.cuda.synchronize()
        t = time.perf_counter()
        tdarisp.build_batch(cs)
        torch.cuda.synchronize()
        tb.append(time.perf_counter() - t)
        res_b = tdarisp.solve_batch(cs, autotune=True)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t)
        nmv_b = sum(r[3].nmatvec for r in res_b)
    t_batch = statistics.median(times)
    t_build = statistics.median(tb)
    for c in cs:
        c.close()
    # sequential, reduced precision
    cs = make(1)
    torch.cuda.synchronize()
    t = time.perf_counter()
    nmv_m, om_m = 0, []
    for c in cs:
        c.build()
        om, X, rs, info = c.solve(want_x=True)
        nmv_m += info.nmatvec
        om_m.append(om)
    torch.cuda.synchronize()
    t_seq_mixed = time.perf_counter() - t
    for c in cs:
        c.close()
    # sequential, plain FP64
    cs = make(0)
    torch.cuda.synchronize()
    t = time.perf_counter()
    nmv_f, om_f = 0, []
    for c in cs:
        c.build()
        om, X, rs, info = c.solve(want_x=True)
        nmv_f += info.nmatvec
        om_f.append(om)
    torch.cuda.synchronize()
    t_seq_fp64 = time.perf_counter() - t
    for c in cs:
        c.close()
    dmax = max(float(np.abs(r[0] - o).max()) for r, o in zip(res_b, om_f))
    dalone = max(float(np.abs(r[0] - o).max()) for r, o in zip(res_b, om_m))
    natoms = [len(m.Z) for m in mols]
    return {"workload": "64 seeded molecules (seeds 1000-1063), atoms log-uniform 20-150 "
                        "(%d-%d, %d total), 10 states each, global hybrid c_x 0.25, 40 eV window, "
                        "tol 1e-5, reduced precision" % (min(natoms), max(natoms), sum(natoms)),
            "timing": "host wall clock around the build of all 64 contexts + tr_solve_batch, device synchronised",
            "steps": max(steps, 1), "warmup": max(warmup, 1),
            "value": nmv_b / t_batch, "unit": "matvecs/s",
            "batched_s": t_batch, "batched_build_s": t_build, "batched_solve_s": t_batch - t_build,
            "sequential_mixed_s": t_seq_mixed, "sequential_fp64_s": t_seq_fp64,
            "speedup_vs_sequential_fp64": t_seq_fp64 / t_batch,
            "speedup_vs_sequential_mixed": t_seq_mixed / t_batch,
            "matvecs": {"batched": nmv_b, "sequential_mixed": nmv_m, "sequential_fp64": nmv_f},
            "max_abs_dOmega_vs_fp64_Ha": dmax, "max_abs_dOmega_vs_alone_Ha": dalone, "generation_s": gen_s}


def run_batched(args):
    """--workload batched: the batched-form figures as a line of their own."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_29257_gb300 import tdarisp
    torch.zeros(1, device="cuda")
    f = batched_figures(tdarisp, torch.cuda.current_stream(), args.steps, args.warmup)
    line = {"metric": "TDA-risp matvecs/s, batched form (64 molecules, build + solve)",
            "value": f["value"], "unit": "matvecs/s", "n_gpus": 1, "steps": f["steps"],
            "warmup": f["warmup"], "ms_per_step": 1e3 * f["batched_s"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32/tf32x3 + f64", "data": "synthetic",
            "config": {"workload": f["workload"], "timing": f["timing"]}}
    line.update({k: v for k, v in f.items() if k not in ("workload", "timing", "value", "unit", "steps", "warmup")})
    print(json.dumps(line))


def spill_figures(tdarisp, mol, C_dev, eps_dev, stream, dev_rows=60):
    """Host placement of the Davidson vectors (Sec. 3.3): the pinned host link
    probed with plain copies (1 GiB each way, CUDA events), then the 200-atom
    reduced-precision solve with all V/W rows in HBM and with only dev_rows of
    them there (the rest in pinned host memory, streamed through two staging
    slots on a copy stream): bytes moved, both solve times, the moved bytes per
    second of the spilled solve, and the roots' agreement."""
    import torch
    n = 1 << 27  # doubles: 1 GiB
    h = torch.empty(n, dtype=torch.float64, pin_memory=True)
    d = torch.empty(n, dtype=torch.float64, device="cuda")
    probe = {}
    for name, dst, src in (("h2d_gbs", d, h), ("d2h_gbs", h, d)):
        for _ in range(2):
            dst.copy_(src, non_blocking=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        cs = torch.cuda.current_stream()
        e0.record(cs)
        for _ in range(5):
            dst.copy_(src, non_blocking=True)
        e1.record(cs)
        torch.cuda.synchronize()
        probe[name] = 5 * 8.0 * n / (e0.elapsed_time(e1) * 1e-3) / 1e9
    del h, d
    out = {"link_probe": probe, "probe": "1 GiB pinned host <-> device copies, 5 each way, CUDA events"}
    for key, rows in (("all_rows_on_device", 0), ("rows_on_device_%d" % dev_rows, dev_rows)):
        ctx = tdarisp.Context(stream=stream.cuda_stream, precision=1, dav_dev_rows=rows, **OPTS)
        ctx.set_molecule(mol.Z, mol.xyz, mol.aux_exp, mol.shells)
        ctx.set_orbitals(C_dev, eps_dev, mol.nocc)
        ctx.build()
        ctx.solve(want_x=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        om, _, _, info = ctx.solve(want_x=False)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        ctx.close()
        out[key] = {"solve_s": dt, "dev_rows": info.dev_rows, "max_space": info.max_space,
                    "host_bytes_moved": int(info.host_bytes_moved), "nmatvec": info.nmatvec,
                    "host_gb_per_solve_s": info.host_bytes_moved / dt / 1e9,
                    "omega_Ha": [float(x) for x in om]}
    a, b = out["all_rows_on_device"], out["rows_on_device_%d" % dev_rows]
    out["max_abs_dOmega_spilled_vs_resident_Ha"] = max(abs(x - y) for x, y in zip(a["omega_Ha"], b["omega_Ha"]))
    return out


# the 24-atom molecule: global hybrid, 5 states to residual 1e-6
SMALL_OPTS = dict(cx=0.25, k_alpha=1.0, k_beta=0.0, omega=0.0, window_ev=40.0, nstates=5, tol=1e-6,
                  max_iter=200)


def small_form(tdarisp, stream, mol, precision, gold, steps, warmup):
    """Build + solve of the 24-atom molecule in one form, timed with CUDA events
    over `steps` whole steps; per-state error against the oracle's dense roots."""
    import torch
    from paper_2603_29257_gb300 import synth
    ctx = tdarisp.Context(stream=stream.cuda_stream, precision=precision, **SMALL_OPTS)
    ctx.set_molecule_from(mol)
    for _ in range(max(warmup, 1)):
        ctx.build()
        ctx.solve(want_x=True, device=True)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    nmv, infos, om = 0, [], None
    for _ in range(steps):
        ctx.build()
        om, X, rs, info = ctx.solve(want_x=True, device=True)
        nmv += info.nmatvec
        infos.append(info)
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    # the block product alone: 10 products of one block of 10 seeded vectors
    d = ctx.dims()
    X = torch.from_numpy(synth.random_trial_block(5, 10, d.nocc, d.nvir)).cuda()
    AX = torch.empty_like(X)
    for _ in range(3):
        ctx.matvec(X, out=AX)
    torch.cuda.synchronize()
    m0 = torch.cuda.Event(enable_timing=True)
    m1 = torch.cuda.Event(enable_timing=True)
    m0.record(stream)
    for _ in range(10):
        ctx.matvec(X, out=AX)
    m1.record(stream)
    torch.cuda.synchronize()
    mv_ms = m0.elapsed_time(m1)
    ctx.close()
    om = om.cpu().numpy()
    err = np.abs(om - gold)
    return {"value": nmv / (ms * 1e-3), "unit": "matvecs/s", "s_to_states": ms / steps * 1e-3,
            "steps": steps, "warmup": max(warmup, 1),
            "niter": [i.niter for i in infos][-1], "nmatvec": [i.nmatvec for i in infos][-1],
            "block_products_alone": {"value": 100 / (mv_ms * 1e-3), "unit": "matvecs/s",
                                     "note": "10 products of one block of 10 resident vectors"},
            "per_state_dOmega_vs_oracle_Ha": [float(x) for x in err],
            "max_abs_dOmega_vs_oracle_Ha": float(err.max()), "omega_Ha": [float(x) for x in om]}


def run_configs(args, tdarisp, stream):
    """The other configurations of the workload family, each reported beside the
    headline: the 24-atom molecule in the FP64 form (config 1) and in the
    reduced-precision and tensor-core forms (config 3), and the batched form of
    64 molecules (config 4)."""
    from paper_2603_29257_gb300 import synth
    out = {}
    mol = synth.molecule_24()
    with open(os.path.join(GOLDEN, "omega_24atom.json")) as fh:
        gold = np.array(json.load(fh)["cases"]["hybrid"]["omega"])
    desc = ("24-atom seeded molecule (10 C/N/O + 14 H, nao 210, nocc 42), global hybrid c_x 0.25, 40 eV "
            "window, 5 states, residual 1e-6; per-state error against the oracle's dense eigh")
    f64 = small_form(tdarisp, stream, mol, 0, gold, SMALL_STEPS, 2)
    out["config1_fp64_24atom"] = dict(workload=desc, dtype="f64", **f64)
    c3 = {"workload": desc}
    for precision, key in ((1, "reduced_precision"), (2, "fp64_tensor_cores")):
        r = small_form(tdarisp, stream, mol, precision, gold, SMALL_STEPS, 2)
        r["dtype"] = FORMS[precision]["dtype"]
        r["speedup_vs_fp64_s_to_states"] = f64["s_to_states"] / r["s_to_states"]
        r["speedup_vs_fp64_value"] = r["value"] / f64["value"]
        c3[key] = r
    out["config3_forms_24atom"] = c3
    if not args.no_batched:
        out["config4_batched"] = batched_figures(tdarisp, stream, 1, 1)
    if not args.no_serve:
        out["config5_serve"] = serve_figures(tdarisp, SERVE_REQUESTS, 1, loads=(0.7,))
    return out


# requests of the serving form in the default run (the offered load 0.7 and saturated)
SERVE_REQUESTS = 40


# whole build + solve steps of the 24-atom configurations
SMALL_STEPS = 20


SERVE_OPTS = dict(cx=0.25, k_alpha=1.0, k_beta=0.0, omega=0.0, window_ev=40.0, tol=1e-5, max_iter=200)


def serve_stream(count, seed0=5000, arrival_seed=5001, lo=30, hi=600, large=0, large_atoms=1500):
    """Seeded request stream: molecule k from seed seed0+k with atoms log-uniform in
    [lo, hi] (the last `large` requests, placed at seeded positions, have
    large_atoms atoms); states U{5..15} and unit-rate exponential gaps from
    arrival_seed.  Molecules above synth.LARGE_ATOMS atoms get their dense linear
    algebra on the GPU."""
    from paper_2603_29257_gb300 import synth
    rng = np.random.default_rng(arrival_seed)
    nst = rng.integers(5, 16, size=count)
    gaps = rng.exponential(1.0, size=count)
    big = set(int(x) for x in rng.choice(count, size=min(large, count), replace=False)) if large else set()
    mols = []
    for k in range(count):
        r = np.random.default_rng(seed0 + k)
        natoms = int(round(np.exp(r.uniform(np.log(lo), np.log(hi)))))
        if k in big:
            natoms = large_atoms
        mols.append(synth.molecule_by_atoms(seed0 + k, natoms, device="auto"))
    return mols, [int(n) for n in nst], np.cumsum(gaps) - gaps[0]


def _replay(tdarisp, mols, nst, arrivals, precision, max_active, build_threads):
    """Submit request k at arrivals[k] seconds (server clock), collect every result."""
    with tdarisp.Server(max_active=max_active, autotune=True, build_threads=build_threads) as srv:
        t0 = srv.clock()
        ids = {}
        for k, (m, n) in enumerate(zip(mols, nst)):
            wait = t0 + arrivals[k] - srv.clock()
            if wait > 0:
                time.sleep(wait)
            ids[srv.submit(m, precision=precision, nstates=n, **SERVE_OPTS)] = k
        res = srv.drain()
    out = [None] * len(mols)
    for r in res:
        if r["status"] != 0:
            raise RuntimeError("request %d failed: %s" % (ids[r["id"]], r["error"]))
        out[ids[r["id"]]] = r
    lat = np.array([r["t_done"] - r["t_submit"] for r in out])
    span = max(r["t_done"] for r in out) - min(r["t_submit"] for r in out)
    return out, {"p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                 "mean_ms": 1e3 * float(lat.mean()), "molecules_per_s": len(out) / span, "span_s": span,
                 "matvecs": int(sum(r["nmatvec"] for r in out)), "j_ao_requests": int(sum(r["j_ao"] for r in out))}


def serve_figures(tdarisp, requests, warmup, loads=(0.3, 0.7, 0.9), fp64_subsample=8, fp64_max_atoms=150,
                  hi=600, large=0, large_atoms=1500):
    """Serving form: a seeded Poisson stream of requests served by the continuous-
    batching server in the reduced-precision form at offered loads rho (rate x mean
    service time of a request served alone) and saturated (all at once); against the
    plain FP64 form served one request at a time on a seeded subsample of the
    requests with at most fp64_max_atoms atoms (the FP64 form grows as N^4: about
    12 s at 200 atoms)."""
    t = time.perf_counter()
    mols, nst, unit_gaps = serve_stream(requests, hi=hi, large=large, large_atoms=large_atoms)
    gen_s = time.perf_counter() - t
    R = len(mols)
    natoms = np.array([len(m.Z) for m in mols])
    # warm-up: module loading, kernel attributes, graph paths
    small = [k for k in range(R) if natoms[k] <= 150][:4]
    for _ in range(max(warmup, 1)):
        _replay(tdarisp, [mols[k] for k in small], [nst[k] for k in small], np.zeros(len(small)), 1, 64, 4)
    # service time of each request served alone (reduced precision)
    alone = []
    with tdarisp.Server(max_active=64, autotune=True) as srv:
        for m, n in zip(mols, nst):
            srv.submit(m, precision=1, nstates=n, **SERVE_OPTS)
            r = srv.drain()[0]
            alone.append(r["t_done"] - r["t_submit"])
    s_mean = float(np.mean(alone))
    out_loads = {}
    ref = None
    for rho in loads:
        res, st = _replay(tdarisp, mols, nst, unit_gaps * s_mean / rho, 1, 64, 4)
        st["lambda_per_s"] = rho / s_mean
        out_loads[str(rho)] = st
        ref = ref or res
    res_sat, sat = _replay(tdarisp, mols, nst, np.zeros(R), 1, 64, 4)
    # plain FP64 form one request at a time (saturated) on a seeded subsample
    pool = [k for k in range(R) if natoms[k] <= fp64_max_atoms]
    pick = sorted(int(x) for x in np.random.default_rng(5002).choice(pool, size=min(fp64_subsample, len(pool)),
                                                                         replace=False))
    res_f, fsat = _replay(tdarisp, [mols[k] for k in pick], [nst[k] for k in pick], np.zeros(len(pick)), 0, 1, 1)
    dmax = max(float(np.abs(res_sat[k]["omega"] - f["omega"]).max()) for k, f in zip(pick, res_f))
    if ref is not None:
        dmax = max(dmax, max(float(np.abs(ref[k]["omega"] - f["omega"]).max()) for k, f in zip(pick, res_f)))
    # the same subsample through the server in the reduced-precision form, one at a time
    _, msub = _replay(tdarisp, [mols[k] for k in pick], [nst[k] for k in pick], np.zeros(len(pick)), 1, 1, 1)
    return {"workload": "%d seeded requests (molecule seeds 5000-%d, arrival seed 5001), atoms log-uniform "
                        "30-%d (%d-%d, median %d)%s, states U{5..15}, global hybrid c_x 0.25, 40 eV window, "
                        "tol 1e-5; Poisson arrivals at load rho = lambda x mean service time alone"
                        % (R, 5000 + R - 1, hi, natoms.min(), natoms.max(), int(np.median(natoms)),
                           (", %d of %d atoms" % (large, large_atoms)) if large else ""),
            "timing": "server clock (host steady clock) from submit to result posted",
            "requests": R, "natoms": [int(x) for x in natoms], "nstates": nst,
            "service_alone_mean_ms": 1e3 * s_mean, "service_alone_max_ms": 1e3 * float(np.max(alone)),
            "loads": out_loads, "saturated": sat,
            "fp64_one_at_a_time": {"subsample": pick, "saturated": fsat,
                                   "reduced_precision_one_at_a_time": msub},
            "throughput_vs_fp64_one_at_a_time_on_subsample": msub["molecules_per_s"] / fsat["molecules_per_s"],
            "max_abs_dOmega_vs_fp64_Ha": dmax, "generation_s": gen_s}


def run_serve(args):
    """--workload serve: the serving figures as a line of their own."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_29257_gb300 import tdarisp
    torch.zeros(1, device="cuda")
    f = serve_figures(tdarisp, args.requests, args.warmup, hi=args.serve_max_atoms, large=args.serve_large,
                      large_atoms=args.serve_large_atoms)
    key = "0.7" if "0.7" in f["loads"] else sorted(f["loads"])[0]
    line = {"metric": "TDA-risp serve p50/p99 ms @1e-5 Ha and molecules/s, serving form",
            "value": f["loads"][key]["p99_ms"], "unit": "ms (p99 latency at load %s)" % key, "n_gpus": 1,
            "steps": 1, "warmup": max(args.warmup, 1), "ms_per_step": 1e3 * f["loads"][key]["span_s"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32/tf32x3 + f64",
            "data": "synthetic", "config": {"workload": f["workload"], "timing": f["timing"]}}
    line.update({k: v for k, v in f.items() if k not in ("workload", "timing")})
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-mixed", action="store_true", help="skip the reduced-precision form")
    ap.add_argument("--no-fp64tc", action="store_true", help="skip the FP64 form on the tensor cores")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other configurations (24-atom forms, batched, serving) of the default run")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched form in the default run")
    ap.add_argument("--workload", default="fp64-200", choices=["fp64-200", "batched", "serve", "matvec", "tddft"],
                    help="batched: 64 molecules in the reduced-precision batched form; "
                         "serve: a Poisson request stream through the serving runtime; "
                         "matvec: block products alone in the form --precision (profiling case); "
                         "tddft: full TDDFT-risp products and solve")
    ap.add_argument("--requests", type=int, default=64, help="requests of the serve workload")
    ap.add_argument("--serve-max-atoms", type=int, default=600, help="largest molecule of the serve request sizes")
    ap.add_argument("--serve-large", type=int, default=0, help="requests of --serve-large-atoms atoms in the stream")
    ap.add_argument("--serve-large-atoms", type=int, default=1500, help="atoms of the large serve requests")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving form in the default run")
    ap.add_argument("--precision", type=int, default=0, choices=[0, 1, 2],
                    help="form of the matvec and tddft workloads: 0 FP64, 1 reduced precision (matvec only), "
                         "2 FP64 on the tensor cores")
    ap.add_argument("--block", type=int, default=30, help="vectors per block of the matvec and tddft workloads")
    ap.add_argument("--j-ao", type=int, default=0, choices=[0, 1],
                    help="matvec workload: Coulomb term from the stored (P|ia) (0) or on the fly in the AO basis (1)")
    ap.add_argument("--case", default="full", choices=["full", "small"],
                    help="small: 100-atom molecule of the same shape, for profiler captures")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "matvec":
        run_matvec(args)
    elif args.workload == "tddft":
        run_tddft(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
