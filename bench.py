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
    for _ in range(args.steps):
        info = step()
        nmv += info.nmatvec
        infos.append(info)
    t1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = t0.elapsed_time(t1)
    launches = ctx.launch_count() - launches0
    prof = ctx.profile_get()
    ctx.profile(False)
    tot = torch.tensor([ms, float(nmv)], dtype=torch.float64, device="cuda")
    if world > 1:
        mx = tot.clone()
        dist.all_reduce(mx[:1], op=dist.ReduceOp.MAX)
        dist.all_reduce(tot[1:], op=dist.ReduceOp.SUM)
        ms_max, nmv_all = float(mx[0]), float(tot[1])
    else:
        ms_max, nmv_all = ms, float(nmv)

    # end to end through the C ABI with host buffers (H2D of C, eps; D2H of omega, X)
    e2e = None
    if not args.no_e2e:
        def host_step():
            ctx.set_orbitals(mol.C, mol.eps, mol.nocc)
            ctx.build()
            return ctx.solve(want_x=True, device=False)[3]
        host_step()
        barrier()
        te0 = time.perf_counter()
        nmv_e = 0
        for _ in range(args.steps):
            nmv_e += host_step().nmatvec
        barrier()
        te = time.perf_counter() - te0
        nmv_e_all = nmv_e * world
        e2e = {"value": nmv_e_all / te, "unit": "matvecs/s",
               "h2d_bytes_per_step": int(mol.C.nbytes + mol.eps.nbytes),
               "d2h_bytes_per_step": int(8 * OPTS["nstates"] * (1 + d.nocc * d.nvir) + 8 * OPTS["nstates"])}

    # reduced-precision form on the same workload (NEXT: FP32 tensors, 3xTF32 K on tcgen05)
    mixed = None
    if not args.no_mixed:
        mixed = run_mixed(args, tdarisp, mol, C_dev, eps_dev, stream, barrier)
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
        # DRAM bytes per launch: the measured/algorithmic ratio of the ncu capture of this
        # kernel (profiles/k_stage1_fp64_100atom.md) times the algorithmic bytes per launch
        traffic = K_STAGE1_TRAFFIC_RATIO * p["bytes"] / p["launches"]
    roof = {"kernel": name, "bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
            "frac": achieved / fp64_peak, "traffic": traffic, "traffic_unit": "bytes per launch",
            "algorithmic_bytes_per_launch": p["bytes"] / max(p["launches"], 1),
            "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz",
            "launches": p["launches"], "avg_launch_ms": p["ms"] / max(p["launches"], 1)}
    kernels = {k: {"ms": round(v["ms"], 3), "launches": v["launches"],
                   "share": round(v["ms"] / sum(x["ms"] for x in prof.values()), 4)}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])[:8]}
    cpu = cpu_baseline(mol, d, nmv / max(args.steps, 1)) if not args.no_cpu else None
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
        "matvec_only": {"value": nmv / (mv_ms * 1e-3) if mv_ms else None, "unit": "matvecs/s",
                        "note": "Davidson matvec time only (events around each block product)"},
        "davidson": {"niter": [i.niter for i in infos], "nmatvec": [i.nmatvec for i in infos],
                     "restarts": [i.nrestart for i in infos], "converged": [i.converged for i in infos]},
        "roofline": roof, "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e, "mixed_form": mixed,
        "gpu_launches": launches, "clocks": clk,
    }
    if mixed:
        mixed["speedup_vs_fp64_value"] = mixed["value"] / line["value"]
        mixed["speedup_vs_fp64_s_to_states"] = line["s_to_states"] / mixed["s_to_states"]
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


def run_mixed(args, tdarisp, mol, C_dev, eps_dev, stream, barrier):
    """Same workload in the reduced-precision form; compared with the FP64 form."""
    import torch
    ref = tdarisp.Context(stream=stream.cuda_stream, **OPTS)
    ref.set_molecule(mol.Z, mol.xyz, mol.aux_exp, mol.shells)
    ref.set_orbitals(C_dev, eps_dev, mol.nocc)
    ref.build()
    om64 = ref.solve(want_x=False)[0]
    ref.close()
    ctx = tdarisp.Context(stream=stream.cuda_stream, precision=1, **OPTS)
    ctx.set_molecule(mol.Z, mol.xyz, mol.aux_exp, mol.shells)
    ctx.set_orbitals(C_dev, eps_dev, mol.nocc)

    def step():
        ctx.build()
        return ctx.solve(want_x=True, device=True)

    for _ in range(max(args.warmup, 1)):
        step()
    barrier()
    ctx.profile(True)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    nmv, infos, om = 0, [], None
    for _ in range(args.steps):
        om, X, rs, info = step()
        nmv += info.nmatvec
        infos.append(info)
    t1.record(stream)
    barrier()
    ms = t0.elapsed_time(t1)
    prof = ctx.profile_get()
    ctx.close()
    om = om.cpu().numpy()
    peaks = read_peaks()
    bf16 = peaks.get("bf16_tflops")
    tf32_peak = bf16 * TF32_OVER_BF16 if bf16 else 1900.0 * TF32_OVER_BF16
    name, p = max(((k, v) for k, v in prof.items() if k.endswith("_tc")), key=lambda kv: kv[1]["ms"])
    useful = p["flops"] / (p["ms"] * 1e-3) / 1e12
    mv_ms = sum(i.t_matvec_ms for i in infos)
    return {
        "value": nmv / (ms * 1e-3), "unit": "matvecs/s", "s_to_states": ms / args.steps * 1e-3,
        "speedup_vs_fp64_value": None, "matvec_only": nmv / (mv_ms * 1e-3) if mv_ms else None,
        "dtype": "f32/tf32x3 (tensor cores) + f64 (integrals, transforms, metrics, Davidson)",
        "max_abs_dOmega_vs_fp64_form_Ha": float(np.abs(om - om64).max()),
        "per_state_dOmega_vs_fp64_form_Ha": [float(x) for x in np.abs(om - om64)],
        "davidson": {"niter": [i.niter for i in infos], "nmatvec": [i.nmatvec for i in infos]},
        "roofline": {"kernel": name, "bound": "tensor", "achieved": 3.0 * useful, "useful_tflops": useful,
                     "peak": tf32_peak, "unit": "TFLOP/s", "frac": 3.0 * useful / tf32_peak,
                     "peak_source": "TF32 dense = measured bf16 burst x nominal TF32/BF16 ratio (1.1/2.25)",
                     "note": "3 tensor products (hi*hi + hi*lo + lo*hi) per useful flop"},
        "kernels": {k: {"ms": round(v["ms"], 3), "launches": v["launches"]}
                    for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])[:8]},
    }


# ------------------------------------------------------------------ CPU oracle

def cpu_baseline(mol, d, nmv_per_step, budget_s=25.0):
    """Oracle on the host cores, bounded sample of the same workload: the oracle
    build for a subset of auxiliary functions and its matvec on 2 vectors, both
    scaled linearly to the full auxiliary counts; one step = build + nmv matvecs."""
    from oracle import tda

    t_start = time.perf_counter()
    heavy = np.nonzero(mol.Z > 1)[0]
    res = []
    for nat in (2, 4):
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
    return {"value": nmv_per_step / t_step, "unit": "matvecs/s", "cores": threads, "kind": "oracle",
            "sample": "oracle build and 2-vector matvec with the aux functions of %d and %d of the %d heavy "
                      "atoms, extrapolated linearly to all; one step = build + %d matvecs"
                      % (n1, n2, full, round(nmv_per_step)),
            "s_per_step_extrapolated": t_step, "wall_s": time.perf_counter() - t_start}


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
    nmv = 330  # matvecs of one GPU solve of this workload (the Davidson count is method-determined)
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(mol, d, nmv, budget_s=5.0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(mol, d, nmv, budget_s=5.0))
    wall = time.perf_counter() - t0
    v = statistics.median([x["value"] for x in vals])
    cb = dict(vals[-1])
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "matvecs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * nmv / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD}, "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "matvecs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}
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
    ap.add_argument("--case", default="full", choices=["full", "small"],
                    help="small: 100-atom molecule of the same shape, for profiler captures")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
