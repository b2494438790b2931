#!/usr/bin/env python
"""Benchmark of the SPH hot path on GB300: particle-neighbour interactions/s
and SPH steps/s, learned-h vs plain-h, on the Sedov blast workload (64^3 =
262,144 particles, Wendland C2, eta = 1.2, h-rho iteration to 1e-6, Monaghan
viscosity alpha = 1, beta = 2, FP64, fixed step).

One timed step = one kick-drift-kick sph_step: tree (keys, sort, permute,
leaves), h-predictor inference and one online training round, h-rho sweeps,
forces, kicks, FP64 totals.  Inputs are resident in HBM; L2 is flushed (a
256 MB write) between timed steps and each step is bracketed by CUDA events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl sph|reference]

--impl reference times the plain FP64 CPU oracle (brute-force neighbours) on
the host cores on a bounded sample of the same workload.  With N > 1 (torchrun)
every rank runs an independent replica (the method is not sharded here).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-neighbor interactions/s and SPH steps/s (learned-h vs plain-h, same GPU)"
UNIT = "interactions/s"
# algorithmic FP64 flops per accepted pair, counted from the pair arithmetic of
# the density sweep and of the force pass (FMA = 2, sqrt/div = 1)
F_DENSITY = 28
F_FORCE = 96
# Peaks derived from unit counts and the 2.07 GHz maximum SM clock (152 SMs):
# FP64 pipe 2 DFMA lanes/clk/SM; FP32 pipe 128 lanes/clk/SM.  The FP64 mode
# evaluates its pair terms in double-float on the FP32 pipe, where one FP64
# multiply-add (2 flops) costs 18 FP32 instructions (df_mul 7 + df_add 11), so
# its ceiling in FP64-accurate flops is 152 * 128 * 2.07e9 * 2 / 18.
FP64_PIPE_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# DRAM bytes per launch of the dominant kernel from one ncu capture (see
# profiles/), with the hash of the sources it was taken on
TRAFFIC = {
    # k_forces_df on the Sedov 64^3 step (profiles/k_forces_df_sedov64_fp64.md):
    # 81.07 MB read + 3.14 MB written
    "forces_fp64_sedov": {"bytes_per_launch": 84208896, "src": "29a20052c842",
                          "files": ["forces.cu", "dfloat.cuh", "sph_internal.cuh"]},
}
FP32_PIPE_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
DF_EMULATED_TFLOPS = 152 * 128 * 2.07e9 * 2 / 18 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sph", choices=["sph", "reference"])
    ap.add_argument("--n-side", type=int, default=None,
                    help="lattice side of the sedov (default 64, the headline workload) and turbulence (default 256) "
                         "workloads; smaller sides serve profiling captures")
    ap.add_argument("--workload", default="sedov", choices=["sedov", "polytrope", "collision", "turbulence", "sod"],
                    help="sedov: 64^3 FP64 (headline); polytrope 2^20, collision 2x2^21, turbulence 256^3: "
                         "FP32 pairs on FP64 positions; sod: the 1D shock tube, 10,000 particles in the tube, FP64")
    ap.add_argument("--curve", default="morton", choices=["morton", "hilbert"],
                    help="space-filling curve of the particle keys (Sec. 2.1, Tree topology)")
    ap.add_argument("--train-steps", type=int, default=16)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


# ------------------------------------------------------------------ distributed
def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def whole_job(times, units, device="cpu"):
    """Whole-job figures of N replicas: the maximum over ranks of each time
    and the sum over ranks of each unit count (one all-reduce each, on the
    process group's backend); the values themselves on one rank."""
    import torch
    import torch.distributed as dist
    mx = torch.tensor(times, dtype=torch.float64, device=device)
    sm = torch.tensor(units, dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return [float(v) for v in mx.cpu()], [float(v) for v in sm.cpu()]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.tmp = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", gpu_id, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = [r.split(",") for r in self.tmp.read().strip().splitlines() if r.strip()]
        os.unlink(self.tmp.name)
        sm = [float(r[0]) for r in rows if len(r) >= 8 and r[0].strip().replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if len(r) >= 8 and r[1].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows if len(r) >= 8 for k in range(4) if "Active" in r[4 + k]
                          and "Not" not in r[4 + k]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ GPU arm
def make_workload(args):
    from paper_2007_03097_gb300 import inputs
    if args.workload == "sedov":
        return inputs.sedov(args.n_side or 64)
    if args.workload == "polytrope":
        return inputs.polytrope(1 << 20)
    if args.workload == "collision":
        return inputs.collision(1 << 21)
    if args.workload == "sod":
        return inputs.sod(10000)
    return inputs.turbulence(args.n_side or 256)


def workload_label(args, w):
    if args.workload == "sedov":
        return (f"sedov blast {args.n_side or 64}^3 = {w.n} particles, Wendland C2, eta 1.2, h_tol 1e-6, "
                f"alpha 1 beta 2, FP64, fixed dt {w.dt:.3e}")
    if args.workload == "polytrope":
        return f"n=1 polytrope, {w.n} particles, Wendland C2, eta 1.2, open boundary, FP32 pairs / FP64 positions"
    if args.workload == "collision":
        return f"two colliding n=1 polytropes, {w.n} particles, closing speed 1, FP32 pairs / FP64 positions"
    if args.workload == "sod":
        return (f"1D Sod shock tube, {w.info['n_tube']} particles in [0, 1) and its mirror image ({w.n} in the "
                f"periodic box), M4, eta 1.2, gamma 1.4, FP64")
    return f"turbulence box {args.n_side or 256}^3 = {w.n} particles, Wendland C4, Mach 2, FP32 pairs / FP64 positions"


def src_hash(files):
    import hashlib
    hsh = hashlib.sha1()
    for f in files:
        with open(os.path.join(ROOT, "paper_2007_03097_gb300", "csrc", f), "rb") as fh:
            hsh.update(fh.read())
    return hsh.hexdigest()[:12]


def run_sph(args):
    import torch

    from paper_2007_03097_gb300 import binding as B
    from paper_2007_03097_gb300 import build, inputs

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    w = make_workload(args)
    fp64 = w.params.get("precision", "fp64") == "fp64"
    params = dict(w.params)
    params.update(hnet_batch=8192, hnet_iters=1, hnet_lr=1e-3, curve=args.curve)
    ctx = B.Context(params, w.n)
    p = B.Particles.from_workload(w, fp64=fp64)
    stream = torch.cuda.current_stream()
    B.sph_build_tree(ctx, p)
    B.sph_density(ctx, p)
    B.sph_forces(ctx, p)
    if w.dt is None:                       # fixed step from the initial CFL condition
        w.dt = float(w.params["cfl"] * torch.min(p.h / p.vsig).item())
    rng = np.random.default_rng(1234)
    theta = np.concatenate([rng.normal(scale=s, size=k) for s, k in
                            ((1 / math.sqrt(5), 320), (0, 64), (1 / 8, 4096), (0, 64), (1 / 8, 64), (0, 1))])
    B.sph_hnet_set_weights(ctx, theta.astype(np.float32))
    # train the h-predictor online on the plain solver's own steps (untimed)
    p_train = dict(params, hnet_iters=40)
    ctx.set_params(p_train)
    for _ in range(args.train_steps):
        B.sph_step(ctx, p, w.dt, use_hnet=B.SPH_HNET_TRAIN)
    ctx.set_params(params)
    for _ in range(args.warmup):
        B.sph_step(ctx, p, w.dt, use_hnet=B.SPH_HNET_SEED | B.SPH_HNET_TRAIN)
    snap = {f: getattr(p, f).clone() for f in ["x", "y", "z", "nnb", "id"] + B._FIELDS}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def restore():
        for f, t in snap.items():
            getattr(p, f).copy_(t)

    def timed(mode):
        restore()
        B.sph_step(ctx, p, w.dt, use_hnet=mode)            # re-establish tree/lists in this mode
        restore()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        stats = []
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            stats.append(B.sph_step(ctx, p, w.dt, use_hnet=mode))
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in ev]
        return ms, stats

    gpu_uuid = str(getattr(torch.cuda.get_device_properties(local), "uuid", local))
    if gpu_uuid and not gpu_uuid.startswith("GPU-") and "-" in gpu_uuid:
        gpu_uuid = "GPU-" + gpu_uuid
    clocks = ClockSampler(gpu_uuid)
    # learned h: the seed of the network trained above on the plain solver's
    # steps (frozen while timed); the same with one online Adam round per step
    # is timed too
    ms_l, st_l = timed(B.SPH_HNET_SEED)
    ms_o, st_o = timed(B.SPH_HNET_SEED | B.SPH_HNET_TRAIN)
    ms_p, st_p = timed(0)
    clk = clocks.stop()

    def summarize(ms, st):
        t = sum(ms) / 1e3
        inter = sum(s["density"]["interactions"] + s["forces"]["interactions"] for s in st)
        return dict(seconds=t, interactions=inter, interactions_per_s=inter / t, steps_per_s=len(ms) / t,
                    ms_per_step=1e3 * t / len(ms),
                    sweeps_per_step=sum(s["density"]["sweeps"] for s in st) / len(st),
                    density_kernel_ms=sum(s["density"]["kernel_ms"] for s in st),
                    force_kernel_ms=sum(s["forces"]["kernel_ms"] for s in st),
                    density_interactions=sum(s["density"]["interactions"] for s in st),
                    force_interactions=sum(s["forces"]["interactions"] for s in st),
                    density_launches=sum(s["density"]["sweeps"] for s in st),
                    list_builds=sum(s["density"]["list_builds"] for s in st),
                    launches=sum(s["launches"] for s in st),
                    hnet_fallback=sum(s["hnet_fallback"] for s in st),
                    hnet_loss=st[-1]["hnet_loss"], ms_tree=sum(s["ms_tree"] for s in st) / len(st),
                    # mean per-step phase times from the library's events: kick/drift and
                    # tree, h seed, density iteration (lists + sweeps), forces and the rest
                    ms_phase={k: sum(f(s) for s in st) / len(st) for k, f in (
                        ("tree", lambda s: s["ms_tree"]), ("hnet", lambda s: s["ms_hnet"]),
                        ("density", lambda s: s["density"]["ms"]), ("forces_kick_totals", lambda s: s["forces"]["ms"]),
                        ("total", lambda s: s["ms_total"]))},
                    tree_moved=[s["tree_moved"] for s in st])

    L = summarize(ms_l, st_l)
    O = summarize(ms_o, st_o)
    P = summarize(ms_p, st_p)

    # end to end through the C ABI with host buffers: H2D of the whole state
    # (every particle array, one slab) from pinned memory, the step, D2H of
    # the whole state, every step
    host = torch.empty_like(p.slab, device="cpu").pin_memory()
    restore()
    host.copy_(p.slab)
    h2d = host.numel()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e_inter = 0
    e0.record(stream)
    for k in range(args.steps):
        p.slab.copy_(host, non_blocking=True)
        s = B.sph_step(ctx, p, w.dt, use_hnet=B.SPH_HNET_SEED)
        e_inter += s["density"]["interactions"] + s["forces"]["interactions"]
        host.copy_(p.slab, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_s = e0.elapsed_time(e1) / 1e3

    # dominant kernel of the learned step and its roofline
    dens_flops = L["density_interactions"] * F_DENSITY
    force_flops = L["force_interactions"] * F_FORCE
    if fp64:
        names = ("k_density<double> (h-rho sweep, double-float)", "k_forces_df (Eqs. 5-6, double-float)")
        peak, peak_src = DF_EMULATED_TFLOPS, ("derived: FP32 pipe (152 SMs x 128 lanes x 2.07 GHz) running "
                                              "double-float FP64 multiply-adds at 18 FP32 instructions per 2 flops")
    else:
        names = ("k_density<float> (h-rho sweep, FP32)", "k_forces_f32 (Eqs. 5-6, FP32)")
        peak, peak_src = FP32_PIPE_TFLOPS, "derived: FP32 pipe, 152 SMs x 128 lanes x 2 flop x 2.07 GHz"
    dominant_density = L["density_kernel_ms"] >= L["force_kernel_ms"]
    if dominant_density:
        kname, flops, kms, launches = names[0], dens_flops, L["density_kernel_ms"], L["density_launches"]
    else:
        kname, flops, kms, launches = names[1], force_flops, L["force_kernel_ms"], args.steps
    achieved = flops / (kms / 1e3) / 1e12
    # DRAM traffic per launch from one ncu capture (profiles/), valid only for
    # the kernel source it was taken on
    traffic = None
    key = ("density" if dominant_density else "forces") + ("_fp64" if fp64 else "_mixed") + "_" + args.workload
    rec = TRAFFIC.get(key)
    if rec and rec["src"] == src_hash(rec["files"]):
        traffic = rec["bytes_per_launch"]
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic, "kernel": kname,
            "launches": launches, "avg_launch_ms": kms / max(launches, 1), "peak_source": peak_src,
            "fp64_pipe_peak": FP64_PIPE_TFLOPS, "fp32_pipe_peak": FP32_PIPE_TFLOPS,
            "other_kernels": {
                "k_density_tflops": dens_flops / max(L["density_kernel_ms"], 1e-9) / 1e9,
                "k_forces_tflops": force_flops / max(L["force_kernel_ms"], 1e-9) / 1e9}}

    # whole-job numbers (max time over ranks; units summed over ranks)
    (t_l, e2e_s), (inter_l, e_inter) = whole_job([L["seconds"], e2e_s], [L["interactions"], e_inter],
                                                  device="cuda")
    lists = B.sph_list_info(ctx)
    lists["slots_per_particle"] = lists["slots_used"] / w.n
    nl, ng = B.sph_tree_info(ctx)
    lists["union_per_group"] = lists["union_used"] / max(ng, 1)
    # candidates against accepted pairs: every lane of a group visits its
    # group's list width in the force pass, so the slots used are the
    # candidate slots of one pass
    pairs = L["force_interactions"] / max(len(ms_l), 1)
    lists["force_pairs_per_pass"] = pairs
    lists["candidate_slots_per_accepted_pair"] = lists["slots_used"] / max(pairs, 1)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, seconds=12.0, label=args.workload)
    if rank == 0:
        out = {
            "metric": METRIC, "value": inter_l / t_l, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_l / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if fp64 else "f32", "data": "synthetic",
            "config": {"workload": workload_label(args, w),
                       "n_particles": w.n, "precision": "fp64" if fp64 else "mixed (FP32 pairs, FP64 positions)",
                       "parallelism": f"replicas x{world}", "curve": args.curve,
                       "l2": "flushed between timed steps (256 MB write)",
                       "step": "learned-h sph_step (seed from the network trained on the plain solver's steps "
                               "before the timed region)"},
            "steps_per_s": world * args.steps / t_l,
            "learned_h": L, "plain_h": P, "learned_online_h": O,
            "learned_vs_plain_steps_per_s": L["steps_per_s"] / P["steps_per_s"],
            "e2e": {"value": e_inter / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d,
                    "steps_per_s": world * args.steps / e2e_s},
            "gpu_launches": L["launches"],
            "neighbour_lists": lists,
            "roofline": roof,
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------------------ CPU oracle
def _oracle_sample(w, n_targets, seed=7):
    import oracle
    op = oracle.Params(**{k: v for k, v in w.params.items() if k in oracle.Params.__dataclass_fields__})
    rng = np.random.default_rng(seed)
    t = np.sort(rng.choice(w.n, size=min(n_targets, w.n), replace=False))
    t0 = time.perf_counter()
    d = oracle.density(op, w.x, w.y, w.z, w.m, w.h, targets=t)
    # forces for the same targets with the seed state's rho/h for the sources
    rho = np.where(np.isnan(d.rho), 1.0, d.rho)
    h = np.where(np.isnan(d.h), w.h, d.h)
    P, c = oracle.eos(op.gamma, rho, w.u)
    f = oracle.forces(op, w.x, w.y, w.z, w.vx, w.vy, w.vz, w.m, h, rho, P, c, targets=t)
    dt = time.perf_counter() - t0
    # brute force: every evaluation of a target tests all n sources
    tests = (int(d.sweeps[t].sum()) + t.size) * w.n
    return int(d.pairs[t].sum()) + f.npairs, dt, t.size, oracle.num_threads(), tests


def cpu_baseline(w, seconds=12.0, label="sedov"):
    """The oracle as it stands on the host cores, on a sample of target
    particles sized for about `seconds` of work; interactions/s."""
    nt2 = 64
    for _ in range(3):                        # grow the sample until it takes about `seconds`
        inter, dt, nt, cores, tests = _oracle_sample(w, nt2)
        if dt >= 0.5 * seconds or nt2 >= w.n:
            break
        nt2 = min(w.n, int(nt2 * seconds / max(dt, 1e-3)))
    return {"value": inter / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "candidate_tests_per_s": tests / dt,
            "sample": f"{nt} random targets of the {w.n}-particle {label} state, brute force over all sources: "
                      f"h-rho iteration + force pass, {dt:.1f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    w = make_workload(args)
    if w.dt is None:
        w.dt = 0.0
    per_step = max(16, int(512 * 262144 / w.n))
    for _ in range(args.warmup):
        _oracle_sample(w, per_step, seed=1)
    inter, secs, nt, cores = 0, 0.0, 0, 1
    for k in range(args.steps):
        i, dt, nt, cores, _ = _oracle_sample(w, per_step, seed=100 + k)
        inter += i
        secs += dt
    v = inter / secs
    out = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": workload_label(args, w), "n_particles": w.n,
                      "step": f"FP64 oracle h-rho iteration + forces for {per_step} sampled targets"},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"{per_step} random targets per step, brute force over all {w.n} sources"},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_sph(args)


if __name__ == "__main__":
    main()
