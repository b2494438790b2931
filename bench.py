#!/usr/bin/env python
"""Benchmark of the SPH hot path on GB300: particle-neighbour interactions/s
and SPH steps/s, learned-h vs plain-h, on one GPU.

Headline workload (default): the periodic turbulence box, 256^3 = 16,777,216
particles on a jittered lattice, Gaussian solenoidal velocity field with
P(k) ~ k^-4, rms Mach 2, gamma 1.01, Wendland C4 (~100 neighbours), FP32 pair
arithmetic on FP64 positions, h-rho iteration to 1e-6, learned-h seeding.

One timed step = one kick-drift-kick sph_step: tree (keys, sort, permute,
leaves), h-predictor inference, neighbour lists, h-rho sweeps, forces, kicks,
FP64 totals.  Inputs are resident in HBM (far larger than L2); L2 is also
flushed (a 256 MB write) between timed steps and each step is bracketed by
CUDA events on the launching stream.

The h-predictor is trained once, before anything is timed, by the library's
own training kernels on the plain solver's h trajectories: 200 plain steps of
the 16^3 lattice with variable h (M4, eta 1.2) and 200 plain steps of the
64^3 Sedov blast; its weights are then frozen and seed every learned step.

Extra keys (N = 1): the two colliding polytropes (2 x 2^21 particles, mixed,
learned vs plain) and the 64^3 Sedov blast in FP64 (double-float pair sums)
with its own roofline.

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
# algorithmic flops per accepted pair, counted from the pair arithmetic of the
# density sweep and of the force pass (FMA = 2, sqrt/div = 1)
F_DENSITY = 28
F_FORCE = 96
# Ceilings derived from unit counts and the 2.07 GHz maximum SM clock (152
# SMs): FP64 pipe 2 DFMA lanes/clk/SM; FP32 pipe 128 lanes/clk/SM.  The FP64
# mode evaluates its pair terms in double-float on the FP32 pipe, where one
# FP64 multiply-add (2 flops) costs 18 FP32 instructions (df_mul 7 + df_add 11).
SM_COUNT, SM_MHZ = 152, 2070.0
FP64_PIPE_TFLOPS = SM_COUNT * 2 * 2 * SM_MHZ * 1e6 / 1e12
FP32_PIPE_TFLOPS = SM_COUNT * 128 * 2 * SM_MHZ * 1e6 / 1e12
# One FP32 instruction is half an FP32 FMA's 2 flops, so the double-float
# ceiling in FP64 flops is the FP32 flop rate x (1/2) x (2/18) = rate / 18.
DF_PER_FP32 = 1.0 / 18.0
# DRAM bytes per launch of a dominant kernel from one ncu capture (profiles/),
# with the hash of the sources it was taken on and the particles of the
# captured launch (traffic scales with the particles at a fixed neighbour
# number, so a capture on a reduced side is scaled by the particle ratio)
TRAFFIC = {
    # dram__bytes_read.sum + dram__bytes_write.sum of one launch (ncu, see profiles/), with the
    # particles of the captured workload; valid while the listed sources hash as recorded
    "forces_fp64_sedov": {"bytes_per_launch": 84436224, "particles": 262144, "src": "e61daca242b6",
                          "files": ["forces.cu", "dfloat.cuh", "neighbors.cu", "sph_internal.cuh"]},
    # captured on the 128^3 box, scaled by the particles (per-particle lists and unions
    # are the same at 256^3)
    "forces_mixed_turbulence": {"bytes_per_launch": 1229722112, "particles": 2097152, "src": "858cf9be8c94",
                                "files": ["forces.cu", "neighbors.cu", "sph_internal.cuh"]},
}
PROTOCOL_TRAIN_STEPS = 200


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sph", choices=["sph", "reference"])
    ap.add_argument("--workload", default="turbulence",
                    choices=["turbulence", "collision", "polytrope", "sedov", "sod"],
                    help="turbulence: 256^3 mixed (headline); collision 2x2^21 and polytrope 2^20: mixed; "
                         "sedov: 64^3 FP64; sod: the 1D shock tube, 10,000 particles in the tube, FP64")
    ap.add_argument("--n-side", type=int, default=None,
                    help="lattice side of the turbulence (default 256) and sedov (default 64) workloads; "
                         "smaller sides serve profiling captures")
    ap.add_argument("--curve", default="morton", choices=["morton", "hilbert"],
                    help="space-filling curve of the particle keys (Sec. 2.1, Tree topology)")
    ap.add_argument("--train-steps", type=int, default=PROTOCOL_TRAIN_STEPS,
                    help="plain steps of each training workload (16^3 lattice, 64^3 Sedov)")
    ap.add_argument("--no-extras", action="store_true", help="skip the collision and Sedov extra keys")
    ap.add_argument("--profile-window", action="store_true",
                    help="start the CUDA profiler only around the timed learned-h steps "
                         "(for ncu --profile-from-start off)")
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


# ------------------------------------------------------------------ workloads
def make_workload(name, n_side=None):
    from paper_2007_03097_gb300 import inputs
    if name == "sedov":
        return inputs.sedov(n_side or 64)
    if name == "polytrope":
        return inputs.polytrope(1 << 20)
    if name == "collision":
        return inputs.collision(1 << 21)
    if name == "sod":
        return inputs.sod(10000)
    return inputs.turbulence(n_side or 256)


def workload_label(name, w, n_side=None):
    if name == "sedov":
        return (f"sedov blast {n_side or 64}^3 = {w.n} particles, Wendland C2, eta 1.2, h_tol 1e-6, "
                f"alpha 1 beta 2, FP64 (double-float pair sums), fixed dt {w.dt:.3e}")
    if name == "polytrope":
        return f"n=1 polytrope, {w.n} particles, Wendland C2, eta 1.2, open boundary, FP32 pairs / FP64 positions"
    if name == "collision":
        return f"two colliding n=1 polytropes, {w.n} particles, closing speed 1, FP32 pairs / FP64 positions"
    if name == "sod":
        return (f"1D Sod shock tube, {w.info['n_tube']} particles in [0, 1) and its mirror image ({w.n} in the "
                f"periodic box), M4, eta 1.2, gamma 1.4, FP64")
    return (f"periodic turbulence box {n_side or 256}^3 = {w.n} particles, k^-4 solenoidal field, rms Mach 2, "
            f"gamma 1.01, Wendland C4 (~100 neighbours), h_tol 1e-6, FP32 pairs / FP64 positions, learned-h")


def src_hash(files):
    import hashlib
    hsh = hashlib.sha1()
    for f in files:
        with open(os.path.join(ROOT, "paper_2007_03097_gb300", "csrc", f), "rb") as fh:
            hsh.update(fh.read())
    return hsh.hexdigest()[:12]


def summarize(ms, st):
    t = sum(ms) / 1e3
    inter = sum(s["density"]["interactions"] + s["forces"]["interactions"] for s in st)
    return dict(seconds=t, interactions=inter, interactions_per_s=inter / t, steps_per_s=len(ms) / t,
                ms_per_step=1e3 * t / len(ms),
                sweeps_per_step=sum(s["density"]["sweeps"] for s in st) / len(st),
                evaluations_per_step=sum(s["density"]["evaluations"] for s in st) / len(st),
                density_kernel_ms=sum(s["density"]["kernel_ms"] for s in st),
                force_kernel_ms=sum(s["forces"]["kernel_ms"] for s in st),
                density_interactions=sum(s["density"]["interactions"] for s in st),
                force_interactions=sum(s["forces"]["interactions"] for s in st),
                density_launches=sum(s["density"]["sweeps"] for s in st),
                list_builds=sum(s["density"]["list_builds"] for s in st),
                launches=sum(s["launches"] for s in st),
                hnet_fallback=sum(s["hnet_fallback"] for s in st),
                hnet_loss=st[-1]["hnet_loss"],
                # mean per-step phase times from the library's events: kick/drift and
                # tree, h seed, density iteration (lists + sweeps), forces and the rest
                ms_phase={k: sum(f(s) for s in st) / len(st) for k, f in (
                    ("tree", lambda s: s["ms_tree"]), ("hnet", lambda s: s["ms_hnet"]),
                    ("density", lambda s: s["density"]["ms"]), ("lists", lambda s: s["density"]["lists_ms"]),
                    ("sweeps", lambda s: s["density"]["kernel_ms"]),
                    ("forces_kick_totals", lambda s: s["forces"]["ms"]),
                    ("total", lambda s: s["ms_total"]))},
                tree_moved=[s["tree_moved"] for s in st])


class Run:
    """One workload on the GPU: context, particles, a snapshot to restore,
    and timed learned / plain steps from the same state."""

    def __init__(self, B, torch, name, n_side, curve, theta, warmup):
        self.B, self.torch = B, torch
        self.w = make_workload(name, n_side)
        w = self.w
        self.fp64 = w.params.get("precision", "fp64") == "fp64"
        self.params = dict(w.params)
        self.params.update(hnet_batch=8192, hnet_iters=1, hnet_lr=1e-3, curve=curve)
        self.ctx = B.Context(self.params, w.n)
        self.p = B.Particles.from_workload(w, fp64=self.fp64)
        self.stream = torch.cuda.current_stream()
        p = self.p
        B.sph_build_tree(self.ctx, p)
        B.sph_density(self.ctx, p)
        B.sph_forces(self.ctx, p)
        if w.dt is None:                       # fixed step from the initial CFL condition
            w.dt = float(self.params["cfl"] * torch.min(p.h / p.vsig).item())
        self.theta = np.asarray(theta, dtype=np.float32)
        B.sph_hnet_set_weights(self.ctx, self.theta)
        for _ in range(warmup):
            B.sph_step(self.ctx, p, w.dt, use_hnet=B.SPH_HNET_SEED)
        self.snap = {f: getattr(p, f).clone() for f in ["x", "y", "z", "nnb", "id"] + B._FIELDS}
        self.flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def restore(self):
        for f, t in self.snap.items():
            getattr(self.p, f).copy_(t)

    def timed(self, mode, steps, world=1, window=False):
        B, torch, p, w = self.B, self.torch, self.p, self.w
        self.restore()
        B.sph_step(self.ctx, p, w.dt, use_hnet=mode)        # re-establish tree/lists in this mode
        self.restore()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        stats = []
        if window:
            torch.cuda.profiler.start()
        for k in range(steps):
            self.flush.zero_()
            ev[k][0].record(self.stream)
            stats.append(B.sph_step(self.ctx, p, w.dt, use_hnet=mode))
            ev[k][1].record(self.stream)
        torch.cuda.synchronize()
        if window:
            torch.cuda.profiler.stop()
        if world > 1:
            torch.distributed.barrier()
        return [a.elapsed_time(b) for a, b in ev], stats

    def e2e(self, steps):
        """The learned step end to end through the C ABI with host buffers:
        H2D of the whole state (every particle array, one slab) from pinned
        memory, the step, D2H of the whole state, every step."""
        B, torch, p, w = self.B, self.torch, self.p, self.w
        host = torch.empty_like(p.slab, device="cpu").pin_memory()
        self.restore()
        B.sph_hnet_set_weights(self.ctx, self.theta)
        host.copy_(p.slab)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        inter = 0
        e0.record(self.stream)
        for _ in range(steps):
            p.slab.copy_(host, non_blocking=True)
            s = B.sph_step(self.ctx, p, w.dt, use_hnet=B.SPH_HNET_SEED)
            inter += s["density"]["interactions"] + s["forces"]["interactions"]
            host.copy_(p.slab, non_blocking=True)
        e1.record(self.stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3, inter, host.numel()

    def lists(self, force_pairs_per_pass):
        B, w = self.B, self.w
        li = B.sph_list_info(self.ctx)
        li["slots_per_particle"] = li["slots_used"] / w.n
        _, ng = B.sph_tree_info(self.ctx)
        li["union_per_group"] = li["union_used"] / max(ng, 1)
        # every lane of a group visits its group's list width in the force
        # pass, so the slots used are the candidate slots of one pass
        li["force_pairs_per_pass"] = force_pairs_per_pass
        li["candidate_slots_per_accepted_pair"] = li["slots_used"] / max(force_pairs_per_pass, 1)
        return li

    def close(self):
        self.ctx.close()


def roofline(L, steps, fp64, workload, fp32_measured):
    """The dominant pair kernel of the learned step against its ALU ceiling."""
    dens_flops = L["density_interactions"] * F_DENSITY
    force_flops = L["force_interactions"] * F_FORCE
    if fp64:
        names = ("k_density<double> (h-rho sweep, double-float)", "k_forces_df (Eqs. 5-6, double-float)")
        ratio, what = DF_PER_FP32, "double-float FP64 multiply-adds at 18 FP32 instructions per 2 flops on "
    else:
        names = ("k_density<float> (h-rho sweep, FP32)", "k_forces_f32 (Eqs. 5-6, FP32)")
        ratio, what = 1.0, ""
    derived = FP32_PIPE_TFLOPS * ratio
    if fp32_measured:
        peak = fp32_measured * ratio
        src = (f"measured: {what}the FP32 FMA-chain rate of this GPU in this run "
               f"({fp32_measured:.1f} TFLOP/s, sph_peak_fp32)")
    else:
        peak, src = derived, f"derived: {what}the FP32 pipe, 152 SMs x 128 lanes x 2 flop x 2.07 GHz"
    dominant_density = L["density_kernel_ms"] >= L["force_kernel_ms"]
    if dominant_density:
        kname, flops, kms, launches = names[0], dens_flops, L["density_kernel_ms"], L["density_launches"]
    else:
        kname, flops, kms, launches = names[1], force_flops, L["force_kernel_ms"], steps
    achieved = flops / (kms / 1e3) / 1e12
    traffic = None
    key = ("density" if dominant_density else "forces") + ("_fp64" if fp64 else "_mixed") + "_" + workload["name"]
    rec = TRAFFIC.get(key)
    if rec and rec["src"] == src_hash(rec["files"]):
        traffic = rec["bytes_per_launch"] * workload["n"] / rec["particles"]
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": kname, "launches": launches, "avg_launch_ms": kms / max(launches, 1),
            "peak_source": src, "derived_peak": derived, "frac_of_derived": achieved / derived,
            "fp64_pipe_peak": FP64_PIPE_TFLOPS, "fp32_pipe_peak": FP32_PIPE_TFLOPS,
            "flops_per_pair": F_DENSITY if dominant_density else F_FORCE,
            "other_kernels": {
                "k_density_tflops": dens_flops / max(L["density_kernel_ms"], 1e-9) / 1e9,
                "k_forces_tflops": force_flops / max(L["force_kernel_ms"], 1e-9) / 1e9}}


def extra_run(B, torch, name, theta, steps, warmup, fp32_measured):
    """A secondary workload: learned vs plain steps/s and its roofline."""
    r = Run(B, torch, name, None, "morton", theta, warmup)
    ms_l, st_l = r.timed(B.SPH_HNET_SEED, steps)
    ms_p, st_p = r.timed(0, steps)
    L, P = summarize(ms_l, st_l), summarize(ms_p, st_p)
    out = {"workload": workload_label(name, r.w), "n_particles": r.w.n,
           "dtype": "df64" if r.fp64 else "f32", "steps": steps,
           "value": L["interactions_per_s"], "unit": UNIT, "ms_per_step": L["ms_per_step"],
           "steps_per_s": L["steps_per_s"], "learned_h": L, "plain_h": P,
           "learned_vs_plain_steps_per_s": L["steps_per_s"] / P["steps_per_s"],
           "learned_vs_plain_evaluations": L["evaluations_per_step"] / P["evaluations_per_step"],
           "roofline": roofline(L, steps, r.fp64, {"name": name, "n": r.w.n}, fp32_measured)}
    r.close()
    return out


def run_sph(args):
    import torch

    from paper_2007_03097_gb300 import binding as B
    from paper_2007_03097_gb300 import build

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    # the h-predictor: trained on the plain solver's trajectories (untimed), frozen
    from paper_2007_03097_gb300 import hnet_protocol
    t0 = time.perf_counter()
    if args.train_steps > 0:
        theta, losses = hnet_protocol.train(steps=args.train_steps)
    else:                                  # profiling runs: the untrained network
        theta, losses = hnet_protocol.initial_theta(), {}
    train_s = time.perf_counter() - t0
    fp32_peak = B.sph_peak_fp32()

    gpu_uuid = str(getattr(torch.cuda.get_device_properties(local), "uuid", local))
    if gpu_uuid and not gpu_uuid.startswith("GPU-") and "-" in gpu_uuid:
        gpu_uuid = "GPU-" + gpu_uuid
    r = Run(B, torch, args.workload, args.n_side, args.curve, theta, args.warmup)
    w = r.w
    clocks = ClockSampler(gpu_uuid)
    # learned h (frozen network), plain h, and learned h with one online Adam
    # round per step (on the context's side stream, beside the force pass)
    ms_l, st_l = r.timed(B.SPH_HNET_SEED, args.steps, world, window=args.profile_window)
    ms_p, st_p = r.timed(0, args.steps, world)
    ms_o, st_o = r.timed(B.SPH_HNET_SEED | B.SPH_HNET_TRAIN, args.steps, world)
    e2e_s, e_inter, h2d = r.e2e(args.steps)
    clk = clocks.stop()
    L, P, O = summarize(ms_l, st_l), summarize(ms_p, st_p), summarize(ms_o, st_o)
    roof = roofline(L, args.steps, r.fp64, {"name": args.workload, "n": w.n}, fp32_peak["tflops"])
    lists = r.lists(L["force_interactions"] / max(len(ms_l), 1))
    (t_l, e2e_s), (inter_l, e_inter) = whole_job([L["seconds"], e2e_s], [L["interactions"], e_inter],
                                                  device="cuda")
    config = {"workload": workload_label(args.workload, w, args.n_side), "n_particles": w.n,
              "precision": "fp64 (double-float pair sums)" if r.fp64 else "mixed (FP32 pairs, FP64 positions)",
              "parallelism": f"replicas x{world}", "curve": args.curve,
              "l2": "inputs larger than L2; also flushed between timed steps (256 MB write)",
              "step": "learned-h sph_step (seed from the frozen network trained on 200 plain steps each of the "
                      "16^3 lattice and the 64^3 Sedov blast before the timed region)"}
    r.close()
    del r
    torch.cuda.empty_cache()

    extras = {}
    if world == 1 and not args.no_extras and args.workload == "turbulence":
        for name in ("collision", "sedov"):
            extras[name] = extra_run(B, torch, name, theta, args.steps, args.warmup, fp32_peak["tflops"])
            torch.cuda.empty_cache()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, seconds=12.0, label=args.workload)
    if rank == 0:
        out = {
            "metric": METRIC, "value": inter_l / t_l, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_l / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "df64" if r_fp64(w) else "f32", "data": "synthetic",
            "config": config,
            "steps_per_s": world * args.steps / t_l,
            "learned_h": L, "plain_h": P, "learned_online_h": O,
            "learned_vs_plain_steps_per_s": L["steps_per_s"] / P["steps_per_s"],
            "learned_vs_plain_evaluations": L["evaluations_per_step"] / P["evaluations_per_step"],
            "hnet_training": {"protocol": f"{args.train_steps} plain steps each of the 16^3 lattice (variable h) "
                                          f"and the 64^3 Sedov blast, 40 Adam iterations per step",
                              "last_loss": losses, "seconds": train_s},
            "e2e": {"value": e_inter / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d,
                    "steps_per_s": world * args.steps / e2e_s},
            "gpu_launches": L["launches"],
            "neighbour_lists": lists,
            "roofline": roof,
            "fp32_fma_peak": fp32_peak,
            "clocks": clk,
            "cpu_baseline": cpu,
            "extra": extras,
        }
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


def r_fp64(w):
    return w.params.get("precision", "fp64") == "fp64"


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


def cpu_baseline(w, seconds=12.0, label="turbulence"):
    """The oracle as it stands on the host cores, on a sample of target
    particles sized for about `seconds` of work; interactions/s."""
    nt2 = 16
    for _ in range(5):                        # grow the sample until it takes about `seconds`
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
    w = make_workload(args.workload, args.n_side)
    if w.dt is None:
        w.dt = 0.0
    # about 0.2 s of brute force per step on 16 host cores at any size
    per_step = max(16, int(512 * 262144 / w.n))
    for _ in range(args.warmup):
        _oracle_sample(w, per_step, seed=1)
    inter, secs, nt, cores = 0, 0.0, 0, 1
    for k in range(args.steps):
        i, dt, nt, cores, _ = _oracle_sample(w, per_step, seed=100 + k)
        inter += i
        secs += dt
    v = inter / secs
    fp64 = r_fp64(w)
    config = {"workload": workload_label(args.workload, w, args.n_side), "n_particles": w.n,
              "precision": "fp64 (double-float pair sums)" if fp64 else "mixed (FP32 pairs, FP64 positions)",
              "parallelism": f"replicas x{world}", "curve": args.curve,
              "l2": "inputs larger than L2; also flushed between timed steps (256 MB write)",
              "step": "learned-h sph_step (seed from the frozen network trained on 200 plain steps each of the "
                      "16^3 lattice and the 64^3 Sedov blast before the timed region)"}
    sample = (f"{per_step} random targets per step of the {w.n}-particle state, FP64 oracle h-rho iteration + "
              f"force pass, brute force over all sources")
    out = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": config,
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
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
