#!/usr/bin/env python3
"""Benchmark: ASM-PCG time-steps/s on the coupled PolyDG monodomain + Barreto-Cressman
step, every step solved by PCG with the two-level additive Schwarz preconditioner to
|r|_2 <= 1e-8 |b|_2 on one GB300.

Default workload (the largest single-GPU configuration): the unit cube in 48^3 jittered
hexahedra (12-facet polyhedra), P2, 1,105,920 DOFs, 1728 subdomains of 4^3 cells = coarse
agglomerates, coarse P1 (6912 DOFs), isotropic sigma = 1, dt = 0.05 ms, Gaussian
stimulus; the workload's 50 steps cover the warm-up and the timed steps.

A "step" is one Crank-Nicolson time step through the C ABI (monodomain_step): ionic
update at the quadrature nodes, right-hand side, initial guess, and the persistent PCG
kernel.  Forms timed on the same setup:
  * mixed + learned (reported): fp32 local inverses in flexible PCG (fp64 residual, dots,
    coarse solve and matvec); initial guess = Galerkin projection onto the learned
    proposal (weights in paper_2512_19536_gb300/guess_p3_voronoi4096.npz) and the last 24
    solution increments;
  * the increments alone (no network), and x0 = U^k, as ablations;
  * fp64 plain: fp64 local inverses in standard PCG, x0 = U^k.
Each preconditioner's split of its work over the CTAs is autotuned at setup
(asm_autotune), which is not part of the timed steps.  The 4096-cell Voronoi P3 workload
(the 2D configuration) is timed in the same run and reported under config.voronoi4096.
The working sets (fp32 store 2.8 GB + K_h 608 MB at 48^3) exceed the 126 MB L2, so no L2
flush is inserted between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload hex48|voronoi4096|batch32|hex32|hex24]
                       [--ionic-form nodal|modal]
Under torchrun (N > 1) every rank runs an independent replica (the path has no
exchange step); rank 0 prints one JSON line with the whole-job throughput.

--workload voronoi4096 reports the 2D workload alone (200 steps); --workload batch32
the batched forms: 32 independent simulations on 8 Voronoi meshes of 1024-16384 cells,
4 per mesh, the 4 simulations of each mesh in lockstep sharing one bf16 eigenbasis (unit:
simulation-steps/s).  --ionic-form modal keeps the ionic state in the DG basis (the
second line of Eq. fully-discrete-1) in every timed form.

The CPU baseline (and --impl reference) is the float64 oracle (oracle/) on the host
cores, timed on whole time steps of a stated sub-problem of the same recipe (the 8^3
cube for the 3D workload) and scaled to the workload by its DOFs (and, in the CPU
baseline, by the GPU's iteration count); the scaling is stated in the line.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ASM-PCG time-steps/s at rel.res 1e-8, mixed+learned vs FP64 plain, 1 GB300"
BATCH_WORKLOAD = ("batch32: 32 coupled simulations, 8 Voronoi meshes 1024-16384 cells "
                  "(log-uniform, seed 4) x 4 conductivities/stimuli, P3, ~64 cells/subdomain")
WORKLOAD = "voronoi4096_p3 coupled monodomain+Barreto-Cressman, 40960 DOFs, 64 subdomains, coarse P1"
HEX_WORKLOAD = ("hex{n}_p2: {n}^3 jittered hexahedra (12-facet polyhedra, seed 3), P2, {dofs} DOFs, "
                "{subs} subdomains of 4^3 = coarse agglomerates, coarse P1 ({n0} DOFs), coupled "
                "monodomain+Barreto-Cressman, 50 steps")


def reduce_over_ranks(torch, times_ms, rates, world, device):
    """Replicas: every rank times its own copy of the workload; the job is as slow as
    its slowest rank (max of the times) and its end-to-end rate that of the slowest
    (min of the rates).  Returns (times_ms, rates) as lists of floats, identical on
    every rank."""
    if world <= 1:
        return list(times_ms), list(rates)
    t = torch.tensor(list(times_ms), dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    r = torch.tensor(list(rates) if rates else [0.0], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(r, op=torch.distributed.ReduceOp.MIN)
    return [float(x) for x in t], ([float(x) for x in r] if rates else [])


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    def __init__(self, dev):
        self.dev, self.proc, self.lines = dev, None, []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return self
        # wait for the first sample: while nvidia-smi initialises NVML, this process's
        # own driver calls can stall, and that must not fall inside the timed region
        import select
        ready, _, _ = select.select([self.proc.stdout], [], [], 15.0)
        if ready:
            first = self.proc.stdout.readline()
            if first.strip():
                self.lines.append(first.strip())
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines += [l for l in out.splitlines() if l.strip()]

    def summary(self):
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            try:
                mhz.append(float(f[0]))
                mx = float(f[1])
            except (ValueError, IndexError):
                continue
            for name, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": mx,
                "samples": len(mhz), "reasons": sorted(reasons)}


def build_case():
    from synth import voronoi4096_p3
    return voronoi4096_p3()


def algorithmic_bytes(ctx_info, pc_info, iterations, launches):
    """Bytes one PCG launch must move (per iteration: K_h blocks, the local inverse
    store, K_0^{-1}, the rows of R_0 and ~12 fp64 vector streams; plus one K_h pass
    and 4 vector streams for the initial residual)."""
    n = ctx_info.n_dofs
    k_bytes = 8 * ctx_info.n_p ** 2 * ctx_info.n_blocks
    per_it = (k_bytes + pc_info["local_store_bytes"] + pc_info["coarse_bytes"]
              + pc_info["restrict_bytes"] + 12 * 8 * n)
    return iterations * per_it + launches * (k_bytes + 4 * 8 * n)


GUESS_WEIGHTS = os.path.join(ROOT, "paper_2512_19536_gb300", "guess_p3_voronoi4096.npz")


def load_guess(pd):
    """The trained guess model, or None if its weights file is missing."""
    import numpy as np
    if not os.path.exists(GUESS_WEIGHTS):
        return None
    z = np.load(GUESS_WEIGHTS)
    return pd.guess_create(int(z["n_p"]), z["params"], z["scales"])


GUESS_POLICY = 3   # Galerkin projection onto the learned proposal and the last 24 solution increments


def time_form(pd, torch, w, ctx, precision, flexible, steps, warmup, stream, clocks=None,
              guess=None, pc=None, policy=None, ionic_form="nodal"):
    if pc is None:
        pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision=precision)
        pd.asm_autotune(pc, rounds=6, iterations=60)   # setup: re-cut the rows by measured CTA times
    sim = pd.sim_create(ctx, pc, u0=w.u_rest, stimulus=w.stimulus, rtol=1e-8, maxit=5000,
                        flexible=flexible)
    if ionic_form != "nodal":
        pd.sim_set_ionic_form(sim, ionic_form)
    if policy is not None:
        pd.sim_set_guess(sim, guess, policy)
    pd.monodomain_step(sim, warmup, stream)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if torch.distributed.is_initialized():
        torch.distributed.barrier()
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.__enter__()
    ev0.record(stream)
    st = pd.monodomain_step(sim, steps, stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.__exit__(None, None, None)
    ms = ev0.elapsed_time(ev1)
    return pc, sim, st, ms


class HostHistory:
    """The last H solutions of one simulation in pinned host memory, kept as a ring (row
    `head` the newest, then older ones upwards, wrapping): a new solution is written into
    the row that the oldest one held, so no step shifts the history on the host.
    `upload` copies the rows to a device [H, n] tensor newest first (two copies where the
    ring wraps); `push_from` reads a solution into the ring (non-blocking from a device
    tensor: the caller synchronises before the next upload)."""

    def __init__(self, torch, H, n, pin=True):
        ring = torch.zeros((H, n), dtype=torch.float64)
        self.ring = ring.pin_memory() if pin else ring
        self.H = H
        self.head = 0
        self.count = 0

    def push_from(self, src, non_blocking=False):
        self.head = (self.head - 1) % self.H
        self.ring[self.head].copy_(src, non_blocking=non_blocking)
        self.count = min(self.H, self.count + 1)

    def upload(self, dst):
        a = self.H - self.head
        dst[:a].copy_(self.ring[self.head:], non_blocking=True)
        if self.head:
            dst[a:].copy_(self.ring[:self.head], non_blocking=True)


def time_e2e(pd, torch, w, ctx, pc, steps, stream, guess=None, warm=12, ionic_form="nodal"):
    """Same metric with the state crossing the host boundary every step: the last
    solutions the step depends on (U^k .. U^{k-24}: the initial guess reads them) copied in
    from pinned host memory and restored with sim_set_history, U^{k+1} copied back to
    pinned host memory.  The same steps as the device-timed forms: `warm` untimed, then
    `steps` timed."""
    sim = pd.sim_create(ctx, pc, u0=w.u_rest, stimulus=w.stimulus, rtol=1e-8, maxit=5000,
                        flexible=True)
    if ionic_form != "nodal":
        pd.sim_set_ionic_form(sim, ionic_form)
    pd.sim_set_guess(sim, guess, GUESS_POLICY)
    n = ctx.n_dofs
    H = 25
    hist = HostHistory(torch, H, n)                 # U^k, U^{k-1}, ... in pinned host memory
    dev_hist = torch.empty((H, n), dtype=torch.float64, device="cuda")
    dev_u = torch.empty(n, dtype=torch.float64, device="cuda")
    for _ in range(warm):
        pd.monodomain_step(sim, 1, stream)
        pd.sim_get_state(sim, dev_u, stream=stream)
        hist.push_from(dev_u.cpu())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        hist.upload(dev_hist)
        pd.sim_set_history(sim, dev_hist[:hist.count], stream)
        pd.monodomain_step(sim, 1, stream)
        pd.sim_get_state(sim, dev_u, stream=stream)
        hist.push_from(dev_u, non_blocking=True)
        torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    sim.close()
    return steps / dt, H * 8 * n, 8 * n


class Oracle:
    """Whole time steps of the float64 oracle (oracle.monodomain with oracle.pcg and the
    two-level oracle.schwarz preconditioner, rtol 1e-8, x0 = U^k) on workload w."""

    def __init__(self, w, ionic_form="nodal"):
        from oracle import assembly, schwarz, monodomain
        self.w = w
        self.d = assembly.assemble(w.mesh, w.p, w.sigma, w.eta0, w.chi_cm, w.dt)
        S = schwarz.build(self.d, w.subdomain, w.coarse, w.q)
        self.md = monodomain.Monodomain(self.d, w.stimulus, u0=w.u_rest, solver="pcg",
                                        prec=S.apply, rtol=1e-8, ionic_form=ionic_form)

    def steps(self, k):
        """k timed steps: (seconds per step, seconds of the ionic update + right-hand side
        per step, PCG iterations per step).  The right-hand side is timed by one extra
        evaluation before each step (it has no side effect on the state)."""
        t_step, t_rhs = 0.0, 0.0
        for _ in range(k):
            t0 = time.perf_counter()
            self.md.rhs(self.md.state)
            t1 = time.perf_counter()
            self.md.step()
            t2 = time.perf_counter()
            t_rhs += t1 - t0
            t_step += t2 - t1
        return t_step / k, t_rhs / k, sum(self.md.iterations[-k:]) / k


def on_cores(n, fn):
    """fn() with this process pinned to its first n allowed cores (None: all of them);
    returns (fn(), cores used)."""
    allowed = sorted(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else None
    if n is None or allowed is None:
        return fn(), (len(allowed) if allowed else os.cpu_count())
    try:
        os.sched_setaffinity(0, set(allowed[:n]))
        return fn(), min(n, len(allowed))
    finally:
        os.sched_setaffinity(0, set(allowed))


def sub_workload(name):
    """The oracle's sub-problem of a workload: the same recipe on a smaller mesh."""
    if name.startswith("hex"):
        from synth import hex_cube_p2
        return hex_cube_p2(n=8)
    from synth import voronoi4096_p3
    return voronoi4096_p3(n_cells=1024, n_parts=16)


def cpu_baseline(name, w_full, n_full, its_gpu, steps=3, warm=1, ionic_form="nodal"):
    """The oracle timed on whole steps of the workload's sub-problem (the same recipe on a
    smaller mesh), on one core and on all cores, and scaled to the workload: by the DOF
    ratio (the oracle's work per step grows linearly with the cells at a fixed iteration
    count) and, for the PCG part, by the ratio of the GPU's iteration count at full size
    to the oracle's on the sub-problem."""
    w = sub_workload(name)
    o = Oracle(w, ionic_form)
    o.steps(warm)
    n_sub = o.d.n_dofs
    (t1, r1, it1), c1 = on_cores(1, lambda: o.steps(steps))
    (ta, ra, ita), ca = on_cores(None, lambda: o.steps(steps))
    scale = n_full / n_sub

    def est(t, r, it):
        return scale * (r + (t - r) * its_gpu / max(it, 1e-9))

    sample = (f"{steps} whole oracle steps (after {warm} warm-up) of the same recipe on "
              f"{w.name} ({w.mesh.n_cells} cells, {n_sub} DOFs, {len(set(w.subdomain.tolist()))} "
              f"subdomains): {ta:.3f} s/step on {ca} cores ({ra:.3f} s ionic update + RHS, "
              f"{ita:.1f} PCG iterations), {t1:.3f} s/step on 1 core; scaled by the DOF ratio "
              f"{scale:.1f} and, for the PCG part, by {its_gpu:.1f}/{ita:.1f} iterations "
              f"(the fp64 plain GPU form's at full size over the oracle's)")
    return {"value": 1.0 / est(ta, ra, ita), "unit": "time-steps/s", "cores": ca, "kind": "oracle",
            "sample": sample,
            "one_core": {"value": 1.0 / est(t1, r1, it1), "unit": "time-steps/s", "cores": c1},
            "sub_problem_steps_per_s": {"all_cores": 1.0 / ta, "one_core": 1.0 / t1}}


def run_reference(args):
    """Reference arm: the float64 CPU oracle of the same method, whole time steps of the
    workload's stated sub-problem, scaled to the workload by the DOF ratio."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if args.workload == "batch32":
        name, n_full, label = "voronoi", None, BATCH_WORKLOAD
    elif args.workload.startswith("hex"):
        n = int(args.workload[3:])
        name, n_full = args.workload, 10 * n ** 3
        label = HEX_WORKLOAD.format(n=n, dofs=n_full, subs=(n // 4) ** 3, n0=4 * (n // 4) ** 3)
    else:
        name, n_full, label = "voronoi4096", 40960, WORKLOAD
    if n_full is None:                       # batch32: all simulations' DOFs
        from synth import voronoi_batch
        n_full = sum(10 * w.mesh.n_cells for w in voronoi_batch())
    o = Oracle(sub_workload(name), args.ionic_form)
    o.steps(args.warmup)
    t_step, t_rhs, its = o.steps(args.steps)
    scale = n_full / o.d.n_dofs
    value = 1.0 / (t_step * scale)
    if args.workload == "batch32":
        value *= 32                          # simulation-steps/s of the 32 simulations
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    w = o.w
    sample = (f"per timed step one whole oracle time step of the same recipe on {w.name} "
              f"({w.mesh.n_cells} cells, {o.d.n_dofs} DOFs; {t_step:.3f} s, {its:.1f} PCG "
              f"iterations), scaled to the workload by the DOF ratio {scale:.1f}")
    unit = "simulation-steps/s" if args.workload == "batch32" else "time-steps/s"
    line = {"metric": METRIC, "value": value, "unit": unit, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": label, "form": "FP64 oracle, plain ASM-PCG, x0 = U^k",
                       "ms_per_step_is": "the measured time of one sampled (sub-problem) step"},
            "cpu_baseline": {"value": value, "unit": unit, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: the workload's steps minus the warm-up)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["hex48", "voronoi4096", "batch32", "hex32", "hex24", "hex16"],
                    default="hex48")
    ap.add_argument("--ionic-form", choices=["nodal", "modal"], default="nodal")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.steps is None:
        args.steps = (200 if args.workload == "voronoi4096" else 100 if args.workload == "batch32"
                      else 50) - args.warmup
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_2512_19536_gb300 as pd
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl")
    stream = torch.cuda.current_stream()
    if args.workload == "batch32":
        return bench_batch(args, pd, torch, stream, rank, world, local)
    if args.workload.startswith("hex"):
        return bench_hex(args, pd, torch, stream, rank, world, local)
    line = bench_voronoi(args, pd, torch, stream, rank, world, local,
                         with_cpu=rank == 0 and world == 1 and not args.no_cpu_baseline)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def bench_voronoi(args, pd, torch, stream, rank, world, local, with_cpu, steps=None, clocks=None):
    """The 2D workload (4096-cell Voronoi, P3): its forms, roofline and CPU baseline."""
    steps = steps or args.steps
    w = build_case()
    ctx = pd.polydg_setup(w.mesh.vertices, w.mesh.cell_ptr, w.mesh.cell_vtx, w.sigma, w.p,
                          w.subdomain, w.chi_cm, w.dt, w.eta0)
    peaks, peak_kind = measured_peaks()
    form = args.ionic_form
    guess = load_guess(pd)
    clocks = clocks or ClockSampler(local)
    pc, sim, st, ms = time_form(pd, torch, w, ctx, "fp32", True, steps, args.warmup,
                                stream, clocks, guess=guess, policy=GUESS_POLICY, ionic_form=form)
    _, _, st_ng, ms_ng = time_form(pd, torch, w, ctx, "fp32", True, steps, args.warmup,
                                   stream, pc=pc, ionic_form=form)
    _, _, st_h, ms_h = time_form(pd, torch, w, ctx, "fp32", True, steps, args.warmup,
                                 stream, pc=pc, policy=GUESS_POLICY, ionic_form=form)
    if guess is not None:
        _, _, st_p, ms_p = time_form(pd, torch, w, ctx, "fp32", True, steps, args.warmup,
                                     stream, pc=pc, guess=guess, policy=0, ionic_form=form)
    else:
        st_p, ms_p = st_ng, ms_ng
    pc64, sim64, st64, ms64 = time_form(pd, torch, w, ctx, "fp64", False, steps,
                                        args.warmup, stream, ionic_form=form)
    _, _, stpp, mspp = time_form(pd, torch, w, ctx, "fp64", 2, steps, args.warmup, stream, pc=pc64,
                                 ionic_form=form)
    e2e_val, h2d, d2h = time_e2e(pd, torch, w, ctx, pc, steps, stream, guess, warm=args.warmup,
                                 ionic_form=form)
    (ms, ms64, ms_ng), (e2e_rank,) = reduce_over_ranks(torch, [ms, ms64, ms_ng], [e2e_val], world, "cuda")
    value = world * steps / (ms * 1e-3)
    value64 = world * steps / (ms64 * 1e-3)
    value_ng = world * steps / (ms_ng * 1e-3)
    info = pc.info()
    launches = st["steps_done"]
    alg = algorithmic_bytes(ctx.info, info, st["total_iterations"], launches)
    achieved = alg / st["pcg_seconds"] / 1e9
    traffic = profile_traffic("pcg_persistent_voronoi4096_fp32.txt",
                              st["total_iterations"] / max(1, launches), 1.0)
    cpu = None
    if with_cpu:
        its64 = st64["total_iterations"] / max(1, st64["steps_done"])
        cpu = cpu_baseline("voronoi4096", w, ctx.n_dofs, its64, steps=2, warm=1, ionic_form=form)
    return {
        "metric": METRIC, "value": value, "unit": "time-steps/s", "n_gpus": world,
        "steps": steps, "warmup": args.warmup, "ms_per_step": ms / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD,
                   "form": ("mixed + learned: fp32 local inverses, flexible PCG; initial guess = "
                            "Galerkin projection onto the network's proposal and the last 24 "
                            "solution increments") if guess is not None else
                   "mixed: fp32 local inverses, flexible PCG, initial guess from the last 24 "
                   "solution increments (guess weights file missing)",
                   "ionic_form": form,
                   "rtol": 1e-8, "iterations_per_step": st["total_iterations"] / steps,
                   "guess_taken_steps": st.get("guesses_taken", 0),
                   "pcg_ms_per_step": 1e3 * st["pcg_seconds"] / steps,
                   "non_pcg_ms_per_step": (ms - 1e3 * st["pcg_seconds"]) / steps,
                   "mixed_without_guess_steps_per_s": value_ng,
                   "mixed_without_guess_iterations_per_step": st_ng["total_iterations"] / steps,
                   "ablation_increments_only_steps_per_s": world * steps / (ms_h * 1e-3),
                   "ablation_increments_only_iterations_per_step": st_h["total_iterations"] / steps,
                   "ablation_proposal_only_steps_per_s": world * steps / (ms_p * 1e-3),
                   "ablation_proposal_only_iterations_per_step": st_p["total_iterations"] / steps,
                   "ablation_proposal_only_taken_steps": st_p.get("guesses_taken", 0),
                   "fp64_plain_steps_per_s": value64,
                   "fp64_plain_iterations_per_step": st64["total_iterations"] / steps,
                   "fp64_pipelined_steps_per_s": world * steps / (mspp * 1e-3),
                   "fp64_pipelined_iterations_per_step": stpp["total_iterations"] / steps,
                   "fp64_pipelined_pcg_ms_per_step": 1e3 * stpp["pcg_seconds"] / steps,
                   "fp64_plain_pcg_ms_per_step": 1e3 * st64["pcg_seconds"] / steps,
                   "mixed_over_fp64": value / value64,
                   "l2_keep_fraction": info["l2_keep_permille"] / 1000.0,
                   "l2": "working set > L2 (no flush needed)",
                   "parallelism": f"replicas x{world}"},
        "clocks": clocks.summary(),
        "e2e": {"value": world * e2e_rank, "unit": "time-steps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": (12 if guess is not None else 10) * steps,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                     "kernel": "pcg_persistent_kernel<fp32 store, n_p=10>",
                     "peak_kind": peak_kind},
        "cpu_baseline": cpu,
    }


def bench_hex(args, pd, torch, stream, rank, world, local):
    """The 3D workload (default 48^3 jittered hexahedra, P2): its 50 coupled steps (warm-up
    included) in the mixed + learned, increments-only, x0 = U^k and fp64 plain forms; then
    the 2D workload's forms for config.voronoi4096."""
    from synth import hex_cube_p2
    n = int(args.workload[3:])
    w = hex_cube_p2(n=n)
    steps = min(args.steps, w.n_steps - args.warmup)
    form = args.ionic_form
    t0 = time.perf_counter()
    ctx = pd.setup_mesh(w.mesh, w.sigma, w.p, w.subdomain, w.chi_cm, w.dt, w.eta0)
    t_setup = time.perf_counter() - t0
    peaks, peak_kind = measured_peaks()
    guess = load_guess(pd)
    clocks = ClockSampler(local)
    t0 = time.perf_counter()
    pc, _, st, ms = time_form(pd, torch, w, ctx, "fp32", True, steps, args.warmup, stream,
                              clocks, guess=guess, policy=GUESS_POLICY, ionic_form=form)
    t_form = time.perf_counter() - t0
    _, _, st_h, ms_h = time_form(pd, torch, w, ctx, "fp32", True, steps, args.warmup,
                                 stream, pc=pc, policy=GUESS_POLICY, ionic_form=form)
    _, _, st_ng, ms_ng = time_form(pd, torch, w, ctx, "fp32", True, steps, args.warmup,
                                   stream, pc=pc, ionic_form=form)
    e2e_val, h2d, d2h = time_e2e(pd, torch, w, ctx, pc, steps, stream, guess, warm=args.warmup,
                                 ionic_form=form)
    info = pc.info()
    pc.close()
    torch.cuda.empty_cache()
    pc64, _, st64, ms64 = time_form(pd, torch, w, ctx, "fp64", False, steps, args.warmup, stream,
                                    ionic_form=form)
    _, _, stpp, mspp = time_form(pd, torch, w, ctx, "fp64", 2, steps, args.warmup, stream, pc=pc64,
                                 ionic_form=form)
    pc64.close()
    (ms, ms64, ms_ng, ms_h), (e2e_rank,) = reduce_over_ranks(torch, [ms, ms64, ms_ng, ms_h], [e2e_val],
                                                             world, "cuda")
    value = world * steps / (ms * 1e-3)
    value64 = world * steps / (ms64 * 1e-3)
    its = st["total_iterations"] / max(1, st["steps_done"])
    alg = algorithmic_bytes(ctx.info, info, st["total_iterations"], st["steps_done"])
    achieved = alg / st["pcg_seconds"] / 1e9
    traffic = profile_traffic(f"pcg_persistent_hex{n}_fp32.txt", its, 1.0)
    cpu = None
    its64 = st64["total_iterations"] / max(1, st64["steps_done"])
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload, w, ctx.n_dofs, its64, ionic_form=form)
    ctx.close()
    torch.cuda.empty_cache()
    # the 2D workload in the same run
    vor = bench_voronoi(args, pd, torch, stream, rank, world, local, with_cpu=False, steps=20)
    pcg_ms = 1e3 * st["pcg_seconds"] / steps
    line = {
        "metric": METRIC, "value": value, "unit": "time-steps/s",
        "n_gpus": world, "steps": steps, "warmup": args.warmup, "ms_per_step": ms / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32",
        "data": "synthetic",
        "config": {"workload": HEX_WORKLOAD.format(n=n, dofs=10 * n ** 3, subs=(n // 4) ** 3,
                                                   n0=4 * (n // 4) ** 3),
                   "form": "mixed + learned: fp32 local inverses, flexible PCG (fp64 residual, dots, "
                           "coarse solve, matvec); initial guess = Galerkin projection onto the "
                           "network's proposal (trained on 2D Voronoi P3 trajectories of the plain "
                           "solver, seeds 0-7) and the last 24 solution increments; the gain over "
                           "fp64 plain is the fp32 inverses' and the increments' (see the "
                           "increments-only ablation: the network's direction does not help on this "
                           "mesh)",
                   "ionic_form": form,
                   "rtol": 1e-8, "iterations_per_step": its,
                   "guess_taken_steps": st.get("guesses_taken", 0),
                   "pcg_ms_per_step": pcg_ms,
                   "non_pcg_ms_per_step": ms / steps - pcg_ms,
                   "ablation_increments_only_steps_per_s": world * steps / (ms_h * 1e-3),
                   "ablation_increments_only_iterations_per_step": st_h["total_iterations"] / steps,
                   "mixed_without_guess_steps_per_s": world * steps / (ms_ng * 1e-3),
                   "mixed_without_guess_iterations_per_step": st_ng["total_iterations"] / steps,
                   "fp64_plain_steps_per_s": value64,
                   "fp64_plain_iterations_per_step": its64,
                   "fp64_pipelined_steps_per_s": world * steps / (mspp * 1e-3),
                   "fp64_pipelined_iterations_per_step": stpp["total_iterations"] / steps,
                   "fp64_pipelined_pcg_ms_per_step": 1e3 * stpp["pcg_seconds"] / steps,
                   "fp64_plain_pcg_ms_per_step": 1e3 * st64["pcg_seconds"] / steps,
                   "mixed_over_fp64": value / value64,
                   "setup_s": {"polydg_setup3d": t_setup,
                               "asm_setup_autotune_and_first_form": t_form},
                   "l2": "working set > L2 (no flush needed)",
                   "parallelism": f"replicas x{world}",
                   "voronoi4096": {k: vor[k] for k in ("value", "ms_per_step", "e2e", "roofline")}
                   | {k: vor["config"][k] for k in ("workload", "iterations_per_step",
                                                    "fp64_plain_steps_per_s",
                                                    "fp64_plain_iterations_per_step",
                                                    "fp64_pipelined_steps_per_s",
                                                    "fp64_plain_pcg_ms_per_step",
                                                    "fp64_pipelined_pcg_ms_per_step",
                                                    "ablation_increments_only_steps_per_s",
                                                    "mixed_without_guess_steps_per_s",
                                                    "guess_taken_steps")}},
        "clocks": clocks.summary(),
        "e2e": {"value": world * e2e_rank, "unit": "time-steps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": (12 if guess is not None else 10) * steps,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                     "kernel": "pcg_persistent_kernel<fp32 store, n_p=10> (distributed coarse rows)",
                     "peak_kind": peak_kind},
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def bench_batch(args, pd, torch, stream, rank, world, local):
    """Batched forms: simulation-steps/s of 32 simulations of uneven sizes."""
    import numpy as np
    from synth import voronoi_batch
    ws = voronoi_batch()
    peaks, peak_kind = measured_peaks()
    S = len(ws)
    per_mesh = 4
    steps = min(args.steps, ws[0].n_steps - args.warmup)     # the workload's steps
    guess = load_guess(pd)

    def make(prec, flex, with_guess):
        out = []
        for w in ws:
            ctx = pd.polydg_setup(w.mesh.vertices, w.mesh.cell_ptr, w.mesh.cell_vtx, w.sigma,
                                  w.p, w.subdomain, w.chi_cm, w.dt, w.eta0)
            pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision=prec)
            sim = pd.sim_create(ctx, pc, u0=w.u_rest, stimulus=w.stimulus, rtol=1e-8,
                                maxit=5000, flexible=flex)
            if with_guess:
                pd.sim_set_guess(sim, guess, GUESS_POLICY)
            out.append((ctx, pc, sim))
        return out

    def timed_batch(trip, clocks=None):
        sims = [x[2] for x in trip]
        bt = pd.batch_create(sims)
        pd.batch_step(bt, args.warmup, stream)
        if torch.distributed.is_initialized():
            torch.distributed.barrier()
        torch.cuda.synchronize()
        if clocks is not None:
            clocks.__enter__()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        st, sec = pd.batch_step(bt, steps, stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        if clocks is not None:
            clocks.__exit__(None, None, None)
        return bt, st, sec, ev0.elapsed_time(ev1)

    # candidate: one bf16 eigenbasis per mesh shared by its 4 simulations (lockstep groups)
    trip = make("fp32", True, True)
    t0 = time.perf_counter()
    shared = []
    for m0 in range(0, S, per_mesh):
        sl = pd.shared_local_setup(trip[m0][0], "bf16")
        shared.append(sl)
        for k in range(m0, m0 + per_mesh):
            pd.sim_set_shared_local(trip[k][2], sl)
    t_eig = time.perf_counter() - t0
    clocks = ClockSampler(local)
    bt, st, sec, ms = timed_batch(trip, clocks)
    its = [s_["total_iterations"] / steps for s_ in st]
    # algorithmic bytes: per group iteration the shared store once plus every member's K_h,
    # coarse and vectors; group iterations >= the largest member's
    alg = 0.0
    for g, sl in enumerate(shared):
        mem = range(g * per_mesh, (g + 1) * per_mesh)
        g_its = max(st[k]["total_iterations"] for k in mem)
        per_it = sl.info()["store_bytes"]
        for k in mem:
            ctx, pc, _ = trip[k]
            inf = pc.info()
            per_it += (8 * ctx.info.n_p ** 2 * ctx.info.n_blocks + inf["coarse_bytes"]
                       + inf["restrict_bytes"] + 12 * 8 * ctx.n_dofs)
        alg += g_its * per_it
    achieved = alg / (sec * 1e9)
    # e2e: every simulation's state (the last 25 solutions the initial guess reads) through
    # pinned host memory each step, the new potential back
    sims = [x[2] for x in trip]
    n_all = sum(ctx.n_dofs for ctx, _, _ in trip)
    H = 25
    hh = [HostHistory(torch, H, ctx.n_dofs) for ctx, _, _ in trip]
    dh = [torch.empty((H, ctx.n_dofs), dtype=torch.float64, device="cuda") for ctx, _, _ in trip]
    du = [torch.empty(ctx.n_dofs, dtype=torch.float64, device="cuda") for ctx, _, _ in trip]
    # a fresh batch of the same form, its warm-up steps recorded on the host
    del bt
    trip_e = make("fp32", True, True)
    for m0 in range(0, S, per_mesh):
        for k in range(m0, m0 + per_mesh):
            pd.sim_set_shared_local(trip_e[k][2], shared[m0 // per_mesh])
    sims = [x[2] for x in trip_e]
    bt = pd.batch_create(sims)
    for _ in range(args.warmup):
        pd.batch_step(bt, 1, stream)
        for s_, d_, h_ in zip(sims, du, hh):
            pd.sim_get_state(s_, d_, stream=stream)
            h_.push_from(d_)
    torch.cuda.synchronize()
    e_steps = steps
    t0 = time.perf_counter()
    for _ in range(e_steps):
        for s_, d_, h_ in zip(sims, dh, hh):
            h_.upload(d_)
            pd.sim_set_history(s_, d_[:h_.count], stream)
        pd.batch_step(bt, 1, stream)
        for s_, d_, h_ in zip(sims, du, hh):
            pd.sim_get_state(s_, d_, stream=stream)
            h_.push_from(d_, non_blocking=True)
        torch.cuda.synchronize()
    e2e_rate = S * e_steps / (time.perf_counter() - t0)
    groups = bt.groups().tolist()
    bt.close()
    del trip, trip_e, sims, shared, du, dh, hh
    torch.cuda.empty_cache()
    # the same simulations with their own fp32 local inverses, one CTA group each
    trip32 = make("fp32", True, True)
    bt32, st32, _, ms32 = timed_batch(trip32)
    its32 = [s_["total_iterations"] / steps for s_ in st32]
    bt32.close()
    del trip32
    torch.cuda.empty_cache()
    # baseline: fp64 plain form, one simulation after another
    trip64 = make("fp64", False, False)
    for _, _, s_ in trip64:
        pd.monodomain_step(s_, args.warmup, stream)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    its64 = []
    for _, _, s_ in trip64:
        its64.append(pd.monodomain_step(s_, steps, stream)["total_iterations"] / steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms64 = ev0.elapsed_time(ev1)
    (ms, ms32, ms64), (e2e_rate,) = reduce_over_ranks(torch, [ms, ms32, ms64], [e2e_rate], world, "cuda")
    e2e_val = world * e2e_rate
    value = world * S * steps / (ms * 1e-3)
    value32 = world * S * steps / (ms32 * 1e-3)
    value64 = world * S * steps / (ms64 * 1e-3)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # whole oracle steps of the 1024-cell recipe, scaled by DOFs to all 32 simulations
        cpu = cpu_baseline("voronoi", None, n_all, float(np.mean(its64)), steps=2, warm=1)
        for key in ("value",):
            cpu[key] *= S
        cpu["one_core"]["value"] *= S
        cpu["unit"] = cpu["one_core"]["unit"] = "simulation-steps/s"
    line = {
        "metric": METRIC + " (batched form)", "value": value, "unit": "simulation-steps/s",
        "n_gpus": world, "steps": steps, "warmup": args.warmup,
        "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32+bf16", "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD,
                   "form": "batched + shared eigenbasis + learned: the 4 simulations of each mesh "
                           "solve in lockstep, each subdomain's local solves one bf16 pass over Q_i^T "
                           "and one over Q_i for all 4 (flexible PCG, fp64 residual/dots/coarse/"
                           "matvec); every simulation's initial guess the Galerkin projection onto "
                           "the network's proposal and its last 24 solution increments; one "
                           "persistent launch per step, captured step graph",
                   "cells": [w.mesh.n_cells for w in ws[::per_mesh]], "dofs": n_all,
                   "ctas_per_sim": groups, "iterations_per_step": its,
                   "eigenbasis_setup_s": t_eig,
                   "batched_fp32_inverses_sim_steps_per_s": value32,
                   "batched_fp32_inverses_iterations_per_step": its32,
                   "fp64_plain_per_sim_launches_sim_steps_per_s": value64,
                   "fp64_plain_iterations_per_step": its64,
                   "shared_over_fp64_plain": value / value64,
                   "l2": "working set > L2 (no flush needed)", "parallelism": f"replicas x{world}"},
        "clocks": clocks.summary(),
        "e2e": {"value": e2e_val, "unit": "simulation-steps/s",
                "h2d_bytes_per_step": 25 * 8 * n_all, "d2h_bytes_per_step": 8 * n_all},
        "gpu_launches": ((11 if guess is not None else 9) * S + 1) * steps,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                     "kernel": "pcg_group_kernel<bf16 store, n_p=10> (whole step time)",
                     "peak_kind": peak_kind},
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def profile_traffic(fname, iterations_per_launch, scale=1.0):
    """DRAM bytes per launch of the persistent kernel from a committed ncu summary
    (profiles/<fname>: dram_bytes_per_iteration), times this run's iterations per launch;
    None if the summary is missing or the kernel source changed since the counters were
    taken."""
    path = os.path.join(ROOT, "profiles", fname)
    try:
        kv = {}
        with open(path) as f:
            for line in f:
                if ":" in line:
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel_source_sha") != kernel_sha():
            return None
        return float(kv["dram_bytes_per_iteration"]) * iterations_per_launch * scale
    except (OSError, KeyError, ValueError):
        return None


def kernel_sha():
    """Hash of what the persistent PCG kernel is compiled from: its source, its device
    helpers and the argument structures it reads (the rest of kernels.h declares other
    launchers and does not change the kernel)."""
    import hashlib
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2512_19536_gb300", "csrc")
    for name in ("kernels_pcg.cu", "device.cuh", "pcg_device.cuh"):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    with open(os.path.join(csrc, "kernels.h")) as f:
        text = f.read()
    for struct in ("GridSync", "PersistArgs"):
        m = re.search(r"struct %s \{.*?\n\};" % struct, text, flags=re.S)
        h.update(m.group(0).encode() if m else b"")
    return h.hexdigest()[:16]


if __name__ == "__main__":
    sys.exit(main())
