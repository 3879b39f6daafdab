#!/usr/bin/env python3
"""Benchmark: ASM-PCG time-steps/s on the coupled PolyDG monodomain + Barreto-Cressman
workload (4096-cell Voronoi mesh of the unit square, P3, anisotropic fibre
conductivity, 64 k-means subdomains = coarse agglomerates, coarse P1, dt = 0.05 ms,
Gaussian stimulus), every step solved by PCG with the two-level additive Schwarz
preconditioner to |r|_2 <= 1e-8 |b|_2 on one GB300.

A "step" is one Crank-Nicolson time step through the C ABI (monodomain_step):
ionic update at the quadrature nodes, right-hand side, initial guess, and the
persistent PCG kernel.  By default the 3 warm-up and 197 timed steps together are the
workload's 200 steps.  Three forms are timed on the same setup:
  * mixed + learned: fp32 local inverses in flexible PCG (fp64 residual, dots, coarse
    solve and matvec) with the learned initial guess (the network trained by
    paper_2512_19536_gb300/guess_train.py on eight other meshes' trajectories, weights in
    paper_2512_19536_gb300/guess_p3_voronoi4096.npz; kept per step only if its residual
    is smaller than U^k's) -- the reported value;
  * mixed: the same with x0 = U^k;
  * fp64 plain: fp64 local inverses in standard PCG, x0 = U^k.
Each preconditioner's split of its work over the CTAs is autotuned at setup
(asm_autotune, six rounds: 26 solves of 60 timed iterations each), which is not part of
the timed steps.
The working set (fp32 store 112 MB + K_h 22.5 MB + vectors) exceeds the 126 MB
L2, so no L2 flush is inserted between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload voronoi4096|batch32]
Under torchrun (N > 1) every rank runs an independent replica (the path has no
exchange step); rank 0 prints one JSON line with the whole-job throughput.

--workload batch32 times the batched forms instead: 32 independent simulations on 8
Voronoi meshes of 1024-16384 cells (log-uniform), 4 per mesh with scalar
conductivities U[0.5, 2] and random stimulus sites.  Reported: the 4 simulations of each
mesh in lockstep sharing one bf16 eigenbasis of every subdomain (all solves of a step in
one persistent launch); beside it the batched form with each simulation's own fp32
inverses and the fp64 plain form stepped one simulation after another; the unit is
simulation-steps/s.
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


GUESS_POLICY = 3   # Galerkin projection onto the learned proposal and the last 16 solution increments


def time_form(pd, torch, w, ctx, precision, flexible, steps, warmup, stream, clocks=None,
              guess=None, pc=None, policy=None):
    if pc is None:
        pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision=precision)
        pd.asm_autotune(pc, rounds=6, iterations=60)   # setup: re-cut the rows by measured CTA times
    sim = pd.sim_create(ctx, pc, u0=w.u_rest, stimulus=w.stimulus, rtol=1e-8, maxit=5000,
                        flexible=flexible)
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


def time_e2e(pd, torch, w, ctx, pc, steps, stream, guess=None, warm=12):
    """Same metric with the state crossing the host boundary every step: the last
    solutions the step depends on (U^k .. U^{k-16}: the initial guess reads them) copied in
    from pinned host memory and restored with sim_set_history, U^{k+1} copied back to
    pinned host memory.  The same steps as the device-timed forms: `warm` untimed, then
    `steps` timed."""
    sim = pd.sim_create(ctx, pc, u0=w.u_rest, stimulus=w.stimulus, rtol=1e-8, maxit=5000,
                        flexible=True)
    pd.sim_set_guess(sim, guess, GUESS_POLICY)
    n = ctx.n_dofs
    H = 17
    host_hist = torch.empty((H, n), dtype=torch.float64).pin_memory()   # row 0 = U^k
    dev_hist = torch.empty((H, n), dtype=torch.float64, device="cuda")
    dev_u = torch.empty(n, dtype=torch.float64, device="cuda")
    host_new = torch.empty(n, dtype=torch.float64).pin_memory()
    sols = []
    for _ in range(warm):
        pd.monodomain_step(sim, 1, stream)
        pd.sim_get_state(sim, dev_u, stream=stream)
        sols.append(dev_u.cpu())
    host_hist.zero_()
    for h in range(min(H, len(sols))):
        host_hist[h].copy_(sols[-1 - h])
    count = min(H, len(sols))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        dev_hist.copy_(host_hist, non_blocking=True)
        pd.sim_set_history(sim, dev_hist[:count], stream)
        count = min(H, count + 1)
        pd.monodomain_step(sim, 1, stream)
        pd.sim_get_state(sim, dev_u, stream=stream)
        host_new.copy_(dev_u, non_blocking=True)
        torch.cuda.synchronize()
        host_hist[1:].copy_(host_hist[:-1].clone())
        host_hist[0].copy_(host_new)
    dt = time.perf_counter() - t0
    sim.close()
    return steps / dt, H * 8 * n, 8 * n


def cpu_baseline(w, its_per_step, sample_its=40):
    """The oracle (oracle.monodomain with oracle.pcg and oracle.schwarz, float64 on
    the host cores) timed on a bounded sample: one right-hand side (ionic update and
    load) and `sample_its` ASM-PCG iterations, extrapolated to `its_per_step`."""
    import numpy as np
    from oracle import assembly, schwarz, monodomain
    from oracle.pcg import pcg
    d = assembly.assemble(w.mesh, w.p, w.sigma, w.eta0, w.chi_cm, w.dt)
    S = schwarz.build(d, w.subdomain, w.coarse, w.q)
    md = monodomain.Monodomain(d, w.stimulus, u0=w.u_rest, solver="pcg", prec=S.apply, rtol=1e-8)
    t0 = time.perf_counter()
    b, _ = md.rhs(md.state)
    t_rhs = time.perf_counter() - t0
    t0 = time.perf_counter()
    pcg(d.K, b, x0=np.zeros_like(b), prec=S.apply, rtol=1e-30, maxit=sample_its)
    t_it = (time.perf_counter() - t0) / sample_its
    t_step = t_rhs + its_per_step * t_it
    return t_step, t_rhs, t_it


def run_reference(args):
    """Reference arm: the FP64 CPU oracle of the same method on the same workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = build_case()
    import numpy as np
    from oracle import assembly, schwarz, monodomain
    from oracle.pcg import pcg
    d = assembly.assemble(w.mesh, w.p, w.sigma, w.eta0, w.chi_cm, w.dt)
    S = schwarz.build(d, w.subdomain, w.coarse, w.q)
    md = monodomain.Monodomain(d, w.stimulus, u0=w.u_rest, solver="pcg", prec=S.apply, rtol=1e-8)
    sample_its = 10
    # one full step fixes the iteration count that each sampled step is scaled to
    b, _ = md.rhs(md.state)
    full = pcg(d.K, b, x0=md.state.U, prec=S.apply, rtol=1e-8)
    its = full.iterations
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        b, _ = md.rhs(md.state)
        t_rhs = time.perf_counter() - t0
        t0 = time.perf_counter()
        pcg(d.K, b, x0=md.state.U, prec=S.apply, rtol=1e-30, maxit=sample_its)
        t_it = (time.perf_counter() - t0) / sample_its
        if k >= args.warmup:
            times.append(t_rhs + its * t_it)
    total = sum(times)
    value = len(times) / total
    cores = os.cpu_count()
    line = {"metric": METRIC, "value": value, "unit": "time-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "form": "FP64 oracle, plain ASM-PCG"},
            "cpu_baseline": {"value": value, "unit": "time-steps/s", "cores": cores,
                             "kind": "oracle",
                             "sample": f"per step: ionic update + RHS and {sample_its} ASM-PCG "
                                       f"iterations, scaled to the {its} iterations of a full "
                                       "step solved once beforehand"},
            "e2e": {"value": value, "unit": "time-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=197)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["voronoi4096", "batch32", "hex48", "hex32", "hex24"], default="voronoi4096")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
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
    w = build_case()
    ctx = pd.polydg_setup(w.mesh.vertices, w.mesh.cell_ptr, w.mesh.cell_vtx, w.sigma, w.p,
                          w.subdomain, w.chi_cm, w.dt, w.eta0)
    peaks, peak_kind = measured_peaks()

    # reported form: mixed precision (fp32 local inverses, flexible PCG) + learned guess
    guess = load_guess(pd)
    clocks = ClockSampler(local)
    pc, sim, st, ms = time_form(pd, torch, w, ctx, "fp32", True, args.steps, args.warmup,
                                stream, clocks, guess=guess, policy=GUESS_POLICY)
    # the same without any initial guess (x0 = U^k)
    _, _, st_ng, ms_ng = time_form(pd, torch, w, ctx, "fp32", True, args.steps, args.warmup,
                                   stream, pc=pc)
    # ablations: the increments alone (no network), and the network's proposal alone
    # (kept only when its residual is below U^k's)
    _, _, st_h, ms_h = time_form(pd, torch, w, ctx, "fp32", True, args.steps, args.warmup,
                                 stream, pc=pc, policy=GUESS_POLICY)
    if guess is not None:
        _, _, st_p, ms_p = time_form(pd, torch, w, ctx, "fp32", True, args.steps, args.warmup,
                                     stream, pc=pc, guess=guess, policy=0)
    else:
        st_p, ms_p = st_ng, ms_ng
    # fp64 plain form on the same workload, for the comparison the metric names
    pc64, sim64, st64, ms64 = time_form(pd, torch, w, ctx, "fp64", False, args.steps,
                                        args.warmup, stream)
    e2e_val, h2d, d2h = time_e2e(pd, torch, w, ctx, pc, args.steps, stream, guess, warm=args.warmup)
    (ms, ms64, ms_ng), (e2e_rank,) = reduce_over_ranks(torch, [ms, ms64, ms_ng], [e2e_val], world, "cuda")
    value = world * args.steps / (ms * 1e-3)
    value64 = world * args.steps / (ms64 * 1e-3)
    value_ng = world * args.steps / (ms_ng * 1e-3)
    e2e_val = world * e2e_rank

    info = pc.info()
    launches = st["steps_done"]
    alg = algorithmic_bytes(ctx.info, info, st["total_iterations"], launches)
    achieved = alg / st["pcg_seconds"] / 1e9
    traffic = profile_traffic(st["total_iterations"] / max(1, launches))
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                "kernel": "pcg_persistent_kernel<fp32 store, n_p=10>",
                "peak_kind": peak_kind}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        its64 = st64["total_iterations"] / max(1, st64["steps_done"])
        t_step, t_rhs, t_it = cpu_baseline(w, its64)
        cpu = {"value": 1.0 / t_step, "unit": "time-steps/s", "cores": os.cpu_count(),
               "kind": "oracle",
               "sample": f"one ionic update + RHS ({t_rhs:.2f} s) and 40 ASM-PCG iterations "
                         f"({t_it * 1e3:.1f} ms each) of the float64 oracle, scaled to "
                         f"{its64:.1f} iterations/step (the fp64 plain form's mean)"}

    line = {
        "metric": METRIC, "value": value, "unit": "time-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD,
                   "form": ("mixed + learned: fp32 local inverses, flexible PCG; initial guess = "
                            "Galerkin projection onto the network's proposal and the last 16 "
                            "solution increments (U^k when that does not lower the error)")
                   if guess is not None else
                   "mixed: fp32 local inverses, flexible PCG, initial guess from the last 16 "
                   "solution increments (guess weights file missing)",
                   "rtol": 1e-8, "iterations_per_step": st["total_iterations"] / args.steps,
                   "guess_taken_steps": st.get("guesses_taken", 0),
                   "mixed_without_guess_steps_per_s": value_ng,
                   "mixed_without_guess_iterations_per_step": st_ng["total_iterations"] / args.steps,
                   "ablation_increments_only_steps_per_s": world * args.steps / (ms_h * 1e-3),
                   "ablation_increments_only_iterations_per_step": st_h["total_iterations"] / args.steps,
                   "ablation_proposal_only_steps_per_s": world * args.steps / (ms_p * 1e-3),
                   "ablation_proposal_only_iterations_per_step": st_p["total_iterations"] / args.steps,
                   "ablation_proposal_only_taken_steps": st_p.get("guesses_taken", 0),
                   "fp64_plain_steps_per_s": value64,
                   "fp64_plain_iterations_per_step": st64["total_iterations"] / args.steps,
                   "mixed_over_fp64": value / value64,
                   "l2_keep_fraction": info["l2_keep_permille"] / 1000.0,
                   "l2": "working set > L2 (no flush needed)",
                   "parallelism": f"replicas x{world}"},
        "clocks": clocks.summary(),
        "e2e": {"value": e2e_val, "unit": "time-steps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": (10 if guess is not None else 9) * args.steps,
        "roofline": roofline,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def bench_hex(args, pd, torch, stream, rank, world, local):
    """The 3D workload: its 50 coupled steps (warm-up included) in the mixed + learned,
    mixed and fp64 plain forms."""
    from synth import hex_cube_p2
    n = int(args.workload[3:])
    w = hex_cube_p2(n=n)
    steps = min(args.steps, w.n_steps - args.warmup)
    ctx = pd.setup_mesh(w.mesh, w.sigma, w.p, w.subdomain, w.chi_cm, w.dt, w.eta0)
    peaks, peak_kind = measured_peaks()
    guess = load_guess(pd)
    clocks = ClockSampler(local)
    pc, _, st, ms = time_form(pd, torch, w, ctx, "fp32", True, steps, args.warmup, stream,
                              clocks, guess=guess, policy=GUESS_POLICY)
    _, _, st_ng, ms_ng = time_form(pd, torch, w, ctx, "fp32", True, steps, args.warmup,
                                   stream, pc=pc)
    _, _, st64, ms64 = time_form(pd, torch, w, ctx, "fp64", False, steps, args.warmup, stream)
    e2e_val, h2d, d2h = time_e2e(pd, torch, w, ctx, pc, steps, stream, guess, warm=args.warmup)
    (ms, ms64, ms_ng), (e2e_rank,) = reduce_over_ranks(torch, [ms, ms64, ms_ng], [e2e_val], world, "cuda")
    value = world * steps / (ms * 1e-3)
    value64 = world * steps / (ms64 * 1e-3)
    info = pc.info()
    alg = algorithmic_bytes(ctx.info, info, st["total_iterations"], st["steps_done"])
    achieved = alg / st["pcg_seconds"] / 1e9
    line = {
        "metric": METRIC + " (3D workload)", "value": value, "unit": "time-steps/s",
        "n_gpus": world, "steps": steps, "warmup": args.warmup, "ms_per_step": ms / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32",
        "data": "synthetic",
        "config": {"workload": HEX_WORKLOAD.format(n=n, dofs=10 * n ** 3, subs=(n // 4) ** 3,
                                                   n0=4 * (n // 4) ** 3),
                   "form": "mixed + learned: fp32 local inverses, flexible PCG; initial guess = "
                           "Galerkin projection onto the network's proposal (trained on 2D "
                           "Voronoi P3 trajectories) and the last 16 solution increments",
                   "rtol": 1e-8, "iterations_per_step": st["total_iterations"] / steps,
                   "guess_taken_steps": st.get("guesses_taken", 0),
                   "mixed_without_guess_steps_per_s": world * steps / (ms_ng * 1e-3),
                   "mixed_without_guess_iterations_per_step": st_ng["total_iterations"] / steps,
                   "fp64_plain_steps_per_s": value64,
                   "fp64_plain_iterations_per_step": st64["total_iterations"] / steps,
                   "mixed_over_fp64": value / value64,
                   "pcg_share_of_step": st["pcg_seconds"] * 1e3 / ms,
                   "l2": "working set > L2 (no flush needed)",
                   "parallelism": f"replicas x{world}"},
        "clocks": clocks.summary(),
        "e2e": {"value": world * e2e_rank, "unit": "time-steps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": (10 if guess is not None else 9) * steps,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                     "kernel": "pcg_persistent_kernel<fp32 store, n_p=10> (distributed coarse rows)",
                     "peak_kind": peak_kind},
        "cpu_baseline": None,
        "cpu_baseline_note": "the float64 oracle needs minutes per step at 1.1 M DOFs; its "
                             "parity is checked on the 4^3 and 10^3 cases and on sampled rows",
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
    # e2e: every simulation's state (the last 17 solutions the initial guess reads) through
    # pinned host memory each step, the new potential back
    sims = [x[2] for x in trip]
    n_all = sum(ctx.n_dofs for ctx, _, _ in trip)
    H = 17
    hh = [torch.zeros((H, ctx.n_dofs), dtype=torch.float64).pin_memory() for ctx, _, _ in trip]
    dh = [torch.empty((H, ctx.n_dofs), dtype=torch.float64, device="cuda") for ctx, _, _ in trip]
    du = [torch.empty(ctx.n_dofs, dtype=torch.float64, device="cuda") for ctx, _, _ in trip]
    hn = [torch.empty(ctx.n_dofs, dtype=torch.float64).pin_memory() for ctx, _, _ in trip]
    # a fresh batch of the same form, its warm-up steps recorded on the host
    del bt
    trip_e = make("fp32", True, True)
    for m0 in range(0, S, per_mesh):
        for k in range(m0, m0 + per_mesh):
            pd.sim_set_shared_local(trip_e[k][2], shared[m0 // per_mesh])
    sims = [x[2] for x in trip_e]
    bt = pd.batch_create(sims)
    count = 0
    for _ in range(args.warmup):
        pd.batch_step(bt, 1, stream)
        for s_, d_, h_ in zip(sims, du, hh):
            pd.sim_get_state(s_, d_, stream=stream)
            h_[1:].copy_(h_[:-1].clone())
            h_[0].copy_(d_)
        count = min(H, count + 1)
    torch.cuda.synchronize()
    e_steps = steps
    t0 = time.perf_counter()
    for _ in range(e_steps):
        for s_, d_, h_ in zip(sims, dh, hh):
            d_.copy_(h_, non_blocking=True)
            pd.sim_set_history(s_, d_[:count], stream)
        pd.batch_step(bt, 1, stream)
        for s_, d_, h_ in zip(sims, du, hn):
            pd.sim_get_state(s_, d_, stream=stream)
            h_.copy_(d_, non_blocking=True)
        torch.cuda.synchronize()
        for h_, n_ in zip(hh, hn):
            h_[1:].copy_(h_[:-1].clone())
            h_[0].copy_(n_)
        count = min(H, count + 1)
    e2e_rate = S * e_steps / (time.perf_counter() - t0)
    groups = bt.groups().tolist()
    bt.close()
    del trip, trip_e, sims, shared, du, dh, hh, hn
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
        # oracle on the smallest mesh's first simulation, scaled by DOFs to all 32
        k = int(np.argmin([w.mesh.n_cells for w in ws]))
        t_step, t_rhs, t_it = cpu_baseline(ws[k], its64[k], sample_its=10)
        scale = n_all / (ws[k].mesh.n_cells * 10)
        cpu = {"value": 1.0 / (t_step * scale) * S, "unit": "simulation-steps/s",
               "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"one step of the {ws[k].mesh.n_cells}-cell simulation (ionic update + "
                         f"RHS and 10 ASM-PCG iterations of the float64 oracle, scaled to "
                         f"{its64[k]:.0f} iterations), scaled by DOFs to all 32 simulations"}
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
                           "the network's proposal and its last 16 solution increments; one "
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
                "h2d_bytes_per_step": 17 * 8 * n_all, "d2h_bytes_per_step": 8 * n_all},
        "gpu_launches": ((9 if guess is not None else 8) * S + 1) * steps,
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


def profile_traffic(iterations_per_launch):
    """DRAM bytes per launch of the persistent kernel from the committed ncu summary,
    scaled to this run's iterations per launch; None if the kernel source changed
    since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "pcg_persistent_voronoi4096_fp32.txt")
    try:
        kv = {}
        with open(path) as f:
            for line in f:
                if ":" in line:
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel_source_sha") != kernel_sha():
            return None
        per_it = float(kv["dram_bytes_per_iteration"])
        return per_it * iterations_per_launch
    except (OSError, KeyError, ValueError):
        return None


def kernel_sha():
    import hashlib
    h = hashlib.sha256()
    for name in ("kernels_pcg.cu", "kernels.h", "device.cuh", "pcg_device.cuh"):
        with open(os.path.join(ROOT, "paper_2512_19536_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    sys.exit(main())
