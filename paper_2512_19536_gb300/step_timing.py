"""Device time of the coupled Crank-Nicolson step, per representation of the ionic state.

Runs the 4096-cell Voronoi P3 workload (anisotropic fibre conductivity, 64 k-means
subdomains = coarse cells, dt = 0.05 ms, Gaussian stimulus) with fp32 local inverses and
flexible PCG to rtol 1e-8 from x0 = U^k, once per ionic form ("nodal": explicit Euler at
every quadrature node; "modal": the DG-basis update of Eq. fully-discrete-1, second
line).  After `warmup` steps it times `steps` steps with CUDA events on the stream they
run on, and splits the time into the PCG launches (the library's own events) and the
rest of the step (ionic update, right-hand side, bookkeeping).  Prints one JSON line per
form.

Run on a GPU: python -m paper_2512_19536_gb300.step_timing [--forms nodal modal]
[--steps 20] [--warmup 3]
"""
from __future__ import annotations

import argparse
import json

from . import _native as pd


def time_form(form, steps, warmup):
    import torch
    from synth import voronoi4096_p3
    w = voronoi4096_p3()
    ctx = pd.setup_mesh(w.mesh, w.sigma, w.p, w.subdomain, w.chi_cm, w.dt, w.eta0)
    pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision="fp32")
    sim = pd.sim_create(ctx, pc, u0=w.u_rest, stimulus=w.stimulus, rtol=w.rtol, maxit=20000,
                        flexible=True)
    pd.sim_set_ionic_form(sim, form)
    stream = torch.cuda.current_stream()
    pd.monodomain_step(sim, warmup, stream=stream)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    st = pd.monodomain_step(sim, steps, stream=stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    total = ev0.elapsed_time(ev1)
    pcg = 1e3 * st["pcg_seconds"]
    out = {"form": form, "workload": "voronoi4096_p3", "steps": steps, "warmup": warmup,
           "ms_per_step": total / steps, "pcg_ms_per_step": pcg / steps,
           "rest_ms_per_step": (total - pcg) / steps,
           "iterations_per_step": st["total_iterations"] / steps, "status": st["status"]}
    sim.close()
    pc.close()
    ctx.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--forms", nargs="+", default=["nodal", "modal"], choices=["nodal", "modal"])
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    a = ap.parse_args(argv)
    for form in a.forms:
        print(json.dumps(time_form(form, a.steps, a.warmup)), flush=True)


if __name__ == "__main__":
    main()
