"""Run coupled time steps of a named synthetic workload through the C ABI and print one
JSON line per step (PCG iterations, relative residual, device time of the PCG launch).

A small driver for profilers and quick checks: it sets up the workload, the
preconditioner in the chosen precision (fp32/bf16 local inverses run flexible PCG) and
the initial-guess policy, then steps one step per call, so the n-th launch of each kernel
belongs to step n.  Workloads: hex<N> (N^3 jittered hexahedra, P2, subdomains of 4^3
cells = coarse agglomerates, coarse P1), voronoi<N> (N-cell Voronoi mesh, P3, k-means
subdomains of ~64 cells = coarse agglomerates, coarse P1).

    python -m paper_2512_19536_gb300.run_steps --workload hex24 --precision fp32 --steps 4
"""
from __future__ import annotations

import argparse
import json

from . import _native as pd


def make_workload(name):
    if name.startswith("hex"):
        from synth import hex_cube_p2
        return hex_cube_p2(n=int(name[3:]))
    from synth import voronoi4096_p3
    n = int(name[len("voronoi"):])
    return voronoi4096_p3(n_cells=n, n_parts=max(1, round(n / 64)))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--workload", default="hex24")
    ap.add_argument("--precision", choices=["fp64", "fp32", "bf16"], default="fp32")
    ap.add_argument("--policy", type=int, default=3, help="initial-guess policy (-1: x0 = U^k)")
    ap.add_argument("--ionic-form", choices=["nodal", "modal"], default="nodal")
    ap.add_argument("--steps", type=int, default=4)
    a = ap.parse_args(argv)
    import torch
    w = make_workload(a.workload)
    ctx = pd.setup_mesh(w.mesh, w.sigma, w.p, w.subdomain, w.chi_cm, w.dt, w.eta0)
    pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision=a.precision)
    sim = pd.sim_create(ctx, pc, u0=w.u_rest, stimulus=w.stimulus, rtol=w.rtol, maxit=20000,
                        flexible=a.precision != "fp64")
    if a.ionic_form != "nodal":
        pd.sim_set_ionic_form(sim, a.ionic_form)
    if a.policy >= 0:
        pd.sim_set_guess(sim, None, a.policy)
    stream = torch.cuda.current_stream()
    for k in range(a.steps):
        st = pd.monodomain_step(sim, 1, stream=stream)
        print(json.dumps({"step": k, "iterations": st["total_iterations"],
                          "relres": st["last_relres"], "pcg_ms": 1e3 * st["pcg_seconds"],
                          "status": st["status"]}), flush=True)
    sim.close()
    pc.close()
    ctx.close()


if __name__ == "__main__":
    main()
