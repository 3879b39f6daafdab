"""Run coupled time steps of a named synthetic workload through the C ABI and print one
JSON line per step (PCG iterations, relative residual, device time of the PCG launch).

A small driver for profilers and quick checks: it sets up the workload, the
preconditioner in the chosen precision (fp32/bf16 local inverses run flexible PCG) and
the initial-guess policy (--guess: with the trained network's proposal, as bench.py's
measured form), then steps one step per call, so the n-th launch of each kernel belongs
to step n.  Workloads: hex<N> (N^3 jittered hexahedra, P2, subdomains of 4^3
cells = coarse agglomerates, coarse P1), voronoi<N> (N-cell Voronoi mesh, P3, k-means
subdomains of ~64 cells = coarse agglomerates, coarse P1).

    python -m paper_2512_19536_gb300.run_steps --workload hex24 --precision fp32 --steps 4

With --shared-rhs R it instead applies the local solves shared by R simulations of the
workload's mesh (shared_local_apply; the mesh's conductivity made the scalar 1, R
conductivities spread over [0.5, 2]) --steps times for the BF16 eigenbasis (tensor cores)
and, in groups of four, for the FP32 one, and prints the device time per application
(CUDA events around each call's launches).
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
    ap.add_argument("--shared-rhs", type=int, default=0)
    ap.add_argument("--guess", action="store_true",
                    help="the trained network (guess_p3_voronoi4096.npz) as the learned proposal")
    a = ap.parse_args(argv)
    import torch
    w = make_workload(a.workload)
    if a.shared_rhs > 0:
        return shared(w, a.shared_rhs, a.steps)
    ctx = pd.setup_mesh(w.mesh, w.sigma, w.p, w.subdomain, w.chi_cm, w.dt, w.eta0)
    pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision=a.precision)
    sim = pd.sim_create(ctx, pc, u0=w.u_rest, stimulus=w.stimulus, rtol=w.rtol, maxit=20000,
                        flexible=a.precision != "fp64")
    if a.ionic_form != "nodal":
        pd.sim_set_ionic_form(sim, a.ionic_form)
    guess = None
    if a.guess:
        import os
        import numpy as np
        z = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "guess_p3_voronoi4096.npz"))
        guess = pd.guess_create(int(z["n_p"]), z["params"], z["scales"])
    if a.policy >= 0:
        pd.sim_set_guess(sim, guess, a.policy)
    stream = torch.cuda.current_stream()
    for k in range(a.steps):
        st = pd.monodomain_step(sim, 1, stream=stream)
        print(json.dumps({"step": k, "iterations": st["total_iterations"],
                          "relres": st["last_relres"], "pcg_ms": 1e3 * st["pcg_seconds"],
                          "status": st["status"]}), flush=True)
    sim.close()
    if guess is not None:
        guess.close()
    pc.close()
    ctx.close()


def shared(w, R, reps):
    import numpy as np
    import torch
    from synth.meshes import isotropic_conductivity
    sig = isotropic_conductivity(w.mesh.n_cells, 1.0, dim=getattr(w.mesh, "dim", 2))
    ctx = pd.setup_mesh(w.mesh, sig, w.p, w.subdomain, w.chi_cm, w.dt, w.eta0)
    n = ctx.n_dofs
    g = torch.Generator(device="cuda").manual_seed(0)
    rs = [torch.randn(n, dtype=torch.float64, device="cuda", generator=g) for _ in range(R)]
    zs = [torch.zeros(n, dtype=torch.float64, device="cuda") for _ in range(R)]
    sigmas = list(np.linspace(0.5, 2.0, R))
    stream = torch.cuda.current_stream()
    out = {"workload": w.name, "rhs": R}
    for prec in ("bf16", "fp32"):
        sl = pd.shared_local_setup(ctx, prec)
        group = R if prec == "bf16" else 4
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = 0.0
        for rep in range(reps):
            torch.cuda.synchronize()
            ev0.record(stream)
            for k0 in range(0, R, group):
                pd.shared_local_apply(sl, rs[k0:k0 + group], zs[k0:k0 + group], sigmas[k0:k0 + group],
                                      stream=stream)
            ev1.record(stream)
            torch.cuda.synchronize()
            if rep > 0:
                ms += ev0.elapsed_time(ev1)
        out[prec] = {"us_per_application": 1e3 * ms / max(1, reps - 1),
                     "store_bytes": sl.info()["store_bytes"]}
        sl.close()
    print(json.dumps(out), flush=True)
    ctx.close()
    return 0


if __name__ == "__main__":
    main()
