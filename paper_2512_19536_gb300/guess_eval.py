"""Evaluate the learned PCG initial guess on workloads it was not trained on.

    python -m paper_2512_19536_gb300.guess_eval [--weights guess_p3_voronoi4096.npz]
        [--seeds 8,9] [--hex 48] [--steps 200]

For each evaluation workload -- the 4096-cell Voronoi P3 recipe with the given seeds (the
training set is seeds 0-7) and the n^3 jittered hexahedral P2 mesh -- the coupled steps run
in the mixed form (fp32 local inverses, flexible PCG to 1e-8) with four initial guesses:
  * subspace:   Galerkin projection onto the network's proposal and the last 24 solution
                increments (policy 3 with the model);
  * increments: the same projection without the network (policy 3, no model);
  * proposal:   the network's proposal alone, kept when its residual is below U^k's
                (policy 0);
  * previous:   x0 = U^k.
One JSON line per workload and form: PCG iterations per step, steps whose solve started
from the learned guess, and time-steps/s (CUDA events around the stepping).
"""
from __future__ import annotations

import argparse
import json
import os

from . import _native as pd

HERE = os.path.dirname(os.path.abspath(__file__))


def run(w, model, policy, steps, stream):
    import torch
    ctx = pd.setup_mesh(w.mesh, w.sigma, w.p, w.subdomain, w.chi_cm, w.dt, w.eta0)
    pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision="fp32")
    sim = pd.sim_create(ctx, pc, u0=w.u_rest, stimulus=w.stimulus, rtol=1e-8, maxit=5000,
                        flexible=True)
    if policy is not None:
        pd.sim_set_guess(sim, model, policy)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    st = pd.monodomain_step(sim, steps, stream=stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    out = {"iterations_per_step": st["total_iterations"] / steps, "guess_taken_steps": st["guesses_taken"],
           "steps_per_s": steps / (ms * 1e-3), "status": st["status"]}
    sim.close()
    pc.close()
    ctx.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--weights", default=os.path.join(HERE, "guess_p3_voronoi4096.npz"))
    ap.add_argument("--seeds", default="8,9")
    ap.add_argument("--hex", type=int, default=48)
    ap.add_argument("--steps", type=int, default=200)
    a = ap.parse_args(argv)
    import numpy as np
    import torch
    from synth import voronoi4096_p3, hex_cube_p2
    z = np.load(a.weights)
    model = pd.guess_create(int(z["n_p"]), z["params"], z["scales"])
    stream = torch.cuda.current_stream()
    cases = [(f"voronoi4096_p3 seed {s}", voronoi4096_p3(seed=int(s)), a.steps) for s in a.seeds.split(",") if s]
    if a.hex > 0:
        w = hex_cube_p2(n=a.hex)
        cases.append((f"hex{a.hex}_p2", w, min(a.steps, w.n_steps)))
    forms = [("subspace", model, 3), ("increments", None, 3), ("proposal", model, 0), ("previous", None, None)]
    for name, w, steps in cases:
        for form, m, policy in forms:
            r = run(w, m, policy, steps, stream)
            print(json.dumps({"workload": name, "form": form, "steps": steps} | r), flush=True)
    return 0


if __name__ == "__main__":
    main()
