"""Train the learned PCG initial guess on trajectories of the plain solver.

    python -m paper_2512_19536_gb300.guess_train --out guess_p3.npz [--steps 2000]
        [--seeds 0,1,2,3,4,5,6,7] [--precision fp64] [--iters 8000] [--batch 4096] [--seed 0]

For each seed, a 4096-cell Voronoi P3 simulation (the 4096-cell workload's recipe with
that seed: mesh, fibre field, subdomains and stimulus site all change) is stepped by the
plain solver -- fp64 local inverses, standard PCG to 1e-8, x0 = U^k -- and its solutions
U^0..U^steps are kept on the device (2000 steps of 8 seeds: 5.2 GB).  Seeds 8 and 9 and
the 48^3 hexahedral mesh are left for evaluation (guess_eval.py).  The
network (include/polydg.h, guess_*) is then trained with Adam on minibatches of
(state k, cell) samples drawn uniformly over all trajectories, one trajectory per step
in turn; lr 1e-3, then 3e-4 for the last 30 % of the steps.  Scales: u_rest = -67,
s_u = 50, s_d = rms increment of the training trajectories, h_ref = their mean cell
diameter, dt_ref = 0.05.  Initial parameters: He-normal weights (seeded numpy), zero
biases, output layer scaled by 0.1.

Everything runs in the library's kernels; this script only draws the samples and moves
arrays.  Writes params (float64, the flat layout of guess_create) and scales to --out.
"""
import argparse
import os
import sys
import time

import numpy as np


def he_init(n_p, hidden, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    F = 9 * n_p + 3
    parts = []
    for shp, is_w in [((hidden, F), True), ((hidden,), False), ((hidden, hidden), True),
                      ((hidden,), False), ((n_p, hidden), True), ((n_p,), False)]:
        if is_w:
            a = rng.standard_normal(shp) * np.sqrt(2.0 / shp[1])
            if shp[0] == n_p:
                a *= 0.1
        else:
            a = np.zeros(shp)
        parts.append(a.reshape(-1))
    return np.concatenate(parts)


def cell_diameters(mesh):
    d = np.empty(mesh.n_cells)
    for c in range(mesh.n_cells):
        v = mesh.vertices[mesh.cell_vtx[mesh.cell_ptr[c]:mesh.cell_ptr[c + 1]]]
        d[c] = np.sqrt(((v[:, None] - v[None]) ** 2).sum(-1)).max()
    return d


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--out", required=True)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--seeds", default="0,1,2,3,4,5,6,7")
    ap.add_argument("--precision", choices=["fp64", "fp32"], default="fp64",
                    help="fp64: the plain solver (standard PCG); fp32: mixed (flexible PCG)")
    ap.add_argument("--iters", type=int, default=8000)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch
    import paper_2512_19536_gb300 as pd
    from synth import voronoi4096_p3

    t0 = time.time()
    runs, diam, incs = [], [], []
    for sd in [int(x) for x in args.seeds.split(",")]:
        w = voronoi4096_p3(seed=sd)
        ctx = pd.polydg_setup(w.mesh.vertices, w.mesh.cell_ptr, w.mesh.cell_vtx, w.sigma, w.p,
                              w.subdomain, w.chi_cm, w.dt, w.eta0)
        pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision=args.precision)
        sim = pd.sim_create(ctx, pc, u0=w.u_rest, stimulus=w.stimulus, rtol=1e-8, maxit=5000,
                            flexible=args.precision != "fp64")
        T = torch.empty((args.steps + 1, ctx.n_dofs), dtype=torch.float64, device="cuda")
        pd.sim_get_state(sim, T[0])
        for k in range(args.steps):
            pd.monodomain_step(sim, 1)
            pd.sim_get_state(sim, T[k + 1])
        sim.close()
        pc.close()
        runs.append((w, ctx, T))
        diam.append(cell_diameters(w.mesh))
        incs.append(float(torch.mean((T[1:] - T[:-1]) ** 2)))
        print(f"trajectory seed {sd}: {args.steps} steps ({time.time() - t0:.1f} s)", flush=True)
    n_p = runs[0][1].info.n_p
    scales = np.array([-67.0, 50.0, float(np.sqrt(np.mean(incs))), float(np.mean(np.concatenate(diam))),
                       0.05])
    model = pd.guess_create(n_p, he_init(n_p, 128, args.seed), scales)
    rng = np.random.Generator(np.random.PCG64(args.seed + 1))
    t1 = time.time()
    for it in range(args.iters):
        w, ctx, T = runs[it % len(runs)]
        smp = np.stack([rng.integers(2, args.steps - 1, args.batch),
                        rng.integers(0, w.mesh.n_cells, args.batch)], axis=1)
        lr = 1e-3 if it < 0.7 * args.iters else 3e-4
        loss = pd.guess_train_step(model, ctx, T, smp, lr)
        if it % 500 == 0 or it == args.iters - 1:
            print(f"step {it}: loss {loss:.4f} ({time.time() - t1:.1f} s)", flush=True)
    params = model.params()[0]
    np.savez(args.out, params=params, scales=scales, n_p=n_p)
    print(f"wrote {args.out}: {params.size} parameters, scales {scales.tolist()}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
