"""Iteration counts and condition estimates of the massively parallel preconditioner.

The experiment of Sec. 5 (Table 1) on synthetic inputs: every subdomain is one fine
element (T_S = T_h), the coarse correction lives on agglomerates of size H = 2h, 4h,
8h, 16h, the coarse degree equals the fine one (p = q), and PCG runs to a relative
residual of 1e-9 inside coupled Crank-Nicolson steps of dt = 2.5 microseconds.  For
each (N_h, H) the sweep reports the average PCG iterations per step, the Lanczos
estimate of the condition number of the preconditioned operator (from the alpha_k,
beta_k of one traced solve), the device time per PCG iteration, and the same for
unpreconditioned CG.

Inputs (synthetic stand-ins for the paper's meshes, which are not available):
  * Voronoi meshes of N_h cells of the unit square (uniform seeds, 5 Lloyd steps);
  * grey matter (cell vertex-average y >= 0.5): isotropic sigma = 0.63; white matter
    (y < 0.5): sigma_l = 0.69 along the vertical direction, sigma_n = 2.571 across it
    (the values of Sec. 5, whose ordering contradicts sigma_l > sigma_n of Sec. 2;
    they are used as printed);
  * agglomerates: seeded k-means of the cell vertex-averages, run separately in the
    grey and the white region so that coarse cells align with the jump of sigma;
    N_h / (H/h)^2 agglomerates in all;
  * initial potential -67 mV, and -50 mV on the cells whose vertex-average lies in
    (x - 0.5)^2 + (y - 1)^2 < 0.016; no external stimulus;
  * the traced solve for the condition estimate: a seeded standard-normal right-hand
    side from x0 = 0.

chi_m C_m is not given in the paper.  The coupled sweep takes chi_m C_m = 1, which at
dt = 2.5 us leaves K mass-dominated; --chi-cm 0.01 --solve-only builds the same systems
with the stiffness weighted 100 times more (K = chi_cm M + dt/2 A) and reports the
traced solve alone (no coupled steps: the explicit ionic update is not meant for that
balance).

Run on a GPU: python -m paper_2512_19536_gb300.schwarz_sweep [--steps 20] [--chi-cm C]
[--solve-only] [--out f.json]
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import _native as pd


def grey_white_conductivity(pts: np.ndarray) -> np.ndarray:
    n = len(pts)
    sig = np.empty((n, 2, 2))
    grey = pts[:, 1] >= 0.5
    sig[grey] = 0.63 * np.eye(2)
    sl, sn = 0.69, 2.571
    white = np.diag([sn, sl])                 # sigma_n I + (sigma_l - sigma_n) e_y e_y^T
    sig[~grey] = white
    return sig


def aligned_agglomerates(pts: np.ndarray, n_agg: int, seed: int) -> np.ndarray:
    from synth.meshes import kmeans_points
    grey = pts[:, 1] >= 0.5
    out = np.empty(len(pts), dtype=np.int32)
    base = 0
    for region, share in ((grey, 0.5), (~grey, 0.5)):
        idx = np.flatnonzero(region)
        k = int(min(len(idx), max(1, round(n_agg * share))))
        lab = kmeans_points(pts[idx], k, seed)
        out[idx] = base + lab
        base += int(lab.max()) + 1
    return out


def initial_potential(pts: np.ndarray, n_p: int) -> np.ndarray:
    u = np.zeros((len(pts), n_p))
    inside = (pts[:, 0] - 0.5) ** 2 + (pts[:, 1] - 1.0) ** 2 < 0.016
    u[:, 0] = np.where(inside, -50.0, -67.0)  # the constant mode of the modal basis is 1
    return u.ravel()


def run_case(mesh, pts, sig, p, coarse, steps, dt, rtol, maxit, seed, chi_cm=1.0,
             solve_only=False):
    """One row entry: average iterations per coupled step (or of the traced solve when
    solve_only), the kappa estimate and the device time per PCG iteration."""
    import torch
    cells = np.arange(mesh.n_cells, dtype=np.int32)
    ctx = pd.polydg_setup(mesh.vertices, mesh.cell_ptr, mesh.cell_vtx, sig, p, cells,
                          chi_cm, dt, 10.0)
    pc = pd.asm_setup(ctx, coarse, q=p, precision="fp64") if coarse is not None else None
    n = ctx.n_dofs
    sim = None
    if not solve_only:
        sim = pd.sim_create(ctx, pc, u0=-67.0, rtol=rtol, maxit=maxit)
        u0 = torch.as_tensor(initial_potential(pts, n // mesh.n_cells), device="cuda")
        pd.sim_set_potential(sim, u0)
        st = pd.monodomain_step(sim, steps)
        if st["status"] != 0:
            raise RuntimeError(f"coupled steps failed: {st}")
    b = torch.as_tensor(np.random.Generator(np.random.PCG64(seed)).standard_normal(n), device="cuda")
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    tr, al, be = pd.pcg_solve_trace(ctx, pc, b, x, rtol=rtol, maxit=maxit)
    lo, hi = pd.lanczos_extremes(al, be)
    if solve_only:                        # time the same solve untraced, on the device
        x.zero_()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record()
        pd.pcg_solve(ctx, pc, b, x, rtol=rtol, maxit=maxit)
        ev1.record()
        torch.cuda.synchronize()
        its = tr["iterations"]
        us_it = 1e3 * ev0.elapsed_time(ev1) / max(its, 1)
    else:
        its = st["total_iterations"] / steps
        us_it = 1e6 * st["pcg_seconds"] / max(st["total_iterations"], 1)
    out = {"its_per_step": its, "kappa": hi / lo, "us_per_iteration": us_it,
           "traced_iterations": tr["iterations"], "n_dofs": n,
           "n_coarse": pc.info()["n_coarse"] if pc is not None else 0}
    if sim is not None:
        sim.close()
    if pc is not None:
        pc.close()
    ctx.close()
    return out


def sweep(n_cells=(512, 1024, 2048, 4096), degrees=(1, 4), ratios=(2, 4, 8, 16), steps=20,
          dt=2.5e-3, rtol=1e-9, maxit=200000, max_coarse=8000, seed=5, chi_cm=1.0,
          solve_only=False, log=sys.stderr):
    from synth.meshes import voronoi_square, cell_points
    from math import comb
    rows = []
    for p in degrees:
        n_p = comb(p + 2, 2)
        for nh in n_cells:
            mesh = voronoi_square(nh, seed + nh, lloyd=5)
            pts = cell_points(mesh)
            sig = grey_white_conductivity(pts)
            for ratio in list(ratios) + [None]:
                entry = {"p": p, "q": p, "n_h": nh, "H_over_h": ratio, "chi_cm": chi_cm,
                         "dt": dt, "mode": "solve" if solve_only else "coupled"}
                t0 = time.time()
                if ratio is None:
                    coarse = None
                else:
                    n_agg = max(2, int(round(nh / ratio ** 2)))
                    if n_agg * n_p > max_coarse:
                        entry["skipped"] = f"coarse space of {n_agg * n_p} DOFs > {max_coarse}"
                        rows.append(entry)
                        print(json.dumps(entry), file=log, flush=True)
                        continue
                    coarse = aligned_agglomerates(pts, n_agg, seed)
                try:
                    entry.update(run_case(mesh, pts, sig, p, coarse, steps, dt, rtol, maxit, seed,
                                          chi_cm, solve_only))
                except (pd.PolyDGError, RuntimeError) as err:
                    entry["failed"] = str(err)
                entry["seconds"] = time.time() - t0
                rows.append(entry)
                print(json.dumps(entry), file=log, flush=True)
    return rows


def markdown(rows, ratios=(2, 4, 8, 16)):
    """Table 1 layout: per degree, rows H (and CG), columns N_h; 'kappa (its)'."""
    out = []
    for p in sorted({r["p"] for r in rows}):
        sub = [r for r in rows if r["p"] == p]
        nhs = sorted({r["n_h"] for r in sub})
        out.append(f"p = q = {p}\n")
        out.append("| H \\ N_h | " + " | ".join(str(n) for n in nhs) + " |")
        out.append("|---|" + "---:|" * len(nhs))
        for ratio in list(ratios) + [None]:
            cells = []
            for nh in nhs:
                r = next((r for r in sub if r["n_h"] == nh and r["H_over_h"] == ratio), None)
                if r is None or "skipped" in r:
                    cells.append("—")
                elif "failed" in r:
                    cells.append("failed")
                else:
                    cells.append(f"{r['kappa']:.4g} ({r['its_per_step']:.1f})")
            out.append(f"| {'CG' if ratio is None else f'{ratio}h'} | " + " | ".join(cells) + " |")
        out.append("")
    return "\n".join(out)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--cells", type=int, nargs="+", default=[512, 1024, 2048, 4096])
    ap.add_argument("--degrees", type=int, nargs="+", default=[1, 4])
    ap.add_argument("--ratios", type=int, nargs="+", default=[2, 4, 8, 16],
                    help="H/h of the agglomerates (the CG row is always added)")
    ap.add_argument("--max-coarse", type=int, default=8000)
    ap.add_argument("--chi-cm", type=float, default=1.0,
                    help="chi_m C_m (not given in the paper; K = chi_cm M + dt/2 A)")
    ap.add_argument("--solve-only", action="store_true",
                    help="no coupled steps: iterations and time of the traced solve alone")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    rows = sweep(tuple(a.cells), tuple(a.degrees), tuple(a.ratios), steps=a.steps,
                 max_coarse=a.max_coarse, chi_cm=a.chi_cm, solve_only=a.solve_only)
    md = markdown(rows, tuple(a.ratios))
    print(md)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(rows, f, indent=1)


if __name__ == "__main__":
    main()
