"""Named synthetic workloads: meshes, partitions, coefficients and parameters.

Each workload is plain data.  The two named ones mirror the paper's test
setting (a 2D unit square with polygonal elements, nested agglomerates as
subdomains and coarse cells) at the sizes the solver is measured on.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .meshes import (Mesh, cartesian_square, voronoi_square, block_partition,
                     kmeans_partition, fibre_conductivity, isotropic_conductivity,
                     jittered_hex_cube, block_partition_3d)


@dataclass
class Workload:
    name: str
    mesh: Mesh
    p: int                     # fine polynomial degree
    q: int                     # coarse polynomial degree
    sigma: np.ndarray          # [nc, dim, dim] per-cell conductivity
    subdomain: np.ndarray      # [nc] int32 subdomain id per cell
    coarse: np.ndarray         # [nc] int32 coarse agglomerate id per cell
    eta0: float = 10.0
    dt: float = 0.1
    chi_cm: float = 1.0
    rtol: float = 1e-8
    n_steps: int = 1
    u_rest: float = -67.0
    stimulus: dict = field(default_factory=dict)


def random_rhs(n: int, seed: int) -> np.ndarray:
    """Seeded standard-normal vector of length n (float64)."""
    return np.random.Generator(np.random.PCG64(seed)).standard_normal(n)


def stimulus_params(seed: int, amplitude: float = 250.0, width: float = 0.05,
                    duration: float = 1.0, dim: int = 2) -> dict:
    """Gaussian external current I = A exp(-|x-x0|^2 / (2 w^2)) while t < duration,
    centred at a seeded point of [0.25, 0.75]^dim."""
    x0 = 0.25 + 0.5 * np.random.Generator(np.random.PCG64(seed)).random(dim)
    out = {"x0": float(x0[0]), "y0": float(x0[1]), "amplitude": amplitude,
           "width": width, "duration": duration}
    if dim == 3:
        out["z0"] = float(x0[2])
    return out


def square16_p2() -> Workload:
    """16x16 unit-square Cartesian mesh, P2, sigma = 1, 4x4 subdomains of 4x4 cells,
    coarse P1 on the subdomains, one step dt = 0.1, eta0 = 10."""
    mesh = cartesian_square(16)
    part = block_partition(16, 4)
    return Workload("square16_p2", mesh, p=2, q=1,
                    sigma=isotropic_conductivity(mesh.n_cells, 1.0),
                    subdomain=part, coarse=part.copy(), eta0=10.0, dt=0.1,
                    rtol=1e-10)


def voronoi4096_p3(n_cells: int = 4096, seed: int = 2, n_parts: int = 64,
                   n_steps: int = 200) -> Workload:
    """Voronoi mesh of n_cells (5 Lloyd steps), P3, anisotropic fibre conductivity
    (sigma_l 1.3, sigma_t 0.2), k-means subdomains = coarse cells, dt = 0.05 ms."""
    mesh = voronoi_square(n_cells, seed, lloyd=5)
    part = kmeans_partition(mesh, n_parts, seed)
    return Workload(f"voronoi{n_cells}_p3", mesh, p=3, q=1,
                    sigma=fibre_conductivity(mesh, 1.3, 0.2, seed),
                    subdomain=part, coarse=part.copy(), eta0=10.0, dt=0.05,
                    rtol=1e-8, n_steps=n_steps, stimulus=stimulus_params(seed))


def voronoi_batch(n_meshes: int = 8, sims_per_mesh: int = 4, seed: int = 4,
                  cells: tuple = (1024, 16384), cells_per_subdomain: int = 64,
                  n_steps: int = 100, p: int = 3) -> list:
    """Independent simulations of uneven sizes: n_meshes Voronoi meshes (5 Lloyd
    steps) whose cell counts are log-uniform in [cells[0], cells[1]], each carrying
    sims_per_mesh simulations that differ in a scalar isotropic conductivity
    sigma ~ U[0.5, 2] and a stimulus site uniform in [0.1, 0.9]^2; k-means
    subdomains of about cells_per_subdomain cells = coarse cells; P3, dt = 0.05 ms.
    Returns a list of n_meshes * sims_per_mesh Workloads (the sims of one mesh
    share its Mesh and partition objects)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lo, hi = np.log(cells[0]), np.log(cells[1])
    counts = np.rint(np.exp(rng.uniform(lo, hi, n_meshes))).astype(int)
    out = []
    for m_id, nc in enumerate(counts):
        mseed = int(1000 * seed + m_id)
        mesh = voronoi_square(int(nc), mseed, lloyd=5)
        parts = max(1, int(round(nc / cells_per_subdomain)))
        part = kmeans_partition(mesh, parts, mseed)
        for s_id in range(sims_per_mesh):
            sig = float(rng.uniform(0.5, 2.0))
            x0 = 0.1 + 0.8 * rng.random(2)
            stim = {"x0": float(x0[0]), "y0": float(x0[1]), "amplitude": 250.0,
                    "width": 0.05, "duration": 1.0}
            out.append(Workload(f"batch{seed}_m{m_id}_s{s_id}", mesh, p=p, q=1,
                                sigma=isotropic_conductivity(mesh.n_cells, sig),
                                subdomain=part, coarse=part, eta0=10.0, dt=0.05,
                                rtol=1e-8, n_steps=n_steps, stimulus=stim))
    return out


def hex_cube_p2(n: int = 48, block: int = 4, seed: int = 3, n_steps: int = 50,
                p: int = 2) -> Workload:
    """n^3 jittered hexahedra on [0,1]^3 (10 % jitter, 12-facet polyhedra), P2
    (10 DOF per cell), isotropic sigma = 1, subdomains = coarse cells = blocks of
    block^3 cells, coarse P1, dt = 0.05 ms, n_steps coupled steps."""
    mesh = jittered_hex_cube(n, seed)
    part = block_partition_3d(n, block)
    return Workload(f"hex{n}_p{p}", mesh, p=p, q=1,
                    sigma=isotropic_conductivity(mesh.n_cells, 1.0, dim=3),
                    subdomain=part, coarse=part.copy(), eta0=10.0, dt=0.05,
                    rtol=1e-8, n_steps=n_steps, stimulus=stimulus_params(seed, dim=3))


def make_workload(name: str, **kw) -> Workload:
    if name == "square16_p2":
        return square16_p2()
    if name.startswith("voronoi"):
        return voronoi4096_p3(**kw)
    if name.startswith("hex"):
        return hex_cube_p2(**kw)
    raise KeyError(name)
