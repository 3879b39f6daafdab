import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: oracle runs of several seconds or more")


_cache = {}


def cached(key, fn):
    if key not in _cache:
        _cache[key] = fn()
    return _cache[key]


@pytest.fixture(scope="session")
def square16():
    from synth import square16_p2
    from oracle import assembly
    def make():
        w = square16_p2()
        d = assembly.assemble(w.mesh, w.p, w.sigma, w.eta0, w.chi_cm, w.dt)
        return w, d
    return cached("square16", make)


@pytest.fixture(scope="session")
def voronoi256():
    """Small anisotropic Voronoi P3 case: several subdomains and a ragged partition."""
    from synth.meshes import voronoi_square, kmeans_partition, fibre_conductivity
    from synth import Workload, stimulus_params
    from oracle import assembly
    def make():
        m = voronoi_square(256, 7)
        part = kmeans_partition(m, 6, 7)
        w = Workload("voronoi256_p3", m, 3, 1, fibre_conductivity(m, 1.3, 0.2, 7), part,
                     part.copy(), eta0=10.0, dt=0.05, rtol=1e-8, n_steps=20,
                     stimulus=stimulus_params(7))
        d = assembly.assemble(m, w.p, w.sigma, w.eta0, w.chi_cm, w.dt)
        return w, d
    return cached("voronoi256", make)
