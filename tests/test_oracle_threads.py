"""The oracle built with OpenMP (per-cell and per-face loops on all host
cores) gives bitwise the results of the single-threaded build: each loop
iteration writes only its own cell or face, and no floating-point value is
reduced across iterations.  The multi-threaded build is what the CPU
baseline times on all cores and what the full-size parity tests run."""
import numpy as np
import pytest

from oracle import Oracle, default_config, oracle_threads_available
from tests._cases import voronoi_case


def _run(mesh, cfg, st, threads, n_steps, mask=None):
    o = Oracle(default_config(**cfg), mesh, threads=threads)
    o.set_radiation(st["N"], st["fr"])
    o.set_gas(st["nH"], st["x5"], st["T"])
    o.set_sources(st["cells"], st["Q"])
    if mask is not None:
        o.set_active(mask)
    dt = o.max_dt()
    out = [o.gradients(), o.face_fluxes()]
    status = [o.step(3 * dt, 3) for _ in range(n_steps)]
    N, fr = o.radiation()
    x5, T = o.gas()
    return o, out + [N, fr, x5, T, o.substeps()], status


@pytest.mark.skipif(not oracle_threads_available(), reason="no OpenMP support in this compiler")
@pytest.mark.parametrize("variant", [dict(), dict(splitting=1, time_order=2), dict(chem_mode=1)])
def test_threads_bitwise_equal(variant):
    mesh, cfg, st = voronoi_case(n=10, **variant)
    o1, a, s1 = _run(mesh, cfg, st, 1, 2)
    o4, b, s4 = _run(mesh, cfg, st, 4, 2)
    assert o1.threads == 1 and o4.threads == 4
    assert s1 == s4
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.skipif(not oracle_threads_available(), reason="no OpenMP support in this compiler")
def test_threads_bitwise_equal_masked():
    mesh, cfg, st = voronoi_case(n=10)
    mask = np.random.default_rng(3).uniform(size=mesh.n_cells) < 0.4
    _, a, s1 = _run(mesh, cfg, st, 1, 1, mask)
    _, b, s4 = _run(mesh, cfg, st, 0, 1, mask)
    assert s1 == s4
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
