"""Input generators: mesh invariants and a brute-force cross-check of the
Voronoi builder against Qhull (scipy.spatial) on a small periodic mesh."""
import numpy as np
import pytest

import synth


def _closure(mesh):
    an = np.stack([mesh.area * mesh.nx, mesh.area * mesh.ny, mesh.area * mesh.nz], 1)
    clo = np.zeros((mesh.n_cells, 3))
    np.add.at(clo, mesh.left, an)
    np.add.at(clo, mesh.right, -an)
    return clo


@pytest.mark.parametrize("n,jit", [(6, 0.3), (12, 0.3), (10, 0.1)])
def test_voronoi_invariants(n, jit):
    L = 3.0
    m = synth.voronoi_mesh(n, L, jit, seed=n)
    h = L / n
    assert m.n_cells == n ** 3
    assert abs(m.volume.sum() / L ** 3 - 1) < 1e-12
    assert np.all(m.volume > 0) and np.all(m.area > 0)
    np.testing.assert_allclose(np.sqrt(m.nx ** 2 + m.ny ** 2 + m.nz ** 2), 1, rtol=1e-14)
    # closed cells: sum_f A n = 0
    assert np.abs(_closure(m)).max() < 1e-12 * h * h
    # each cell pair at most once, no self faces, both ids in range
    assert np.all(m.left < m.right)
    pairs = m.left.astype(np.int64) * m.n_cells + m.right
    assert len(np.unique(pairs)) == m.n_faces
    # normal points from left generator to right generator (periodic image)
    g = m.gen
    d = g[m.right] - g[m.left]
    d -= L * np.round(d / L)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    np.testing.assert_allclose(np.stack([m.nx, m.ny, m.nz], 1), d, atol=1e-12)
    # face centroid lies on the bisector plane of the two generators
    fc = np.stack([m.fx, m.fy, m.fz], 1)
    mid = g[m.left] + 0.5 * (g[m.right] - g[m.left] - L * np.round((g[m.right] - g[m.left]) / L))
    off = fc - mid
    off -= L * np.round(off / L)
    assert np.abs((off * d).sum(1)).max() < 1e-10 * h
    assert 7.0 < m.faces_per_cell < 8.5


def test_voronoi_matches_qhull():
    """Volumes and neighbour pairs equal those of scipy's Qhull tessellation
    of the points plus their 26 periodic images."""
    spatial = pytest.importorskip("scipy.spatial")
    n, L = 6, 1.0
    m = synth.voronoi_mesh(n, L, 0.3, seed=4)
    pts = m.gen
    shifts = np.array([(i, j, k) for i in (-1, 0, 1) for j in (-1, 0, 1) for k in (-1, 0, 1)], float) * L
    allp = np.concatenate([pts + s for s in shifts])
    C = len(pts)
    base = 13 * C  # shift (0,0,0) is index 13
    vor = spatial.Voronoi(allp)
    vols = np.empty(C)
    for i in range(C):
        reg = vor.regions[vor.point_region[base + i]]
        assert -1 not in reg
        vols[i] = spatial.ConvexHull(vor.vertices[reg]).volume
    np.testing.assert_allclose(m.volume, vols, rtol=1e-9)
    # neighbour pairs with a face of non-negligible area
    qpairs = set()
    for (a, b), rv in zip(vor.ridge_points, vor.ridge_vertices):
        if a // C != 13 and b // C != 13:
            continue
        if -1 in rv:
            continue
        poly = vor.vertices[rv]
        c0 = poly.mean(0)
        area = 0.5 * np.linalg.norm(sum(np.cross(poly[k] - c0, poly[(k + 1) % len(poly)] - c0)
                                        for k in range(len(poly))))
        if area > 1e-8 * (L / n) ** 2:
            i, j = sorted((a % C, b % C))
            qpairs.add((i, j))
    ours = {(int(i), int(j)) for i, j in zip(m.left, m.right)
            if m.area[(m.left == i) & (m.right == j)][0] > 1e-8 * (L / n) ** 2}
    assert ours == qpairs


def test_bcc_mesh_invariants_and_qhull():
    """Staggered 2 x n^3 grid: the analytic truncated octahedra close (sum A n
    = 0), decompose into pyramids (sum_f A (x_f - s).n = 3V), fill the box,
    face centres are the generator midpoints on the bisector, and volumes,
    neighbour pairs and face areas equal Qhull's tessellation of the
    generators plus their 26 periodic images."""
    spatial = pytest.importorskip("scipy.spatial")
    n, L = 3, 1.5
    m = synth.bcc_mesh(n, L)
    C, h = m.n_cells, L / n
    assert C == 2 * n ** 3 and m.n_faces == 14 * n ** 3
    assert abs(m.volume.sum() / L ** 3 - 1) < 1e-14
    assert np.abs(_closure(m)).max() < 1e-14 * h * h
    g = m.gen
    d = g[m.right] - g[m.left]
    d -= L * np.round(d / L)
    dn = d / np.linalg.norm(d, axis=1, keepdims=True)
    np.testing.assert_allclose(np.stack([m.nx, m.ny, m.nz], 1), dn, atol=1e-14)
    fc = np.stack([m.fx, m.fy, m.fz], 1)
    off = fc - (g[m.left] + 0.5 * d)
    off -= L * np.round(off / L)
    assert np.abs(off).max() < 1e-14 * L
    pyr = np.zeros(C)
    for side, sg in ((m.left, 1.0), (m.right, -1.0)):
        x = fc - g[side]
        x -= L * np.round(x / L)
        np.add.at(pyr, side, sg * m.area * (x * np.stack([m.nx, m.ny, m.nz], 1)).sum(1))
    np.testing.assert_allclose(pyr / 3, m.volume, rtol=1e-13)
    # Qhull
    shifts = np.array([(i, j, k) for i in (-1, 0, 1) for j in (-1, 0, 1) for k in (-1, 0, 1)], float) * L
    allp = np.concatenate([g + s for s in shifts])
    vor = spatial.Voronoi(allp)
    base = 13 * C
    for i in range(C):
        reg = vor.regions[vor.point_region[base + i]]
        assert -1 not in reg
        assert abs(spatial.ConvexHull(vor.vertices[reg]).volume / m.volume[i] - 1) < 1e-9
    qarea = {}
    for (a, b), rv in zip(vor.ridge_points, vor.ridge_vertices):
        if (a // C != 13 and b // C != 13) or -1 in rv:
            continue
        poly = vor.vertices[rv]
        c0 = poly.mean(0)
        area = 0.5 * np.linalg.norm(sum(np.cross(poly[k] - c0, poly[(k + 1) % len(poly)] - c0)
                                        for k in range(len(poly))))
        if area > 1e-9 * h * h:
            qarea[tuple(sorted((a % C, b % C)))] = area
    ours = {tuple(sorted((int(i), int(j)))): a for i, j, a in zip(m.left, m.right, m.area)}
    assert set(ours) == set(qarea)
    for key, a in ours.items():
        assert abs(qarea[key] / a - 1) < 1e-9


def test_hii_region_setup():
    """The expanding-HII-region workload: density n0 in the core and
    n0 (r0/r)^2 outside, total source rate per bin as stated, mirror symmetry
    of the cell set about the box centre."""
    mesh, cfg, st = synth.hii_region(12)
    L = cfg["box"]
    c = mesh.centroids() - 0.5 * L
    c -= L * np.round(c / L)
    r = np.linalg.norm(c, axis=1)
    assert np.allclose(st["nH"][r < 0.0915], 3.2)
    far = r > 0.2
    np.testing.assert_allclose(st["nH"][far] * r[far] ** 2, 3.2 * 0.0915 ** 2, rtol=1e-12)
    np.testing.assert_allclose(st["Q"].sum(0), [1e50, 5e48, 3e48], rtol=1e-12)
    assert (r[st["cells"]] < 0.05).all() and (np.sort(r)[: len(st["cells"])] < 0.05).all()
    half = L / 12 / 2
    q = np.round(c / half).astype(np.int64) % 24
    key = {tuple(v) for v in q}
    assert all(tuple((-v) % 24) in key for v in q)


def test_cartesian_mesh():
    m = synth.cartesian_mesh(4, 2.0)
    assert m.n_cells == 64 and m.n_faces == 192
    assert abs(m.volume.sum() - 8.0) < 1e-14
    assert np.abs(_closure(m)).max() < 1e-15
    assert m.faces_per_cell == 3.0


def test_generators_seeded():
    a = synth.lognormal_density(100, 1e-3, 1.0, 5)
    b = synth.lognormal_density(100, 1e-3, 1.0, 5)
    np.testing.assert_array_equal(a, b)
    assert abs(np.median(synth.lognormal_density(100001, 1e-3, 1.0, 1)) / 1e-3 - 1) < 0.02
    pts = synth.jittered_lattice(8, 1.0, 0.3, 2)
    rho_pts, rho = synth.grf_density(pts, 1.0, 16, 1.5, 2e-4, 3)
    assert abs(rho.mean() / 2e-4 - 1) < 1e-12 and rho_pts.shape == (512,)
    peaks = synth.density_peaks(rho, 5)
    assert len(peaks) == 5
    vals = rho[tuple(peaks.T)]
    assert np.all(np.diff(vals) <= 0)
    m = synth.voronoi_mesh(8, 1.0, 0.3, seed=2)
    probe = m.gen + 0.01
    assert np.all(synth.locate_cells(m, probe) == np.arange(m.n_cells))


def test_density_recipes():
    """The synthetic densities as the input recipe states them: the GRF g
    has zero mean, unit variance and a measured power-spectrum slope of -2
    (shell-averaged |g_k|^2 fitted over 2 <= |k| <= 16 grid modes); exp(sigma
    g) then has log-standard deviation sigma and the requested grid mean, and
    the cells take the value of their nearest grid node; the i.i.d. lognormal
    field has the requested median and log-width; the source peaks are strict
    local maxima over the 26 periodic neighbours, highest first."""
    ng = 64
    g = synth.grf_field(ng, -2.0, 4)
    assert abs(g.mean()) < 1e-12 and abs(g.std() - 1) < 1e-12
    P = np.abs(np.fft.fftn(g)) ** 2
    k = np.fft.fftfreq(ng) * ng
    kk = np.sqrt(k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2)
    shells = np.arange(2, 17)
    Pk = np.array([P[(kk >= s - 0.5) & (kk < s + 0.5)].mean() for s in shells])
    slope = np.polyfit(np.log(shells), np.log(Pk), 1)[0]
    assert abs(slope + 2.0) < 0.1, slope
    pts = np.random.default_rng(1).uniform(0, 10.0, size=(500, 3))
    nH, rho = synth.grf_density(pts, 10.0, ng, 1.5, 2e-4, 4)
    assert rho.mean() == pytest.approx(2e-4, rel=1e-12)
    assert np.log(rho).std() == pytest.approx(1.5, rel=1e-12)
    ijk = np.floor(pts / 10.0 * ng).astype(int) % ng
    np.testing.assert_array_equal(nH, rho[ijk[:, 0], ijk[:, 1], ijk[:, 2]])
    ln = synth.lognormal_density(200000, 1e-3, 1.0, 2)
    assert np.median(ln) == pytest.approx(1e-3, rel=0.01)
    assert np.log(ln).std() == pytest.approx(1.0, rel=0.01)
    peaks = synth.density_peaks(rho, 50)
    vals = rho[peaks[:, 0], peaks[:, 1], peaks[:, 2]]
    assert np.all(np.diff(vals) <= 0)
    for p in peaks[:10]:
        for d in np.ndindex(3, 3, 3):
            off = np.array(d) - 1
            if off.any():
                q = (p + off) % ng
                assert rho[tuple(p)] > rho[tuple(q)]
