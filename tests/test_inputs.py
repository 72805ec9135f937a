"""The seeded workloads have the shapes, sizes and value ranges their
recipes state (CPU only, no method arithmetic)."""
import numpy as np

import sfm_inputs as inputs


def test_config1_recipe():
    p = inputs.config1()
    assert (p.nx, p.ny, p.nz, p.nsub) == (48, 48, 48, 8)
    assert set(np.unique(p.c)) == {1500.0, 3000.0}
    assert np.all(p.c[:24] == 1500.0) and np.all(p.c[24:] == 3000.0)
    assert np.all(p.m_sub == 4) and np.all(p.k_sub == 8)
    assert p.nrec == 8 and p.nshots == 1 and p.nsteps == 500


def test_config3_cuts_and_depths():
    p = inputs.config3()
    for cuts, n in ((p.xcuts, p.nx), (p.ycuts, p.ny), (p.zcuts, p.nz)):
        assert cuts[0] == 0 and cuts[-1] == n
        assert set(np.diff(cuts)) <= {16, 20, 24, 32}
    assert p.nsub == 495
    assert set(np.unique(p.m_sub)) <= {4, 8}
    assert p.k_sub.min() >= 8 and p.k_sub.max() <= 24
    for s in range(p.nsub):
        x0, x1, y0, y1, z0, z1 = p.sub_box(s)
        if min(x1 - x0, y1 - y0, z1 - z0) <= 16:
            assert p.k_sub[s] <= 20
    assert p.nshots == 64 and p.nrec == 256
    assert p.c.min() >= 1500.0 and p.c.max() <= 4500.0


def test_surrogate_blocks_range():
    blocks = inputs.surrogate_blocks(4, n=12)
    assert blocks.shape == (4, 12, 12, 12)
    assert blocks.min() >= 1500.0 and blocks.max() <= 4500.0
    assert not np.allclose(blocks[0], blocks[1])


def test_paper_layout_recipe():
    """Section "Numerical experiments": 7 x 7 x 3 unit cubes, m = 25,
    n = 3, c independent of z with a slow fracture of contrast 10/3, source
    at (3.5, 1.5, 1.5), traces along (x, 0, 1.5)."""
    p = inputs.paper_layout(cells_per_unit=10)
    assert p.ncuts == (7, 7, 3) and p.nsub == 147
    assert p.h == 0.1 and (p.nx, p.ny, p.nz) == (70, 70, 30)
    assert np.all(p.m_sub == 25) and np.all(p.k_sub == 3)
    assert np.all(p.c == p.c[:1])                       # no z dependence
    assert abs(p.c.max() / p.c.min() - 10.0 / 3.0) < 1e-12
    frac = p.c[0] == p.c.min()
    assert 0.005 < frac.mean() < 0.1                    # thin
    np.testing.assert_allclose(p.src_xyz, [[3.5, 1.5, 1.5]])
    assert p.nrec == p.nx + 1
    assert np.all(p.rec_xyz[:, 1] == 0.0) and np.all(p.rec_xyz[:, 2] == 1.5)
    # shortest wavelength 0.78 at c = 1 at the Ricker band edge 2.5 f_peak
    assert abs(1.0 / (2.5 * p.f_peak) - 0.78) < 1e-12
    assert p.meta["t_end"] == 12.5


def test_workloads_are_seeded():
    a, b = inputs.paper_layout(cells_per_unit=6), inputs.paper_layout(cells_per_unit=6)
    assert np.array_equal(a.c, b.c)
    c = inputs.paper_layout(seed=7, cells_per_unit=6)
    assert not np.array_equal(a.c, c.c)
