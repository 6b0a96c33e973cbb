"""The seeded input generators (no LBM arithmetic; they serve the oracle and
the CUDA path alike): determinism, the fractions they promise, and the
structure of their fields."""
import importlib.util
import os

import numpy as np
import pytest

from paper_1007_1388_gb300 import workloads as W


def test_random_flags_and_pdfs():
    rng = np.random.default_rng(5)
    fl = W.random_flags(rng, (20, 16, 12), 0.25, 0.3)
    assert fl.shape == (12, 16, 20) and set(np.unique(fl)) <= {0, 1, 2}
    assert abs((fl != 0).mean() - 0.25) < 0.03
    f = W.random_pdfs(np.random.default_rng(6), (20, 16, 12), 1e-2, fl)
    assert f.shape == (19, 12, 16, 20)
    assert np.all(f[:, fl != 0] == 0) and np.abs(f).max() <= 1e-2


@pytest.mark.parametrize("porosity", [0.75, 0.9])
def test_sphere_packing_reaches_its_porosity_deterministically(porosity):
    dims = (40, 32, 24)
    a = W.sphere_packing(np.random.default_rng(11), dims, porosity)
    b = W.sphere_packing(np.random.default_rng(11), dims, porosity)
    assert np.array_equal(a, b)
    fluid = (a == 0).mean()
    # stops at the first sphere that takes the solid fraction past 1 - porosity
    assert porosity - 4 / 3 * np.pi * 6**3 / np.prod(dims) <= fluid <= porosity + 1e-12
    assert set(np.unique(a)) <= {0, 1}


@pytest.mark.parametrize("porosity", [0.3, 0.5, 0.7])
def test_overlapping_spheres_reach_any_porosity(porosity):
    dims = (48, 40, 32)
    a = W.overlapping_spheres(np.random.default_rng(3), dims, porosity)
    assert np.array_equal(a, W.overlapping_spheres(np.random.default_rng(3), dims, porosity))
    fluid = (a == 0).mean()
    assert porosity - 0.02 <= fluid <= porosity
    # x and z are periodic: solid cells touch both ends of those axes
    assert (a[:, :, 0] != 0).any() and (a[:, :, -1] != 0).any()
    assert (a[0] != 0).any() and (a[-1] != 0).any()


def test_batch_instances_ranges_and_determinism():
    a = W.batch_instances(seed=7, n=6, lo=16, hi=24)
    b = W.batch_instances(seed=7, n=6, lo=16, hi=24)
    for (da, ta, fa), (db, tb, fb) in zip(a, b):
        assert da == db and ta == tb and np.array_equal(fa, fb)
        assert all(16 <= v <= 24 for v in da) and 0.55 <= ta <= 1.2
        assert fa.shape == da[::-1]


def test_bench_wall_links_cover_both_walls():
    """The curved-wall bench variant's links: every pull from the -y / +y wall
    of an n^3 channel, with the bottom and top distances."""
    pytest.importorskip("torch")
    spec = importlib.util.spec_from_file_location(
        "bench", os.path.join(os.path.dirname(os.path.dirname(__file__)), "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    import paper_1007_1388_gb300 as L

    n = 6
    cells, dirs, q = bench._wall_links(L, n, (0.3, 0.7))
    e = L.lbm_directions()[0]
    assert len(cells) == 10 * n * n
    y = (cells // n) % n
    for c, d, qq, yy in zip(cells, dirs, q, y):
        assert e[d][1] != 0
        assert (yy == 0 and e[d][1] == 1 and qq == 0.3) or (yy == n - 1 and e[d][1] == -1 and qq == 0.7)
    assert len(set(zip(cells.tolist(), dirs.tolist()))) == len(cells)
