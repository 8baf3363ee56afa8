"""Seeded input generators: determinism, shapes and value ranges."""
import numpy as np

from paper_2404_10928_gb300 import phantoms as ph


def test_linear_array_disks():
    a = ph.linear_array_disks()
    b = ph.linear_array_disks()
    assert a.x_true.shape == (64 * 64,)
    assert np.array_equal(a.x_true, b.x_true)
    nz = a.x_true[a.x_true > 0]
    assert nz.size > 0 and nz.min() >= 0.5 and nz.max() <= 1.0
    assert a.sensors.shape == (64, 2)
    # array 2 mm beyond the grid's outer edge (pixel boundary at 3.2 mm)
    assert np.allclose(a.sensors[:, 1], 5.2e-3)
    assert np.isclose(a.sensors[1, 0] - a.sensors[0, 0], 0.2e-3)


def test_ring_vessels():
    p = ph.ring_vessels()
    assert p.x_true.shape == (256 * 256,)
    assert p.noise_unit.shape == (256, 2048)
    assert np.allclose(np.hypot(p.sensors[:, 0], p.sensors[:, 1]), 20e-3)
    frac = np.mean(p.x_true > 0)
    assert 0.01 < frac < 0.5
    assert np.array_equal(p.x_true, ph.ring_vessels().x_true)


def test_vessel_tree_3d_small():
    p = ph.planar_vessel_tree(n=32)
    assert p.x_true.shape == (32 ** 3,)
    assert p.sensors.shape == (1024, 3)
    assert np.all(p.sensors[:, 2] > 0.5 * 32 * 2e-4)
    assert np.any(p.x_true > 0)


def test_add_noise_level():
    rng = np.random.default_rng(0)
    clean = rng.normal(size=(4, 100))
    unit = rng.standard_normal((4, 100))
    noisy = ph.add_noise(clean, unit, 0.01)
    assert np.allclose((noisy - clean) / unit, 0.01 * np.abs(clean).max())


def test_oracle_and_library_share_no_code():
    """The oracle imports nothing from the library and vice versa; both may take
    inputs from the phantoms module only."""
    import os
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for dirpath, _, files in os.walk(os.path.join(root, "oracle")):
        for f in files:
            if f.endswith((".py", ".c", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+paper_2404_10928_gb300", src, re.M), f
                assert "import_module" not in src, f
    pkg = os.path.join(root, "paper_2404_10928_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", src, re.M), f
                assert "pa_oracle" not in src and "liboracle" not in src, f
