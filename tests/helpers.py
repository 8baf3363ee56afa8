"""Shared test helpers: seeded cases and comparison metrics."""
import numpy as np

from paper_2404_10928_gb300 import phantoms as ph

# Tolerances (relative L2 against the FP64 oracle) for the FP32 GPU path.
OP_TOL = 1e-5     # one application of A or A^T
RECON_TOL = 1e-4  # after a full reconstruction


def rel_l2(a, b) -> float:
    """||a - b|| / ||b|| (complex arrays compare as complex)."""
    cplx = np.iscomplexobj(a) or np.iscomplexobj(b)
    dt = np.complex128 if cplx else np.float64
    a = np.asarray(a, dtype=dt).ravel()
    b = np.asarray(b, dtype=dt).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def f32(a) -> np.ndarray:
    """Round to float32 and back: the exact values both sides consume."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def operator_cases():
    """Small seeded problems spanning tiles, ragged tails and the degenerate cases."""
    R = ph.ring_sensors
    cases = {
        "linear64-disks": ph.linear_array_disks(),
        "ragged-37x53-ring13-k301": ph.custom(2, (37, 53), (1e-4, 1e-4), R(13, 4e-3), 301, seed=3),
        "truncated-40x40-k90": ph.custom(2, (40, 40), (1e-4, 1e-4), R(16, 3e-3), 90, seed=4),
        "t0-amp-33x20": ph.custom(2, (33, 20), (1e-4, 1e-4), R(9, 3e-3), 200, seed=5,
                                  t0=3 / ph.SAMPLE_RATE, amp_scale=1 / (2 * np.pi * 1500.0)),
        "anisotropic-70x9": ph.custom(2, (70, 9), (0.7e-4, 1.3e-4), R(11, 4e-3), 260, seed=6),
        "single-pixel-k2": ph.custom(2, (1, 1), (1e-4, 1e-4), np.array([[0.0, 5.625e-5]]), 2,
                                     seed=7, density=1.0),
        "3d-20x17x12-planar": ph.custom(3, (20, 17, 12), (2e-4, 2e-4, 2e-4),
                                        ph.planar_array(6, 5, 0.8e-3, 3.5e-3), 200, seed=8),
        "3d-33x9x17-ragged": ph.custom(3, (33, 9, 17), (1.5e-4, 2e-4, 1e-4),
                                       ph.planar_array(4, 7, 0.6e-3, -3e-3), 151, seed=9),
    }
    # sensors inside the grid's bounding box, between pixel centres
    inside = ph.custom(2, (30, 30), (1e-4, 1e-4), np.zeros((1, 2)), 120, seed=10)
    xs, ys, _ = inside.pixel_axes()
    inside.sensors = np.array([[xs[3] + 5e-5, ys[7] + 5e-5], [xs[20] + 5e-5, ys[25] - 5e-5],
                               [xs[14] - 5e-5, ys[0] - 5e-5], [0.0, 4e-3]])
    cases["sensors-inside-grid"] = inside
    return cases


# ----------------------------------------------------------------------------
# CGLS past the semi-convergence knee.  These problems amplify FP32-level
# perturbations of the recursion by 1e4-1e6 after ~10 iterations (measured by
# tests/test_cgls_sensitivity.py with the FP64 oracle alone), so a full-length
# FP32 reconstruction is compared with the oracle through the spread of an
# ensemble of perturbed oracle runs, each within what the FP32 path is allowed:
# FP32 storage of every vector, and every operator output perturbed at the
# operator tolerance OP_TOL (two seeds).  The GPU result must lie within
# CGLS_ENVELOPE_FACTOR times the ensemble's largest departure.
# ----------------------------------------------------------------------------
CGLS_ENVELOPE_FACTOR = 2.0
CGLS_ENSEMBLE = (
    {"round_fp32": True},
    {"op_noise": OP_TOL, "noise_seed": 1},
    {"op_noise": OP_TOL, "noise_seed": 2, "round_fp32": True},
)


def cgls_with_iterates(orc, geo, y, n_iter, **kw):
    """Oracle CGLS without the final clamp; returns (iterates, history)."""
    its = []
    _, hist = orc.cgls(geo, y, n_iter, nonneg=False, iterates=its, **kw)
    return its, hist


def cgls_spread(orc, geo, y, n_iter, ref_iterates, ref_hist, members=CGLS_ENSEMBLE):
    """Largest departure of the ensemble from the exact oracle run, per
    iteration: (x relative L2 [n_iter], |history difference| / ||r_0||^2
    [n_iter+1], the final x departure of each member)."""
    dx = np.zeros(n_iter)
    dh = np.zeros(n_iter + 1)
    finals = []
    for kw in members:
        its, hist = cgls_with_iterates(orc, geo, y, n_iter, **kw)
        d = [rel_l2(a, b) for a, b in zip(its, ref_iterates)]
        finals.append(d[-1])
        dx = np.maximum(dx, d)
        dh = np.maximum(dh, np.abs(hist - ref_hist) / ref_hist[0])
    return dx, dh, finals
