"""The index-checked build (``build(checked=True)``, compiled with -DPA_CHECKED)
on the small parity cases: every window element, tap, combine slice and bulk
copy source is checked against its window and row, a failed check latches
PA_ERR_DEVICE_CHECK instead of touching memory out of range.  Here no check may
fire, and every result must equal the unchecked build's bit for bit (the
checks add branches, not arithmetic)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# Runs the cases with the library PA_LIB_PATH selects and saves every output.
RUN = r'''
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[2]); sys.path.insert(0, sys.argv[2] + "/tests")
from helpers import operator_cases
from paper_2404_10928_gb300 import phantoms as ph
from paper_2404_10928_gb300.api import Batch, Plan
out = {}
rng = np.random.default_rng(5)
for name, prob in sorted(operator_cases().items()):
    x = torch.tensor(rng.uniform(0, 1, prob.n_pixels), dtype=torch.float32, device="cuda")
    y = torch.tensor(rng.standard_normal((prob.n_sensors, prob.n_samples)), dtype=torch.float32,
                     device="cuda")
    with Plan.from_problem(prob) as plan:
        out[name + ":A"] = plan.forward(x).cpu().numpy()
        out[name + ":AT"] = plan.adjoint(y).cpu().numpy()
        out[name + ":cgls5"] = plan.reconstruct(plan.forward(x), "cgls", 5).cpu().numpy()
        out[name + ":ATframes"] = plan.adjoint_frames(torch.stack([y, 2 * y])).cpu().numpy()
        plan.sync_status()  # raises on a latched index check
frames = [ph.custom(2, (37, 53), (1e-4, 1e-4), ph.ring_sensors(13, 4e-3), 301, seed=3),
          ph.custom(2, (33, 33), (1e-4, 1e-4), ph.ring_sensors(7, 3e-3), 90, seed=4)]
plans = [Plan.from_problem(p, adj_cluster=1) for p in frames]
ys = [pl.forward(torch.tensor(p.x_true, dtype=torch.float32, device="cuda"))
      for pl, p in zip(plans, frames)]
xs = [torch.zeros(p.n_pixels, dtype=torch.float32, device="cuda") for p in frames]
with Batch(plans) as b:
    b.landweber(ys, xs, [1e-9, 1e-9], 3, history=True)
    for f, x in enumerate(xs):
        out[f"batch{f}"] = x.cpu().numpy()
for pl in plans:
    pl.sync_status()
    pl.close()
np.savez(sys.argv[1], **out)
'''


def _run(path, lib, env_lib):
    env = dict(os.environ)
    if env_lib:
        env["PA_LIB_PATH"] = lib
    else:
        env.pop("PA_LIB_PATH", None)
    res = subprocess.run([sys.executable, "-c", RUN, str(path), ROOT], env=env, cwd=ROOT,
                         capture_output=True, text=True, timeout=900)
    assert res.returncode == 0, res.stderr[-3000:]
    return np.load(path)


def test_checked_build_reports_nothing_and_matches(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_10928_gb300 import build
    plain_lib = build.build()
    checked_lib = build.build(checked=True)
    assert checked_lib != plain_lib
    plain = _run(tmp_path / "plain.npz", plain_lib, False)
    checked = _run(tmp_path / "checked.npz", checked_lib, True)
    assert sorted(plain.files) == sorted(checked.files)
    for k in plain.files:
        assert np.array_equal(plain[k], checked[k]), k
