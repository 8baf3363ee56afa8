"""Autotuner host logic (no GPU): size classes, candidate sets, selection and cache."""
import json

from paper_2404_10928_gb300 import autotune, phantoms as ph


def test_size_key_buckets():
    k = autotune.size_key("GB300", 2, 65536, 256, 2048)
    assert k == "GB300|2d|N65536|S256|K2048|yf32"
    assert autotune.size_key("GB300", 2, 65537, 200, 1500, "f16") == \
        "GB300|2d|N131072|S256|K2048|yf16"


def test_candidates_respect_sensor_count():
    c = list(autotune.candidates(6))
    assert all(cl in (1, 2) for cl, _, _, _ in c)  # 4 and 8 need at least 8 and 16 sensors
    n_fwd = len(autotune.FWD_SENSORS) * len(autotune.FWD_THREADS)
    n_adj = len(autotune.ADJ_CLUSTERS) * len(autotune.ADJ_WARPS) - 1
    big = list(autotune.candidates(512))
    assert len(big) == n_fwd + n_adj and len(set(big)) == len(big)
    assert all(nt in (64, 128, 256) and aw in (4, 8) for _, _, nt, aw in big)


def test_selection_and_cache(tmp_path):
    prob = ph.custom(2, (40, 30), (1e-4, 1e-4), ph.ring_sensors(64, 5e-3), 300, seed=1)
    calls = []

    def fake(prob_, c, spc, nt, aw):
        calls.append((c, spc, nt, aw))
        return (1.0 + 0.1 * abs(c - 4) + 0.01 * abs(spc - 16) + 0.001 * abs(nt - 256)
                + 0.0001 * abs(aw - 4))

    path = tmp_path / "tune.json"
    t = autotune.Autotuner(str(path), measure=fake, gpu_name="GB300")
    best = t.best(prob)
    assert autotune.Autotuner.plan_options(best) == {"adj_cluster": 4, "fwd_sensors_per_cta": 16,
                                                     "fwd_threads": 256, "adj_warps": 4}
    assert len(calls) == len(list(autotune.candidates(prob.n_sensors)))
    # the adjoint is timed with the forward at its defaults, the forward with
    # the adjoint at its defaults
    assert {(s, n) for c, s, n, aw in calls if (c, aw) != (1, 8)} == {(32, 128)}
    assert {(c, aw) for c, s, n, aw in calls if (s, n) != (32, 128)} == {(1, 8)}
    # cached: a second tuner reads the file and does not measure again
    t2 = autotune.Autotuner(str(path), measure=lambda *a: 1 / 0, gpu_name="GB300")
    assert t2.best(prob)["fwd_threads"] == 256
    assert t2.best(prob)["adj_cluster"] == 4
    data = json.loads(path.read_text())
    assert list(data) == [t.key(prob)]
