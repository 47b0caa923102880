"""The synthetic workload recipes against the settings the paper states
(Sec. 3.2, Sec. 3.3) and the stated manifests of the batch and serving
mixes.  No GPU, no oracle."""
import math

import numpy as np

from paper_2602_11734_gb300 import workloads as W


def test_fontainebleau_seed_probability_is_one_seed_per_grain():
    # S_d = 6 phi_s Delta^3 / (pi d^3) (Sec. 3.3) places, on average, one seed
    # per grain: expected seeds x the volume of a sphere of radius d / 2 (in
    # voxels of edge Delta) equals the solid volume.
    for phi_s, d in ((0.85, 225.0), (0.85, 200.0), (0.70, 250.0)):
        sd = W.fontainebleau_seed_probability(phi_s, d)
        grain_voxels = (4.0 / 3.0) * math.pi * (d / 2.0) ** 3 / W.FONTAINEBLEAU_VOXEL_UM ** 3
        assert math.isclose(sd * grain_voxels, phi_s, rel_tol=1e-12)
    # a larger grain means fewer seeds, as the cube of the diameter
    assert math.isclose(W.fontainebleau_seed_probability(0.85, 200.0) /
                        W.fontainebleau_seed_probability(0.85, 250.0), 1.25 ** 3, rel_tol=1e-12)


def test_fontainebleau_sweep_setting():
    # 500^3, porosity 0.15, one reference probability 8e-4, s = 0 .. 40 in
    # steps of 5, five realizations each (Sec. 3.3): 45 distinct seeds.
    assert W.FONTAINEBLEAU_SPACINGS == (0, 5, 10, 15, 20, 25, 30, 35, 40)
    runs = [W.fontainebleau(s, r) for s in W.FONTAINEBLEAU_SPACINGS for r in range(5)]
    assert len({p["seed"] for p in runs}) == 45
    for p in runs:
        assert (p["nx"], p["ny"], p["nz"]) == (500, 500, 500)
        assert math.isclose(p["target_solid_fraction"], 0.85, abs_tol=1e-12)
        assert p["g_face"] == p["g_edge"] == p["g_corner"] == 8e-4
        assert 0.0 < p["cd"] < 1e-4


def test_fig3_setting():
    # Sec. 3.2: seed probability 2e-4, reference probability 8e-4, porosity
    # 0.2, diamond spacing s = 15 (and none for Fig. 3b), 200^3 .. 1000^3.
    assert W.FIG3_EDGES == tuple(range(200, 1001, 100))
    for s_on in (True, False):
        p = W.fig3_size(400, s_on)
        assert p["cd"] == 2e-4 and p["g_face"] == p["g_edge"] == p["g_corner"] == 8e-4
        assert math.isclose(p["target_solid_fraction"], 0.80)
        assert p["spacing_s"] == (15 if s_on else 0)


def test_sweep_500_grid_and_seeds():
    runs = W.sweep_500()
    assert len(runs) == 25
    assert [p["seed"] for p in runs] == list(range(25))
    pts = {(round(1.0 - p["target_solid_fraction"], 6), p["spacing_s"]) for p in runs}
    assert pts == {(por, s) for por in W.SWEEP_POROSITY for s in W.SWEEP_SPACING}
    assert all(p["cd"] == 1e-4 and p["nx"] == 500 for p in runs)


def test_batch_96_manifest():
    runs = W.batch_96()
    assert len(runs) == 96 and [p["seed"] for p in runs] == list(range(96))
    assert {p["nx"] for p in runs} <= {128, 160, 192, 256}
    por = np.array([1.0 - p["target_solid_fraction"] for p in runs])
    assert por.min() >= 0.10 and por.max() <= 0.30
    assert all(10 <= p["spacing_s"] <= 40 and p["cd"] == 2e-4 for p in runs)
    assert runs == W.batch_96()  # seeded: the same manifest every time


def test_serve_mix_follows_its_weights():
    runs = W.serve_requests()
    assert len(runs) == 2000 and runs == W.serve_requests()
    edges = np.array([p["nx"] for p in runs])
    for e, w in zip(W.SERVE_EDGES, W.SERVE_WEIGHTS):
        share = float((edges == e).mean())
        assert abs(share - w) < 4.0 * math.sqrt(w * (1.0 - w) / len(runs)) + 1e-9, (e, share, w)
    assert all(0 <= p["spacing_s"] <= 40 and p["cd"] == 1e-4 for p in runs)
