"""The benchmark's algorithmic model (the work its roofline fractions divide
by), checked against closed forms and a Monte Carlo estimate rather than
against its own formulas. CPU only."""
import math
import sys
from pathlib import Path

import numpy as np

sys.path.insert(0, str(Path(__file__).resolve().parents[1]))

import bench  # noqa: E402
from paper_1507_06643_gb300 import inputs  # noqa: E402


def test_pairs_per_particle_is_the_cutoff_sphere_count():
    # at number density rho each particle has rho * (4/3) pi r_c^3 neighbours,
    # each pair shared by two particles
    w = inputs.large_n4m("mixed")
    total, intra = bench.pair_counts(w)
    assert abs(total / w.n_total - 2.0 * math.pi) < 1e-9     # rho = 3, r_c = 1
    assert 0.0 < intra < total


def test_intra_domain_fraction_matches_monte_carlo():
    """Pairs of a uniform fluid whose two particles share a brick: the model's
    product over axes of (1 - 3 r_c / (8 b)) against a direct estimate
    (a particle uniform in a brick, its partner uniform in the cutoff
    sphere around it)."""
    w = inputs.large_n4m("mixed")
    total, intra = bench.pair_counts(w)
    r = w.replicas[0]
    b = np.asarray(r.box) / np.asarray(r.bricks)
    rng = np.random.default_rng(5)
    n = 400_000
    x = rng.random((n, 3)) * b
    d = rng.standard_normal((n, 3))
    d *= (rng.random(n) ** (1.0 / 3.0) * w.r_cut / np.linalg.norm(d, axis=1))[:, None]
    y = x + d
    same = np.all((y >= 0.0) & (y < b), axis=1).mean()
    assert abs(intra / total - same) < 0.01, (intra / total, same)


def test_step_roofline_bound():
    """The whole-step bound: 68 B per particle against the HBM peak and
    (Gaussian 180 + force 20 + map or SER arithmetic 95) lane operations per
    unique pair against 152 x 128 lanes at the clock; the larger wins."""
    w = inputs.large_n4m("mixed")
    peaks = {"hbm_gbs": 6693.8, "sm_max_mhz": 2070.0}
    r = bench.step_roofline(w, "HYBRID", 2.44, peaks, "measured")
    pairs = 2.0 * math.pi
    assert abs(r["ops_per_particle"] - pairs * 295.0) < 1e-6
    t_alu = w.n_total * pairs * 295.0 / (152 * 128 * 2.07e9)
    t_hbm = w.n_total * 68.0 / 6693.8e9
    assert r["bound"] == "alu" and t_alu > t_hbm
    assert abs(r["model_us"] - 1e6 * t_alu) < 1e-6
    assert abs(r["frac"] - t_alu / 2.44e-3) < 1e-12
    # FP64 moves 116 B per particle; SER has no SSA map but both sweeps
    r64 = bench.step_roofline(inputs.large_n4m("fp64"), "SER", 28.6, peaks, "measured")
    assert r64["bytes_per_particle"] == 116.0
    assert abs(r64["ops_per_particle"] - pairs * (180.0 + 20.0 + 95.0)) < 1e-6


def test_phase_model_units():
    w = inputs.large_n4m("mixed")
    bound, work, unit = bench.algorithmic_model(w, "force", "HYBRID", "mixed", 2)
    assert (bound, unit) == ("hbm", "GB/s") and work == w.n_total * 64.0
    bound, work, unit = bench.algorithmic_model(w, "ssa", "HYBRID", "mixed", 2)
    _, intra = bench.pair_counts(w)
    assert (bound, unit) == ("alu", "Gop/s") and abs(work - intra * 275.0) < 1e-3
