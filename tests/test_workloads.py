"""CPU checks of the seeded input generators shared by the oracle, the tests and bench.py."""
import math

import workloads as W


def test_direction_cases_split_the_circle():
    cases = W.direction_cases(4)
    assert len(cases) == 4
    for k, c in enumerate(cases):
        d = c["traction_dir"]
        assert abs(math.hypot(d[0], d[1]) - 1.0) < 1e-15 and d[2] == 0.0
        assert abs(math.atan2(d[1], d[0]) % (2 * math.pi) - (k * math.pi / 2) % (2 * math.pi)) < 1e-12
        assert c["sigma_y"] == W.MATERIAL["sigma_y"] and c["hardening"] == W.MATERIAL["hardening"]


def test_seeded_cases_are_reproducible_and_in_range():
    a, b = W.irregular_cases(0, 16), W.irregular_cases(0, 16)
    assert a == b and len(a) == 16
    for c in a:
        assert 300.0 <= c["sigma_y"] <= 600.0 and 1e3 <= c["hardening"] <= 2e4
        assert abs(math.hypot(*c["traction_dir"][:2]) - 1.0) < 1e-12
    assert W.irregular_cases(1, 4) != a[:4]


def test_case_workload_changes_only_material_and_load():
    c = {"sigma_y": 333.0, "hardening": 4444.0, "traction_dir": (0.0, 1.0, 0.0)}
    w = W.case_workload(W.CUBE12, c)
    assert w.nel == W.CUBE12.nel and w.cuts == W.CUBE12.cuts and w.n_steps == W.CUBE12.n_steps
    assert w.material["sigma_y"] == 333.0 and w.material["hardening"] == 4444.0
    assert w.material["young"] == W.MATERIAL["young"] and w.material["poisson"] == W.MATERIAL["poisson"]
    assert w.traction_dir == (0.0, 1.0, 0.0)
    assert W.CUBE12.material["sigma_y"] == W.MATERIAL["sigma_y"]      # the base workload is untouched


def test_irregular_partition_segments():
    """Seeded cuts: every segment has 4..12 elements and the cuts cover the axis."""
    for seed in range(5):
        w = W.irregular_cube(80, seed)
        for cuts in w.cuts:
            assert cuts[0] == 0 and cuts[-1] == 80
            seg = [b - a for a, b in zip(cuts, cuts[1:])]
            assert all(4 <= s <= 12 for s in seg)
    assert W.CUBE80_IRREGULAR.n_sub == 810
