"""CPU checks of the CUDA library: it builds, loads without a GPU, exports every
declared entry point, and its host plan (index maps, B coefficients, fixing dofs)
is bit-exact with the oracle's independent construction."""
import os
import re

import numpy as np
import pytest

import workloads as W
import paper_1205_1926_gb300 as T
from oracle.ssn import ElastoplasticModel

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    lib = T.load()
    names = declared_functions()
    assert len(names) >= 25
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(T.SIGNATURES), set(names) ^ set(T.SIGNATURES)


@pytest.mark.parametrize("w", [W.TINY_1x1x2, W.SMALL4, W.SMALL6_RAGGED, W.CUBE12, W.CUBE24_IRREGULAR,
                               W.Workload(name="rollers", nel=(3, 2, 4), cuts=((0, 1, 3), (0, 2), (0, 2, 4)),
                                          dirichlet={"x0": 1, "y0": 2, "z0": 4, "x1": 6})])
def test_plan_maps_bit_exact_with_oracle(w):
    p = T.Plan(w)
    m = ElastoplasticModel(w)
    s = p.sizes()
    assert s["n_mult"] == m.dec.m and s["n_dof"] == m.dec.n_dof and s["n_gp"] == m.dec.n_gp
    assert s["n_sub"] == m.dec.n_sub and s["n_coarse"] == 6 * m.dec.n_sub
    rows, cols, vals = p.export_B()
    B = m.dec.B.tocoo()
    o = np.lexsort((B.col, B.row))
    np.testing.assert_array_equal(rows, B.row[o])
    np.testing.assert_array_equal(cols, B.col[o])
    np.testing.assert_array_equal(vals, B.data[o])          # Helmert coefficients bit-exact
    fx = p.export_fixing()
    subs = p.export_subdomains()
    for i, sd in enumerate(m.dec.subs):
        np.testing.assert_array_equal(fx[i], sd.fixing_dofs())
        assert tuple(subs[i][:3]) == sd.origin and tuple(subs[i][3:6]) == sd.dims
        assert subs[i][6] == m.dec.dof_off[i] and subs[i][7] == m.dec.elem_off[i]


def test_plan_sizes_of_the_timed_workload():
    """64^3 bricks in 8^3 boxes: decomposed dofs, multipliers and coarse size by direct count."""
    from tests.test_oracle_fem import brute_force_multiplier_count
    s = T.Plan(W.CUBE64).sizes()
    assert s["n_sub"] == 512 and s["n_dof"] == 512 * 3 * 9 ** 3 and s["n_coarse"] == 3072
    assert s["n_mult"] == brute_force_multiplier_count(W.CUBE64) == 308544
    assert s["max_band"] == 3 * (81 + 9 + 1) + 2 == 275


def test_plan_rejects_bad_input():
    lib = T.load()
    bad = W.SMALL4.with_(cuts=((0, 3, 2), (0, 2, 4), (0, 2, 4)))
    with pytest.raises(T.TfetiError):
        T.Plan(bad)
    with pytest.raises(T.TfetiError):
        T.Plan(W.SMALL4, material=dict(W.MATERIAL, poisson=0.5))
    assert lib.tfeti_status_str(6) == b"not converged"


def test_device_calls_fail_cleanly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(T.TfetiError):
        T.Context(W.TINY_1x1x2)


def test_case_entry_points_reject_bad_arguments():
    """The case calls check their arguments on the host before touching the device."""
    import ctypes as C
    lib = T.load()
    out = C.c_void_p()
    assert lib.tfeti_setup_case(None, 450.0, 1e4, None, C.byref(out)) == 1
    assert lib.tfeti_setup_case(None, 450.0, 1e4, None, None) == 1
    assert lib.ssn_time_step_cases(None, 1, None, 0, 1e-6, 1e-8, 30, 100, None) == 1
    hs = (C.c_void_p * 1)(None)
    ps = (C.c_void_p * 1)(None)
    assert lib.ssn_time_step_cases(C.cast(hs, C.c_void_p), 0, C.cast(ps, C.c_void_p), 0, 1e-6, 1e-8, 30, 100,
                                   None) == 1
    assert lib.ssn_time_step_cases(C.cast(hs, C.c_void_p), 1, C.cast(ps, C.c_void_p), 0, 1e-6, 1e-8, 30, 100,
                                   None) == 1


def test_plan_sizes_of_the_uneven_box_workload():
    """80^3 bricks in the seeded 9 x 10 x 9 partition: 810 boxes, multipliers by direct count, and the
    largest half bandwidth (a 12 x 12 box face: 3 (13 * 13 + 13 + 1) + 2)."""
    from tests.test_oracle_fem import brute_force_multiplier_count
    w = W.CUBE80_IRREGULAR
    s = T.Plan(w).sizes()
    assert s["n_sub"] == 810 == w.n_sub and s["n_coarse"] == 6 * 810
    assert s["n_mult"] == brute_force_multiplier_count(w)
    assert s["max_band"] == 3 * (13 * 13 + 13 + 1) + 2
