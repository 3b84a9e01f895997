"""Pins of the oracle's semismooth Newton (Algorithms 2, 4, 5) against closed forms and the paper's tables."""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle.direct import solve_direct, scatter_to_decomposed
from oracle.ssn import ElastoplasticModel, run_load_history

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))

# Uniaxial bar: rollers on x=0 (u_x), y=0 (u_y), z=0 (u_z); traction along x on x=1.
UNIAXIAL = W.Workload(name="uniaxial", nel=(2, 2, 2), cuts=((0, 1, 2), (0, 2), (0, 1, 2)),
                      dirichlet={"x0": 1, "y0": 2, "z0": 4}, traction_face="x1", traction_dir=(1.0, 0.0, 0.0))


@pytest.mark.parametrize("n_steps", [1, 4])
def test_uniaxial_stress_closed_form(n_steps):
    """Homogeneous uniaxial stress with linear hardening: e11 = s/E + (s - sy)/H, e22 = -nu s/E - (s - sy)/(2H)."""
    m = ElastoplasticModel(UNIAXIAL)
    E, nu, sy, H = (W.MATERIAL[k] for k in ("young", "poisson", "sigma_y", "hardening"))
    f1 = m.traction_load((1.0, 0.0, 0.0))
    s_final = 1.8 * sy
    prev = 0.0
    for k in range(1, n_steps + 1):
        s = s_final * k / n_steps
        info = m.time_step((s - prev) * f1, newton_tol=1e-12, pcg_rtol=1e-14)
        prev = s
        assert info["converged"]
        e11 = s / E + max(s - sy, 0.0) / H
        e22 = -nu * s / E - max(s - sy, 0.0) / (2 * H)
        for sub in m.dec.subs:
            ul = m.u[m.dec.dof_off[sub.p]:m.dec.dof_off[sub.p + 1]].reshape(-1, 3)
            np.testing.assert_allclose(ul[:, 0], e11 * sub.coords[:, 0], rtol=1e-9, atol=1e-12 * abs(e11))
            np.testing.assert_allclose(ul[:, 1], e22 * sub.coords[:, 1], rtol=1e-9, atol=1e-12 * abs(e11))
            np.testing.assert_allclose(ul[:, 2], e22 * sub.coords[:, 2], rtol=1e-9, atol=1e-12 * abs(e11))
        np.testing.assert_allclose(m.sigma[:, 0], s, rtol=1e-9)
        np.testing.assert_allclose(m.sigma[:, 1:], 0.0, atol=1e-8 * s)
        np.testing.assert_allclose(m.kappa, max(s - sy, 0.0) / H, rtol=1e-9, atol=1e-15)


def test_uniaxial_cyclic_closed_form():
    """Load, unload, reverse (the cyclic schedule's phases) on the uniaxial bar.  With isotropic hardening
    the yield radius after loading is sigma_y + H kappa, so unloading stays elastic until the stress
    reaches minus that radius; beyond it the reverse flow raises kappa by the excess over H and lowers the
    plastic strain by the same amount: e11 = s/E + ep, e22 = -nu s/E - ep/2."""
    m = ElastoplasticModel(UNIAXIAL)
    E, nu, sy, H = (W.MATERIAL[k] for k in ("young", "poisson", "sigma_y", "hardening"))
    f1 = m.traction_load((1.0, 0.0, 0.0))
    ep = kappa = prev = 0.0
    for level in (0.9, 1.8, 0.6, -0.6, -1.5, -2.0, -1.0, 0.0):
        s = level * sy
        info = m.time_step((s - prev) * f1, newton_tol=1e-12, pcg_rtol=1e-14)
        prev = s
        assert info["converged"]
        radius = sy + H * kappa
        if abs(s) > radius:
            dk = (abs(s) - radius) / H
            kappa += dk
            ep += np.sign(s) * dk
        e11 = s / E + ep
        e22 = -nu * s / E - ep / 2
        scale = abs(e11) + abs(ep) + 1e-30
        for sub in m.dec.subs:
            ul = m.u[m.dec.dof_off[sub.p]:m.dec.dof_off[sub.p + 1]].reshape(-1, 3)
            np.testing.assert_allclose(ul[:, 0], e11 * sub.coords[:, 0], rtol=1e-9, atol=1e-10 * scale)
            np.testing.assert_allclose(ul[:, 1], e22 * sub.coords[:, 1], rtol=1e-9, atol=1e-10 * scale)
        np.testing.assert_allclose(m.sigma[:, 0], s, rtol=1e-9, atol=1e-9 * sy)
        np.testing.assert_allclose(m.kappa, kappa, rtol=1e-9, atol=1e-15)


def test_elastic_step_two_newton_iterations_and_criterion_one():
    w = W.SMALL6_RAGGED
    m = ElastoplasticModel(w)
    t_y = m.first_yield_traction()
    f1 = m.traction_load(w.traction_dir)
    df = 0.9 * t_y * f1
    info = m.time_step(df, newton_tol=1e-10, pcg_rtol=1e-14)
    assert info["criterion"][0] == GOLDEN["newton_first_criterion"]["value"]
    assert info["newton"] == GOLDEN["elastic_step_newton_iterations"]["value"]
    assert info["plastic"][0] == 0 and info["plastic_committed"] == 0
    u_ref = scatter_to_decomposed(ElastoplasticModel(w), solve_direct(ElastoplasticModel(w), df))
    assert np.linalg.norm(m.u - u_ref) <= 1e-10 * np.linalg.norm(u_ref)
    # yield is reached exactly at t_y: the peak von Mises stress equals 0.9 sigma_y
    assert m.von_mises().max() == pytest.approx(0.9 * W.MATERIAL["sigma_y"], rel=1e-9)


def test_plastic_step_local_quadratic_convergence():
    w = W.CUBE12
    m = ElastoplasticModel(w)
    t_y = m.first_yield_traction()
    f1 = m.traction_load(w.traction_dir)
    info = m.time_step(1.5 * t_y * f1, newton_tol=1e-11, pcg_rtol=1e-14)
    crit = info["criterion"]
    assert info["converged"] and crit[0] == 1.0 and info["plastic_committed"] > 0
    tail = [(a, b) for a, b in zip(crit[1:], crit[2:]) if a < 5e-2 and b > 1e-12]
    assert tail, crit
    for a, b in tail:
        assert b <= 1e3 * a * a, crit


@pytest.mark.slow
def test_rate_independence_of_plastic_set():
    """Monotone loading: one step and ten steps end with nearly the same plastic set (Sec. 5)."""
    w = W.CUBE12.with_(newton_tol=1e-8, pcg_rtol=1e-11)
    m1, _, t_y = run_load_history(w.with_(n_steps=1))
    m10, _, _ = run_load_history(w, t_y=t_y)
    p1 = int((m1.kappa > 0).sum())
    p10 = int((m10.kappa > 0).sum())
    assert p10 > 0
    assert abs(p1 - p10) / p10 <= 4 * GOLDEN["rate_independence_plastic_rel_diff"]["value"]
