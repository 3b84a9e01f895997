"""Pins of the oracle's Algorithm 3 (TFETI + PCGP) against an undecomposed direct solve and its invariants."""
import numpy as np
import pytest

import workloads as W
from oracle.decomp import FixingNodeInverse, RegularisedInverse
from oracle.direct import solve_direct, scatter_to_decomposed
from oracle.ssn import ElastoplasticModel
from oracle.tfeti import TFETISolver


def elastic_system(w, seed=0):
    m = ElastoplasticModel(w)
    rng = np.random.default_rng(seed)
    f = m.traction_load((1.0, 0.3, -0.2)) + 0.01 * rng.standard_normal(m.dec.n_dof)
    Kb, f, _ = m.assemble(np.zeros(m.dec.n_dof), f)
    return m, Kb, f


@pytest.mark.parametrize("w", [W.TINY_1x1x2, W.SMALL4, W.SMALL6_RAGGED])
def test_tfeti_equals_undecomposed_direct_solve(w):
    m, Kb, f = elastic_system(w)
    sol = m.tfeti(Kb).solve(f, rtol=1e-14)
    u_ref = scatter_to_decomposed(m, solve_direct(m, f))
    assert np.linalg.norm(sol["u"] - u_ref) <= 1e-10 * np.linalg.norm(u_ref)
    assert sol["converged"]


def test_plastic_tangent_tfeti_equals_direct():
    """Same check on a tangent with plastic Gauss points (non-constant D)."""
    w = W.SMALL4
    m = ElastoplasticModel(w)
    rng = np.random.default_rng(7)
    m.sigma = rng.standard_normal((m.dec.n_gp, 6)) * 60.0
    du = scatter_to_decomposed(m, 4e-4 * rng.standard_normal(3 * m.grid.n_nodes))
    Kb, f, st = m.assemble(du, m.traction_load((0.5, 0.0, 1.0)))
    assert 0 < st["plastic"].sum() < m.dec.n_gp
    sol = m.tfeti(Kb).solve(f, rtol=1e-14)
    u_ref = scatter_to_decomposed(m, solve_direct(m, f, du=du))
    assert np.linalg.norm(sol["u"] - u_ref) <= 1e-10 * np.linalg.norm(u_ref)


def test_u_lambda_independent_of_generalised_inverse():
    m, Kb, f = elastic_system(W.SMALL6_RAGGED, seed=1)
    s1 = m.tfeti(Kb).solve(f, rtol=1e-14)
    kd = [RegularisedInverse(K, s.rigid_modes(), rho=3.7e4) for K, s in zip(Kb, m.dec.subs)]
    s2 = TFETISolver(m.dec, Kb, kd, R=m.R).solve(f, rtol=1e-14)
    assert np.linalg.norm(s1["u"] - s2["u"]) <= 1e-10 * np.linalg.norm(s1["u"])
    assert np.linalg.norm(s1["lam"] - s2["lam"]) <= 1e-10 * np.linalg.norm(s1["lam"])


def test_feasibility_at_every_iterate_and_saddle_point_residual():
    m, Kb, f = elastic_system(W.SMALL4, seed=2)
    solver = m.tfeti(Kb)
    e = -(solver.R.T @ f)
    scale = np.linalg.norm(e)
    errs = []
    sol = solver.solve(f, rtol=1e-12, check_feasibility=lambda lam: errs.append(np.linalg.norm(solver.N @ lam - e)))
    assert len(errs) == sol["iterations"] > 3
    assert max(errs) <= 1e-12 * scale                      # N lambda = e holds at every PCGP iterate
    u, lam = sol["u"], sol["lam"]
    res = solver.K @ u + m.dec.B.T @ lam - f                 # first row of eq. (equ:sps)
    assert np.linalg.norm(res) <= 1e-9 * np.linalg.norm(f)
    assert np.linalg.norm(m.dec.B @ u) <= 1e-10 * np.linalg.norm(u)


def test_preconditioner_does_not_change_solution_and_reduces_iterations():
    m, Kb, f = elastic_system(W.SMALL6_RAGGED, seed=3)
    s1 = m.tfeti(Kb).solve(f, rtol=1e-13)
    s2 = TFETISolver(m.dec, Kb, [FixingNodeInverse(K, s.fixing_dofs()) for K, s in zip(Kb, m.dec.subs)],
                     R=m.R, precond="none").solve(f, rtol=1e-13)
    assert np.linalg.norm(s1["u"] - s2["u"]) <= 1e-9 * np.linalg.norm(s1["u"])
    assert s1["iterations"] < s2["iterations"]


def test_zero_rhs_gives_zero_iterations():
    m, Kb, f = elastic_system(W.TINY_1x1x2)
    sol = m.tfeti(Kb).solve(np.zeros_like(f), rtol=1e-8)
    assert sol["iterations"] == 0 and np.all(sol["u"] == 0) and np.all(sol["lam"] == 0)


def test_pcgp_residual_history_decreases_overall():
    m, Kb, f = elastic_system(W.SMALL6_RAGGED, seed=4)
    hist = []
    m.tfeti(Kb).solve(f, rtol=1e-10, history=hist)
    assert hist[0] == pytest.approx(1.0, rel=1e-12) or hist[0] <= 1.0
    assert hist[-1] <= 1e-10 and len(hist) < 200
