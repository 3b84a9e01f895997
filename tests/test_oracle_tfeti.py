"""Pins of the oracle's Algorithm 3 (TFETI + PCGP) against an undecomposed direct solve and its invariants."""
import numpy as np
import pytest

import workloads as W
from oracle.decomp import FixingNodeInverse, RegularisedInverse
from oracle.direct import solve_direct, scatter_to_decomposed
from oracle.ssn import ElastoplasticModel
from oracle.tfeti import TFETISolver, dirichlet_schur_blocks


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


# ---------------------------------------------------------------------------- Dirichlet preconditioner
# 2x2x2 bricks in boxes of one brick, fixed on z = 0 and z = 1: every node carries a gluing or a
# Dirichlet row.
ONE_ELEMENT_BOXES = W.Workload(name="boxes_of_one", nel=(2, 2, 2), cuts=((0, 1, 2), (0, 1, 2), (0, 1, 2)),
                               dirichlet={"z0": 7, "z1": 7}, traction_face="x1")


def dirichlet_solver(m, Kb):
    return TFETISolver(m.dec, Kb, [FixingNodeInverse(K, s.fixing_dofs()) for K, s in zip(Kb, m.dec.subs)],
                       R=m.R, precond="dirichlet")


def test_dirichlet_equals_lumped_without_interior_nodes():
    """Boxes of one brick: every node carries a gluing or Dirichlet row, nothing is eliminated, so
    Sbar = K and the two preconditioners of Sec. 4.2 coincide."""
    m, Kb, f = elastic_system(ONE_ELEMENT_BOXES, seed=4)
    w = np.random.default_rng(5).standard_normal(m.dec.B.shape[0])
    lump = m.tfeti(Kb).apply_precond(w)
    dirich = dirichlet_solver(m, Kb).apply_precond(w)
    assert np.linalg.norm(dirich - lump) <= 1e-13 * np.linalg.norm(lump)


@pytest.mark.parametrize("w", [W.SMALL6_RAGGED, W.CUBE12])
def test_dirichlet_schur_blocks_kernel_and_order(w):
    """Sbar_p annihilates the rigid-body modes restricted to the constrained nodes (K R = 0 carries
    over to the Schur complement) and lies below K_bb in the Loewner order; floating subdomains have
    exactly six zero eigenvalues."""
    m, Kb, f = elastic_system(w, seed=6)
    blocks = dirichlet_schur_blocks(m.dec, m.dec.B, Kb)
    for p, (idx, S) in enumerate(blocks):
        Rb = m.dec.subs[p].rigid_modes()[idx - m.dec.dof_off[p]]
        assert np.abs(S @ Rb).max() <= 1e-9 * np.abs(S).max()
        loc = idx - m.dec.dof_off[p]
        Kbb = Kb[p].toarray()[np.ix_(loc, loc)]
        ev = np.linalg.eigvalsh(Kbb - S)
        assert ev.min() >= -1e-9 * np.abs(Kbb).max()
        es = np.linalg.eigvalsh(S)
        assert np.sum(es < 1e-9 * es.max()) == 6


def test_dirichlet_pcgp_solution_and_fewer_iterations():
    """Same solution as the undecomposed direct solve, in fewer PCGP iterations than the lumped
    preconditioner (Table 1: the Dirichlet preconditioner needs fewer iterations)."""
    m, Kb, f = elastic_system(W.CUBE12, seed=7)
    sd = dirichlet_solver(m, Kb).solve(f, rtol=1e-12)
    sl = m.tfeti(Kb).solve(f, rtol=1e-12)
    u_ref = scatter_to_decomposed(m, solve_direct(m, f))
    assert np.linalg.norm(sd["u"] - u_ref) <= 1e-9 * np.linalg.norm(u_ref)
    assert sd["converged"] and sd["iterations"] < sl["iterations"]
