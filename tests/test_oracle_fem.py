"""Pins of the oracle's hex8 discretisation (Sec. 3.1, eqs. (F_def), (K_def)) and decomposition (Sec. 4.1-4.2)."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle.decomp import Decomposition, FixingNodeInverse, RegularisedInverse
from oracle.fem import Grid, element_strain_matrices, element_stiffness, gauss_weight_detj, NODE_OFFSETS
from oracle.material import Material
from oracle.ssn import ElastoplasticModel

MAT = Material.from_dict(W.MATERIAL)


def test_patch_test_linear_field_gives_exact_constant_strain():
    """An affine displacement field yields its exact (constant) strain at every Gauss point."""
    w = W.SMALL6_RAGGED
    m = ElastoplasticModel(w)
    rng = np.random.default_rng(0)
    A = rng.standard_normal((3, 3))
    b = rng.standard_normal(3)
    u = np.concatenate([(s.coords @ A.T + b).ravel() for s in m.dec.subs])
    eps = 0.5 * (A + A.T)
    exact = np.array([eps[0, 0], eps[1, 1], eps[2, 2], 2 * eps[0, 1], 2 * eps[1, 2], 2 * eps[0, 2]])
    np.testing.assert_allclose(m.strains(u), np.broadcast_to(exact, (m.dec.n_gp, 6)), atol=1e-12)


def test_element_stiffness_matches_exact_tensor_integration():
    """2x2x2 Gauss is exact for a brick's elastic stiffness.  Compare with the exact integral of the
    index form K_(a i),(b j) = int dN_a/dx_k C_ikjl dN_b/dx_l, C_ikjl = lam d_ik d_jl + mu (d_ij d_kl + d_il d_kj),
    evaluated with exact 1-D integrals of the separable trilinear shape functions."""
    from fractions import Fraction as Fr
    h = (Fr(3, 10), Fr(1, 2), Fr(7, 10))
    lam, mu = Fr(11074380, 100), Fr(8019380, 100)

    def one_d(s, t, ds, dt, hd):
        # int_0^h f_s^(ds) f_t^(dt), f_0 = 1 - x/h, f_1 = x/h
        if ds and dt:
            return (1 if s == t else -1) / hd
        if ds or dt:
            sgn = (1 if (s if ds else t) == 1 else -1)
            return Fr(sgn, 2)
        return hd / 3 if s == t else hd / 6

    def grad_integral(a, b, k, l):
        out = Fr(1)
        for d in range(3):
            out *= one_d(NODE_OFFSETS[a][d], NODE_OFFSETS[b][d], d == k, d == l, h[d])
        return out

    K_exact = np.zeros((24, 24))
    for a in range(8):
        for b in range(8):
            for i in range(3):
                for j in range(3):
                    v = lam * grad_integral(a, b, i, j) + mu * grad_integral(a, b, j, i)
                    if i == j:
                        v += mu * sum(grad_integral(a, b, k, k) for k in range(3))
                    K_exact[3 * a + i, 3 * b + j] = float(v)
    hf = tuple(float(v) for v in h)
    C = Material(206900.0, 0.29, 450.0, 1e4).C * 0
    C[:3, :3] = float(lam)
    for i in range(3):
        C[i, i] = float(lam + 2 * mu)
        C[3 + i, 3 + i] = float(mu)
    K = element_stiffness(element_strain_matrices(hf), np.broadcast_to(C, (1, 8, 6, 6)), gauss_weight_detj(hf))[0]
    np.testing.assert_allclose(K, K_exact, rtol=1e-12, atol=1e-11 * np.abs(K_exact).max())


def test_element_kernel_is_rigid_body_modes():
    h = (0.25, 0.25, 0.25)
    K = element_stiffness(element_strain_matrices(h), np.broadcast_to(MAT.C, (1, 8, 6, 6)), gauss_weight_detj(h))[0]
    ev = np.linalg.eigvalsh(K)
    assert np.sum(np.abs(ev) < 1e-9 * ev.max()) == 6 and ev.min() > -1e-9 * ev.max()


def test_traction_load_total_equals_traction_times_area():
    w = W.SMALL6_RAGGED
    m = ElastoplasticModel(w)
    t = np.array([0.3, -1.2, 2.0])
    f = m.dec.traction_load("z1", t)
    tot = f.reshape(-1, 3).sum(axis=0)
    np.testing.assert_allclose(tot, t * w.length[0] * w.length[1], rtol=1e-13)


def brute_force_multiplier_count(w):
    """Count B rows from the rule: Dirichlet component -> k rows, free component with k copies -> k-1 rows."""
    grid = Grid(w.nel, w.length)
    masks = w.dirichlet_masks()
    m = 0
    for k in range(grid.nnode_axis[2]):
        for j in range(grid.nnode_axis[1]):
            for i in range(grid.nnode_axis[0]):
                copies = 1
                for d, c in enumerate((i, j, k)):
                    if c in w.cuts[d][1:-1]:
                        copies *= 2
                mask = grid.node_dirichlet_mask(grid.node_id(i, j, k), masks)
                for comp in range(3):
                    m += copies if (mask >> comp) & 1 else copies - 1
    return m


@pytest.mark.parametrize("w", [W.TINY_1x1x2, W.SMALL4, W.SMALL6_RAGGED, W.CUBE12])
def test_constraint_matrix_orthonormal_full_rank(w):
    m = ElastoplasticModel(w)
    B = m.dec.B
    assert B.shape[0] == brute_force_multiplier_count(w)
    BBt = (B @ B.T).toarray()
    np.testing.assert_allclose(BBt, np.eye(B.shape[0]), atol=1e-14)      # orthonormal rows, Ker B^T = 0
    # a continuous field (all copies equal) with zero Dirichlet values satisfies B v = 0
    rng = np.random.default_rng(1)
    g = rng.standard_normal(3 * m.grid.n_nodes)
    nid = np.arange(m.grid.n_nodes)
    mask = m.grid.node_dirichlet_mask(nid, m.dec.masks)
    for c in range(3):
        g[c::3][(mask >> c) & 1 == 1] = 0.0
    v = np.concatenate([g[(3 * s.global_node[:, None] + np.arange(3)).ravel()] for s in m.dec.subs])
    assert np.abs(B @ v).max() < 1e-13 * np.abs(v).max()


def test_size_table_cube12():
    # sizes of the 12^3 / 2x2x2 workload by direct counting: decomposed dofs and multipliers
    m = ElastoplasticModel(W.CUBE12)
    assert m.dec.n_dof == 8 * 3 * 7 ** 3 and m.dec.B.shape[0] == 2148 and m.dec.n_gp == 13824


@pytest.mark.parametrize("w", [W.TINY_1x1x2, W.SMALL6_RAGGED])
def test_subdomain_kernel_and_generalised_inverse(w):
    m = ElastoplasticModel(w)
    Kb, _, _ = m.assemble(np.zeros(m.dec.n_dof), np.zeros(m.dec.n_dof))
    for p, s in enumerate(m.dec.subs):
        K = Kb[p].toarray()
        R = s.rigid_modes()
        np.testing.assert_allclose(R.T @ R, np.eye(6), atol=1e-13)
        assert np.abs(K @ R).max() <= 1e-12 * np.abs(K).max()
        ev = np.linalg.eigvalsh(K)
        assert np.sum(np.abs(ev) < 1e-10 * ev.max()) == 6
        kd = FixingNodeInverse(Kb[p], s.fixing_dofs())
        Kdag = np.stack([kd.apply(e) for e in np.eye(K.shape[0])], axis=1)
        np.testing.assert_allclose(K @ Kdag @ K, K, atol=1e-9 * np.abs(K).max())   # K K^+ K = K
        rg = RegularisedInverse(Kb[p], R)
        np.testing.assert_allclose(K @ rg.M @ K, K, atol=1e-9 * np.abs(K).max())
    # Ker K intersect Ker B = {0}: [K; B] has full column rank
    KB = np.vstack([sp.block_diag(Kb).toarray(), m.dec.B.toarray()])
    sv = np.linalg.svd(KB, compute_uv=False)
    assert sv.min() > 1e-8 * sv.max()
