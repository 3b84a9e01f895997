"""Pins of the oracle's material point (Sec. 2.2-2.4, Sec. 3.1) against closed forms and invariants."""
import json
import os

import numpy as np
import pytest

from oracle.material import Material, lame, norm_sigma
import workloads as W

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
MAT = Material.from_dict(W.MATERIAL)


def voigt_strain_to_tensor(e):
    """Engineering-shear strain vector (e11, e22, e33, 2e12, 2e23, 2e13) -> 3x3 tensor."""
    t = np.zeros((3, 3))
    t[0, 0], t[1, 1], t[2, 2] = e[0], e[1], e[2]
    t[0, 1] = t[1, 0] = e[3] / 2
    t[1, 2] = t[2, 1] = e[4] / 2
    t[0, 2] = t[2, 0] = e[5] / 2
    return t


def stress_tensor_to_voigt(s):
    return np.array([s[0, 0], s[1, 1], s[2, 2], s[0, 1], s[1, 2], s[0, 2]])


def test_lame_against_printed_values():
    g = GOLDEN["material"]
    lam, mu = lame(g["young"], g["poisson"])
    assert round(lam, g["lambda_printed_decimals"]) == pytest.approx(g["lambda_printed"], abs=1e-9)
    # the printed mu is a factor-10 slip of the formula printed beside it
    assert round(10 * mu) == g["mu_printed"]
    assert (g["young"], g["poisson"], g["sigma_y"], g["hardening"]) == tuple(
        W.MATERIAL[k] for k in ("young", "poisson", "sigma_y", "hardening"))


def test_hooke_matrix_is_tensor_hooke_law():
    rng = np.random.default_rng(1)
    for _ in range(20):
        e = rng.standard_normal(6)
        eps = voigt_strain_to_tensor(e)
        sig = MAT.lam * np.trace(eps) * np.eye(3) + 2 * MAT.mu * eps       # eq. (Hook_law)
        np.testing.assert_allclose(MAT.C @ e, stress_tensor_to_voigt(sig), rtol=1e-13, atol=1e-9)


def test_deviator_and_norm_are_frobenius():
    rng = np.random.default_rng(2)
    for _ in range(20):
        s = rng.standard_normal((3, 3))
        s = s + s.T
        dev = s - np.trace(s) / 3 * np.eye(3)
        v = stress_tensor_to_voigt(s)
        np.testing.assert_allclose(MAT.E_sig @ v, stress_tensor_to_voigt(dev), atol=1e-14)
        assert norm_sigma((MAT.E_sig @ v)[None])[0] == pytest.approx(np.linalg.norm(dev), rel=1e-14)
        # E_eps maps a strain vector to the stress-form deviator of the strain tensor
        e = rng.standard_normal(6)
        et = voigt_strain_to_tensor(e)
        np.testing.assert_allclose(MAT.E_eps @ e, stress_tensor_to_voigt(et - np.trace(et) / 3 * np.eye(3)),
                                   atol=1e-14)


def shear_closed_form(gamma, mu, sy, H):
    """Simple shear from zero state: stress tau and hardening for engineering shear gamma."""
    gy = sy / (np.sqrt(3) * mu)
    if gamma <= gy:
        return mu * gamma, 0.0
    return sy / np.sqrt(3) + mu * H / (3 * mu + H) * (gamma - gy), (np.sqrt(3) * mu * gamma - sy) / (3 * mu + H)


@pytest.mark.parametrize("factor", [0.5, 0.999, 1.001, 2.0, 7.5])
def test_simple_shear_single_step(factor):
    gy = MAT.sigma_y / (np.sqrt(3) * MAT.mu)
    g = factor * gy
    eta = np.zeros((1, 6))
    eta[0, 3] = g
    ds, dk, pl = MAT.stress_increment(np.zeros((1, 6)), np.zeros(1), eta)
    tau, kap = shear_closed_form(g, MAT.mu, MAT.sigma_y, MAT.H)
    assert ds[0, 3] == pytest.approx(tau, rel=1e-13)
    np.testing.assert_allclose(ds[0, [0, 1, 2, 4, 5]], 0, atol=1e-9)
    assert dk[0] == pytest.approx(kap, rel=1e-12, abs=1e-18)
    assert bool(pl[0]) == (factor > 1)


def test_simple_shear_radial_path_independent_of_steps():
    gy = MAT.sigma_y / (np.sqrt(3) * MAT.mu)
    g_final = 5 * gy
    for n in (1, 3, 10):
        sig, kap = np.zeros((1, 6)), np.zeros(1)
        for k in range(n):
            eta = np.zeros((1, 6))
            eta[0, 3] = g_final / n
            ds, dk, _ = MAT.stress_increment(sig, kap, eta)
            sig, kap = sig + ds, kap + dk
        tau, kk = shear_closed_form(g_final, MAT.mu, MAT.sigma_y, MAT.H)
        assert sig[0, 3] == pytest.approx(tau, rel=1e-12)
        assert kap[0] == pytest.approx(kk, rel=1e-12)


def test_consistency_after_plastic_return():
    sig, kap, eta = W.seeded_gauss_point_inputs(4000, seed=3)
    ds, dk, pl = MAT.stress_increment(sig, kap, eta)
    assert 200 < pl.sum() < 3800
    phi_new = MAT.yield_function(sig + ds, kap + dk)
    scale = MAT.sigma_y + MAT.H * (kap + dk)
    assert np.all(np.abs(phi_new[pl]) <= 1e-12 * scale[pl])
    assert np.all(phi_new[~pl] <= 1e-12 * scale[~pl])
    assert np.all(dk[~pl] == 0.0) and np.all(dk[pl] > 0.0)
    # elastic branch: dsigma = C eta exactly
    np.testing.assert_array_equal(ds[~pl], (eta @ MAT.C.T)[~pl])


def test_tangent_is_derivative_of_stress_operator():
    sig, kap, eta = W.seeded_gauss_point_inputs(300, seed=4)
    tau = sig + eta @ MAT.C.T
    phi = MAT.yield_function(tau, kap)
    keep = np.abs(phi) > 1e-3 * MAT.sigma_y          # away from the kink Phi = 0
    sig, kap, eta = sig[keep], kap[keep], eta[keep]
    D = MAT.tangent(sig, kap, eta)
    h = 1e-7 * np.abs(eta).max()
    for j in range(6):
        ep, em = eta.copy(), eta.copy()
        ep[:, j] += h
        em[:, j] -= h
        fd = (MAT.stress_increment(sig, kap, ep)[0] - MAT.stress_increment(sig, kap, em)[0]) / (2 * h)
        err = np.abs(fd - D[:, :, j]).max(axis=1) / np.abs(D).max(axis=(1, 2))
        assert err.max() < 1e-6


def test_tangent_symmetric_and_spectral_bounds():
    sig, kap, eta = W.seeded_gauss_point_inputs(2000, seed=5)
    D = MAT.tangent(sig, kap, eta)
    np.testing.assert_allclose(D, np.swapaxes(D, 1, 2), atol=1e-9 * MAT.lam)
    _, _, pl = MAT.stress_increment(sig, kap, eta)
    assert pl.any() and (~pl).any()
    np.testing.assert_array_equal(D[~pl], np.broadcast_to(MAT.C, D[~pl].shape))
    # eq. (T_k^o-est): C >= T^o >= H/(3 mu + H) C, i.e. generalised eigenvalues in [H/(3mu+H), 1]
    Lc = np.linalg.cholesky(MAT.C)
    Li = np.linalg.inv(Lc)
    lo = MAT.H / (3 * MAT.mu + MAT.H)
    for Dg in D[pl][:200]:
        ev = np.linalg.eigvalsh(Li @ (0.5 * (Dg + Dg.T)) @ Li.T)
        assert ev.min() >= lo * (1 - 1e-10) and ev.max() <= 1 + 1e-10
