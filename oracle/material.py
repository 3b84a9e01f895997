"""Material point: Hooke law, von Mises return mapping and consistent tangent.

Test infrastructure only (see the package docstring).

Follows Sec. 2.2 (Hooke law, eq. (Hook_law)), Sec. 2.4 (trial stress (trial),
elastic predictor (elast_pred), plastic corrector (plast_corr), operators
(stress_op), (hardening_op), Clarke derivative (stress_op_deriv_elast),
(stress_op_deriv_plast)) in the vector notation of Sec. 3.1:
stress vectors (s11, s22, s33, s12, s23, s13), strain vectors with engineering
shears (e11, e22, e33, 2e12, 2e23, 2e13), matrices C, E_eps, E_sig = P E_eps and
the norm ||tau||_sigma = sqrt(tau^T P tau).

All functions take arrays with a leading batch axis (one row per Gauss point).
"""
from __future__ import annotations

import numpy as np

SQRT_3_2 = np.sqrt(1.5)
SQRT_2_3 = np.sqrt(2.0 / 3.0)


def lame(young: float, poisson: float):
    """Lame coefficients from E and nu (Sec. 5 formulas).

    The paper prints mu = 801 938, a factor-10 slip; its own formula
    E / (2 (1 + nu)) gives 80 193.8, which is what is used here.
    """
    lam = young * poisson / ((1.0 + poisson) * (1.0 - 2.0 * poisson))
    mu = young / (2.0 * (1.0 + poisson))
    return lam, mu


def hooke_matrix(lam: float, mu: float) -> np.ndarray:
    """C of Sec. 3.1: maps a strain vector to a stress vector."""
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    for i in range(3):
        C[i, i] = lam + 2.0 * mu
        C[3 + i, 3 + i] = mu
    return C


def dev_strain_matrix() -> np.ndarray:
    """E_eps of Sec. 3.1 (deviatoric part of a strain vector, in stress form)."""
    E = np.zeros((6, 6))
    E[:3, :3] = -1.0
    for i in range(3):
        E[i, i] = 2.0
        E[3 + i, 3 + i] = 1.5
    return E / 3.0


P_MATRIX = np.diag([1.0, 1.0, 1.0, 2.0, 2.0, 2.0])


def dev_stress_matrix() -> np.ndarray:
    """E_sig = P E_eps (Sec. 3.1): deviatoric part of a stress vector."""
    return P_MATRIX @ dev_strain_matrix()


def norm_sigma(tau: np.ndarray) -> np.ndarray:
    """||tau||_sigma = sqrt(tau^T P tau), row-wise (Sec. 3.1)."""
    return np.sqrt(np.einsum("ni,ij,nj->n", tau, P_MATRIX, tau))


# Exact ties of the elastic-predictor test: a point returned to the yield surface at
# step k satisfies Phi(sigma_k, kappa_k) = 0 in exact arithmetic, which eq.
# (elast_pred) and the tangent of Sec. 3.1 treat as elastic (Phi <= 0).  Rounding
# leaves it at +-1 ulp, so |Phi| <= TIE (sigma_y + H kappa_k) counts as Phi = 0.
TIE = 1e-12


class Material:
    """Linear isotropic hardening von Mises material (Sec. 2.3, 2.4)."""

    def __init__(self, young: float, poisson: float, sigma_y: float, hardening: float):
        self.young, self.poisson = float(young), float(poisson)
        self.sigma_y, self.H = float(sigma_y), float(hardening)
        self.lam, self.mu = lame(self.young, self.poisson)
        self.C = hooke_matrix(self.lam, self.mu)
        self.E_eps = dev_strain_matrix()
        self.E_sig = dev_stress_matrix()

    @classmethod
    def from_dict(cls, d: dict) -> "Material":
        return cls(d["young"], d["poisson"], d["sigma_y"], d["hardening"])

    # -- Sec. 3.1, algebraic Phi and n-hat ------------------------------------
    def yield_function(self, tau: np.ndarray, kappa: np.ndarray) -> np.ndarray:
        """Phi(tau, kappa) = sqrt(3/2) ||E_sig tau||_sigma - (sigma_y + H kappa)."""
        dev = tau @ self.E_sig.T
        return SQRT_3_2 * norm_sigma(dev) - (self.sigma_y + self.H * kappa)

    def is_plastic(self, phi: np.ndarray, kappa: np.ndarray) -> np.ndarray:
        """Plastic branch of eq. (elast_pred): Phi > 0, with exact ties (|Phi| within TIE of the
        yield stress, the rounding of a return-mapped state) read as Phi = 0, i.e. elastic."""
        return phi > TIE * (self.sigma_y + self.H * kappa)

    def n_hat(self, tau: np.ndarray) -> np.ndarray:
        """n-hat(tau) = E_sig tau / ||E_sig tau||_sigma (eq. (hat_n))."""
        dev = tau @ self.E_sig.T
        return dev / norm_sigma(dev)[:, None]

    # -- eqs. (stress_op), (hardening_op) -------------------------------------
    def trial(self, sigma_k: np.ndarray, eta: np.ndarray) -> np.ndarray:
        """Trial stress sigma_k + C eta (eq. (trial))."""
        return sigma_k + eta @ self.C.T

    def stress_increment(self, sigma_k, kappa_k, eta):
        """T_k(eta): returns (dsigma, dkappa, plastic_flag).

        Elastic predictor if Phi(trial) <= 0 (eq. (elast_pred)), otherwise the
        plastic corrector (eq. (plast_corr)); dkappa = Phi^+ / (3 mu + H).
        """
        tau = self.trial(sigma_k, eta)
        phi = self.yield_function(tau, kappa_k)
        plastic = self.is_plastic(phi, kappa_k)
        phi_plus = np.where(plastic, phi, 0.0)
        c = 3.0 * self.mu / (3.0 * self.mu + self.H)
        ds = eta @ self.C.T
        if np.any(plastic):
            n = self.n_hat(tau[plastic])
            ds[plastic] -= (c * SQRT_2_3 * phi_plus[plastic])[:, None] * n
        dk = phi_plus / (3.0 * self.mu + self.H)
        return ds, dk, plastic

    def tangent(self, sigma_k, kappa_k, eta) -> np.ndarray:
        """Clarke derivative T^o_k(eta) of Sec. 3.1, one 6x6 matrix per point.

        C if Phi(sigma_k + C eta, kappa_k) <= 0, else
        C - 2mu c E_eps - 2mu c sqrt(2/3) (sigma_y + H kappa_k)/||E_sig tau||_sigma (nbar nbar^T - E_eps),
        c = 3 mu / (3 mu + H).
        """
        tau = self.trial(sigma_k, eta)
        phi = self.yield_function(tau, kappa_k)
        D = np.broadcast_to(self.C, (tau.shape[0], 6, 6)).copy()
        plastic = self.is_plastic(phi, kappa_k)
        if np.any(plastic):
            tp = tau[plastic]
            nbar = self.n_hat(tp)
            dn = norm_sigma(tp @ self.E_sig.T)
            c = 3.0 * self.mu / (3.0 * self.mu + self.H)
            coef = 2.0 * self.mu * c * SQRT_2_3 * (self.sigma_y + self.H * kappa_k[plastic]) / dn
            outer = np.einsum("ni,nj->nij", nbar, nbar)
            D[plastic] = (self.C - 2.0 * self.mu * c * self.E_eps)[None] \
                - coef[:, None, None] * (outer - self.E_eps[None])
        return D
