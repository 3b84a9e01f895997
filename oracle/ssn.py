"""Algorithms 1, 2, 4, 5: load steps, semismooth Newton and subdomain assembly (test infrastructure only).

One load step (Algorithm 4, body of the time loop):

    du_0 = o
    for i = 1, 2, ...:
        per subdomain, Algorithm 5 at du_{i-1}: dsigma_T = T_k(G_T R_T du), dkappa_T = T_kappa(...),
            f^p = df^p - sum_T |T| dsigma_T^T G_T R_T,
            K^p = sum_T |T| (T^o_k(G_T R_T du) G_T R_T)^T G_T R_T
        Algorithm 3 on (K, f) -> delta u
        du_i = du_{i-1} + delta u
        stop if ||du_i - du_{i-1}|| / (||du_i|| + ||du_{i-1}||) <= eps_Newton
    u_{k+1} = u_k + du_i; sigma, kappa += T_k, T_kappa evaluated at du_i.

Readings: |T| is w_g det J at each Gauss point of a hex8 brick; the committed
stress is re-evaluated at the final du (Algorithm 1 evaluates T_k at the
solution), not the one Newton iterate behind that Algorithm 5 last produced;
if ||du_i|| + ||du_{i-1}|| = 0 the step has converged; norms are Euclidean over
the decomposed displacement vector.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .decomp import Decomposition, FixingNodeInverse
from .fem import Grid, element_strain_matrices, element_stiffness, element_internal_force, gauss_weight_detj
from .material import Material, SQRT_3_2, norm_sigma
from .tfeti import TFETISolver


class ElastoplasticModel:
    """Discretised body with Gauss-point state sigma_k, kappa_k and displacement u_k (Algorithm 1)."""

    def __init__(self, workload, material: dict | None = None, precond: str = "lumped"):
        self.w = workload
        self.grid = Grid(workload.nel, workload.length)
        self.dec = Decomposition(self.grid, workload.cuts, workload.dirichlet_masks())
        self.mat = Material.from_dict(material if material is not None else workload.material)
        self.Bg = element_strain_matrices(self.grid.h)
        self.wdet = gauss_weight_detj(self.grid.h)
        self.edofs = [s.element_dofs() for s in self.dec.subs]
        self.fixing = [s.fixing_dofs() for s in self.dec.subs]
        self.precond = precond
        n_gp = self.dec.n_gp
        self.sigma = np.zeros((n_gp, 6))
        self.kappa = np.zeros(n_gp)
        self.u = np.zeros(self.dec.n_dof)
        self.R = self.dec.rigid_basis()

    # -- Gauss-point indexing: gp = 8 (elem_off[p] + local element) + g ----------------
    def gp_slice(self, p):
        e0, e1 = self.dec.elem_off[p], self.dec.elem_off[p + 1]
        return slice(8 * e0, 8 * e1)

    def strains(self, du: np.ndarray) -> np.ndarray:
        """eta = G_T R_T du at every Gauss point, (n_gp, 6)."""
        out = np.zeros((self.dec.n_gp, 6))
        for p, s in enumerate(self.dec.subs):
            dul = du[self.dec.dof_off[p]:self.dec.dof_off[p + 1]]
            ue = dul[self.edofs[p]]                                   # (E, 24)
            out[self.gp_slice(p)] = np.einsum("gia,ea->egi", self.Bg, ue).reshape(-1, 6)
        return out

    def return_map(self, du: np.ndarray, sigma=None, kappa=None):
        """T_k and T_kappa at every Gauss point for the increment du."""
        sigma = self.sigma if sigma is None else sigma
        kappa = self.kappa if kappa is None else kappa
        eta = self.strains(du)
        ds, dk, plastic = self.mat.stress_increment(sigma, kappa, eta)
        return ds, dk, plastic, eta

    def assemble(self, du: np.ndarray, df: np.ndarray, subdomains=None):
        """Algorithm 4's subdomain loop calling Algorithm 5 for every subdomain (or the listed ones):
        K^p (sparse) and f^p (decomposed), plus dsigma, dkappa and plastic flags at the Gauss points."""
        n_gp = self.dec.n_gp
        ds_all, dk_all = np.zeros((n_gp, 6)), np.zeros(n_gp)
        pl_all = np.zeros(n_gp, dtype=bool)
        K_blocks = []
        f = df.copy()
        for p, s in enumerate(self.dec.subs):
            if subdomains is not None and p not in subdomains:
                continue
            sl = self.gp_slice(p)
            E = s.n_elements
            ue = du[self.dec.dof_off[p]:self.dec.dof_off[p + 1]][self.edofs[p]]          # (E, 24)
            eta = np.einsum("gia,ea->egi", self.Bg, ue).reshape(-1, 6)
            ds, dk, pl = self.mat.stress_increment(self.sigma[sl], self.kappa[sl], eta)
            D = self.mat.tangent(self.sigma[sl], self.kappa[sl], eta)
            ds_all[sl], dk_all[sl], pl_all[sl] = ds, dk, pl
            Ke = element_stiffness(self.Bg, D.reshape(E, 8, 6, 6), self.wdet)
            Fe = element_internal_force(self.Bg, ds.reshape(E, 8, 6), self.wdet)
            ed = self.edofs[p]
            rows = np.repeat(ed, 24, axis=1).ravel()
            cols = np.tile(ed, (1, 24)).ravel()
            K_blocks.append(sp.csr_matrix((Ke.ravel(), (rows, cols)), shape=(s.n_dof, s.n_dof)))
            fl = f[self.dec.dof_off[p]:self.dec.dof_off[p + 1]]
            np.subtract.at(fl, ed.ravel(), Fe.ravel())
        return K_blocks, f, {"dsigma": ds_all, "dkappa": dk_all, "plastic": pl_all}

    def internal_force(self, du: np.ndarray) -> np.ndarray:
        """F_k(du) of eq. (F_def) on the decomposed dofs."""
        ds, _, _, _ = self.return_map(du)
        f = np.zeros(self.dec.n_dof)
        for p, s in enumerate(self.dec.subs):
            Fe = element_internal_force(self.Bg, ds[self.gp_slice(p)].reshape(s.n_elements, 8, 6), self.wdet)
            fl = f[self.dec.dof_off[p]:self.dec.dof_off[p + 1]]
            np.add.at(fl, self.edofs[p].ravel(), Fe.ravel())
        return f

    def tfeti(self, K_blocks, kdag=None):
        if kdag is None:
            kdag = [FixingNodeInverse(K, fx) for K, fx in zip(K_blocks, self.fixing)]
        return TFETISolver(self.dec, K_blocks, kdag, R=self.R, precond=self.precond)

    def traction_load(self, t) -> np.ndarray:
        return self.dec.traction_load(self.w.traction_face, t)

    # -- Algorithm 4 (one time step) -------------------------------------------------------
    def time_step(self, df: np.ndarray, newton_tol: float, pcg_rtol: float, newton_maxit: int = 30,
                  pcg_maxit: int = 5000, log: list | None = None):
        du = np.zeros(self.dec.n_dof)
        info = {"newton": 0, "pcg": [], "criterion": [], "plastic": [], "converged": False}
        for i in range(1, newton_maxit + 1):
            K_blocks, f, st = self.assemble(du, df)
            sol = self.tfeti(K_blocks).solve(f, rtol=pcg_rtol, maxit=pcg_maxit)
            du_new = du + sol["u"]
            den = np.linalg.norm(du_new) + np.linalg.norm(du)
            crit = 0.0 if den == 0.0 else np.linalg.norm(du_new - du) / den
            du = du_new
            info["newton"] = i
            info["pcg"].append(sol["iterations"])
            info["criterion"].append(crit)
            info["plastic"].append(int(st["plastic"].sum()))
            if log is not None:
                log.append({"i": i, "pcg": sol["iterations"], "crit": crit, "plastic": int(st["plastic"].sum())})
            if crit <= newton_tol:
                info["converged"] = True
                break
        ds, dk, plastic, _ = self.return_map(du)          # commit at the converged increment
        self.sigma = self.sigma + ds
        self.kappa = self.kappa + dk
        self.u = self.u + du
        info["plastic_committed"] = int(plastic.sum())
        info["du"] = du
        return info

    # -- load magnitude of the workloads -------------------------------------------------------
    def first_yield_traction(self, rtol: float = 1e-12) -> float:
        """t_y = sigma_y / max_g sqrt(3/2) ||dev sigma_g|| for the elastic response to a unit traction."""
        assert not self.sigma.any() and not self.kappa.any()
        f1 = self.traction_load(self.w.traction_dir)
        K_blocks, f, _ = self.assemble(np.zeros(self.dec.n_dof), f1)
        u = self.tfeti(K_blocks).solve(f, rtol=rtol)["u"]
        sig = self.strains(u) @ self.mat.C.T
        q = SQRT_3_2 * norm_sigma(sig @ self.mat.E_sig.T)
        return self.mat.sigma_y / q.max()

    def von_mises(self, sigma=None):
        sigma = self.sigma if sigma is None else sigma
        return SQRT_3_2 * norm_sigma(sigma @ self.mat.E_sig.T)


def run_load_history(workload, n_steps: int | None = None, newton_tol=None, pcg_rtol=None, t_y=None):
    """Algorithm 1/4 over the workload's ramp; returns the model and per-step info."""
    model = ElastoplasticModel(workload)
    if t_y is None:
        t_y = model.first_yield_traction()
    fr = workload.load_fractions(n_steps)
    f1 = model.traction_load(workload.traction_dir)
    infos = []
    prev = 0.0
    for a in fr:
        df = (a - prev) * t_y * f1
        prev = a
        infos.append(model.time_step(df, newton_tol or workload.newton_tol, pcg_rtol or workload.pcg_rtol,
                                     workload.newton_maxit, workload.pcg_maxit))
    return model, infos, t_y
