"""Algorithm 3: TFETI linear solve by projected preconditioned CG (test infrastructure only).

Solves min 1/2 v^T K v - f^T v subject to B v = 0 (eq. (equ.3radky)) through the
dual problem (eq. (equ:sps3)) with

    F = B K^dagger B^T,  N = -R^T B^T,  d = B K^dagger f,  e = -R^T f,
    P_N = I - N^T (N N^T)^{-1} N,  H = (N N^T)^{-1},

and the steps of Algorithm 3 in the paper's order: lambda_Im = N^T H e,
d~ = d - F lambda_Im, PCGP on lambda_Ker with r^0 = d~, then
alpha = H N (d - F lambda) and u = K^dagger (f - B^T lambda) + R alpha.

Preconditioners (Sec. 4.2): lumped, F^-1 ~ B K B^T; Dirichlet, F^-1 ~ Bbar Sbar Bbar^T
with Sbar_p the Schur complement of K_p onto the nodes that carry Dirichlet or
gluing conditions (all three components of such a node), eliminating the other
("interior") nodes, and Bbar the columns of B at those nodes.  The stopping test sits
after the updates and reads ||w^{j-1}|| <= eps ||r^0|| (Algorithm 3).  If
||w^0|| = 0 the loop ends with lambda_Ker = 0 and zero iterations.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


def constrained_node_dofs(dec, B: sp.spmatrix, p: int) -> np.ndarray:
    """Local dofs of subdomain p's nodes that carry a row of B (Dirichlet or gluing), all three
    components of each such node, in local order."""
    lo, hi = dec.dof_off[p], dec.dof_off[p + 1]
    has_col = np.diff(B.tocsc()[:, lo:hi].indptr) > 0
    node = has_col.reshape(-1, 3).any(axis=1)
    return np.nonzero(np.repeat(node, 3))[0]


def dirichlet_schur_blocks(dec, B: sp.spmatrix, K_blocks) -> list:
    """Per subdomain (global dof indices of the constrained nodes, Sbar_p), with
    Sbar_p = K_bb - K_bi K_ii^{-1} K_ib (dense Cholesky of the interior block)."""
    out = []
    for p, Kp in enumerate(K_blocks):
        Kp = sp.csr_matrix(Kp)
        n = Kp.shape[0]
        b = constrained_node_dofs(dec, B, p)
        i = np.setdiff1d(np.arange(n), b)
        Kbb = Kp[b][:, b].toarray()
        if i.size:
            Kib = Kp[i][:, b].toarray()
            Kii = Kp[i][:, i].toarray()
            X = sla.cho_solve(sla.cho_factor(Kii, lower=True), Kib)
            S = Kbb - Kib.T @ X
        else:
            S = Kbb
        out.append((dec.dof_off[p] + b, 0.5 * (S + S.T)))
    return out


class TFETISolver:
    def __init__(self, dec, K_blocks, kdag_blocks, R: sp.spmatrix | None = None, precond: str = "lumped"):
        """dec: Decomposition; K_blocks: per-subdomain sparse K_p; kdag_blocks: objects with .apply."""
        self.dec = dec
        self.B = dec.B
        self.K = sp.block_diag(K_blocks, format="csr")
        self.kdag = kdag_blocks
        self.R = dec.rigid_basis() if R is None else R
        self.N = sp.csr_matrix(-(self.R.T @ self.B.T))            # N = -R^T B^T
        NNt = (self.N @ self.N.T).toarray()
        self.NNt_chol = sla.cho_factor(NNt, lower=True)            # H = (N N^T)^{-1} via Cholesky
        self.precond = precond
        self.f_applies = 0
        if precond == "dirichlet":
            self.dirichlet_blocks = dirichlet_schur_blocks(dec, self.B, K_blocks)

    # -- operators ---------------------------------------------------------------
    def apply_kdag(self, x: np.ndarray) -> np.ndarray:
        y = np.empty_like(x)
        off = self.dec.dof_off
        for p, kd in enumerate(self.kdag):
            y[off[p]:off[p + 1]] = kd.apply(x[off[p]:off[p + 1]])
        return y

    def apply_F(self, lam: np.ndarray) -> np.ndarray:
        """F lambda = B K^dagger B^T lambda."""
        self.f_applies += 1
        return self.B @ self.apply_kdag(self.B.T @ lam)

    def apply_H(self, v: np.ndarray) -> np.ndarray:
        return sla.cho_solve(self.NNt_chol, v)

    def project(self, x: np.ndarray) -> np.ndarray:
        """P_N x = x - N^T (N N^T)^{-1} N x."""
        return x - self.N.T @ self.apply_H(self.N @ x)

    def apply_precond(self, w: np.ndarray) -> np.ndarray:
        if self.precond == "lumped":
            return self.B @ (self.K @ (self.B.T @ w))
        if self.precond == "dirichlet":
            v = self.B.T @ w
            z = np.zeros_like(v)
            for idx, S in self.dirichlet_blocks:
                z[idx] = S @ v[idx]
            return self.B @ z
        if self.precond == "none":
            return w.copy()
        raise ValueError(self.precond)

    # -- Algorithm 3 ---------------------------------------------------------------
    def solve(self, f: np.ndarray, rtol: float = 1e-8, maxit: int = 5000, history: list | None = None,
              check_feasibility=None):
        N, B = self.N, self.B
        d = B @ self.apply_kdag(f)                          # d = B K^dagger f
        e = -(self.R.T @ f)                                 # e = -R^T f
        lam_im = N.T @ self.apply_H(e)                      # lambda_Im = N^T H e
        d_tilde = d - self.apply_F(lam_im)                  # d~ = d - F lambda_Im
        r = d_tilde.copy()                                  # r^0 = d~
        lam_ker = np.zeros_like(r)                          # lambda_Ker^0 = o
        r0_norm = np.linalg.norm(r)
        p = None
        yw_prev = None
        it = 0
        w_norm = None
        converged = False
        for j in range(1, maxit + 1):
            w = self.project(r)                              # w^{j-1} = P_N r^{j-1}
            w_norm = np.linalg.norm(w)
            if j == 1 and w_norm == 0.0:
                converged = True
                break
            z = self.apply_precond(w)                        # z^{j-1}
            y = self.project(z)                              # y^{j-1} = P_N z^{j-1}
            yw = y @ w
            if p is None:
                p = y.copy()                                 # p^1 = y^0 (beta^1 = 0)
            else:
                beta = yw / yw_prev
                p = y + beta * p
            Fp = self.apply_F(p)
            gamma = yw / (p @ Fp)
            lam_ker = lam_ker + gamma * p
            r = r - gamma * Fp
            yw_prev = yw
            it = j
            if history is not None:
                history.append(w_norm / r0_norm if r0_norm > 0 else 0.0)
            if check_feasibility is not None:
                check_feasibility(lam_im + lam_ker)
            if w_norm <= rtol * r0_norm:                     # stop test on ||w^{j-1}||
                converged = True
                break
        lam = lam_im + lam_ker
        alpha = self.apply_H(N @ (d - self.apply_F(lam)))   # alpha = H N (d - F lambda)
        u = self.apply_kdag(f - B.T @ lam) + self.R @ alpha
        return {"u": u, "lam": lam, "alpha": alpha, "iterations": it, "converged": converged,
                "w_norm": w_norm, "r0_norm": r0_norm, "d": d, "e": e}
