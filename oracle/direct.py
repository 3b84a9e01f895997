"""Undecomposed direct solve (test infrastructure only).

Assembles the global stiffness over global nodes, removes the Dirichlet dofs
(the tilde-restriction of Sec. 3.1, eq. (non_system)) and solves the linear
system with a sparse direct solver.  Used only to pin the TFETI solve: its
solution must coincide with every subdomain copy of the TFETI displacement.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def global_stiffness(model, du=None):
    """Global K (3 n_nodes square) from the element tangents at du (default: state tangent at du = 0)."""
    dec = model.dec
    du = np.zeros(dec.n_dof) if du is None else du
    eta = model.strains(du)
    D = model.mat.tangent(model.sigma, model.kappa, eta)
    from .fem import element_stiffness
    rows, cols, vals = [], [], []
    for p, s in enumerate(dec.subs):
        E = s.n_elements
        Ke = element_stiffness(model.Bg, D[model.gp_slice(p)].reshape(E, 8, 6, 6), model.wdet)
        gdof = (3 * s.global_node[s.element_local_nodes()][:, :, None] + np.arange(3)).reshape(E, 24)
        rows.append(np.repeat(gdof, 24, axis=1).ravel())
        cols.append(np.tile(gdof, (1, 24)).ravel())
        vals.append(Ke.ravel())
    n = 3 * model.grid.n_nodes
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def assemble_global_vector(model, f_dec: np.ndarray) -> np.ndarray:
    """Sum the subdomain copies of a decomposed load into global dofs."""
    dec = model.dec
    g = np.zeros(3 * model.grid.n_nodes)
    for p, s in enumerate(dec.subs):
        gd = (3 * s.global_node[:, None] + np.arange(3)).ravel()
        np.add.at(g, gd, f_dec[dec.dof_off[p]:dec.dof_off[p + 1]])
    return g


def fixed_dofs(model) -> np.ndarray:
    nid = np.arange(model.grid.n_nodes)
    mask = model.grid.node_dirichlet_mask(nid, model.dec.masks)
    fixed = [(mask >> c) & 1 for c in range(3)]
    return np.flatnonzero(np.stack(fixed, axis=1).ravel())


def solve_direct(model, f_dec: np.ndarray, du=None) -> np.ndarray:
    """Global displacement solving K~ u~ = f~ with u = 0 on the Dirichlet dofs."""
    K = global_stiffness(model, du)
    f = assemble_global_vector(model, f_dec)
    n = K.shape[0]
    free = np.setdiff1d(np.arange(n), fixed_dofs(model))
    u = np.zeros(n)
    u[free] = spla.spsolve(sp.csc_matrix(K[free][:, free]), f[free])
    return u


def scatter_to_decomposed(model, u_global: np.ndarray) -> np.ndarray:
    dec = model.dec
    out = np.zeros(dec.n_dof)
    for p, s in enumerate(dec.subs):
        gd = (3 * s.global_node[:, None] + np.arange(3)).ravel()
        out[dec.dof_off[p]:dec.dof_off[p + 1]] = u_global[gd]
    return out
