"""TFETI tearing: box subdomains, constraint matrix B, kernel R, generalised inverse.

Test infrastructure only (see the package docstring).

Follows Sec. 4.1: the body is torn into subdomains and *all* subdomains float;
gluing and Dirichlet conditions are rows of one constraint matrix
B = [B_G; B_U] (eq. (equ.set.matrix.B)) in its orthonormal form.  The kernel of
each subdomain stiffness K_p is spanned by rigid-body modes whose orthonormal
basis forms R (Sec. 4.2).  K^dagger is the fixing-node generalised inverse of
Remark 1: the rows/columns of a few fixing dofs are removed so that the rest,
K_rr, is non-singular and Cholesky-factorisable without fill outside its band.

Readings of points the paper leaves open (all stated once here):

* subdomain id p = I + sx (J + sy K) for box (I, J, K); local node
  (li, lj, lk) has id li + (ax+1)(lj + (ay+1) lk), local dof 3 lnode + c;
  the decomposed vector is the concatenation of the subdomain vectors;
* the copies of a global node are ordered by subdomain id;
* B rows come in (global node, component) order.  A component fixed by a
  Dirichlet mask at that node gives one identity row per copy; a free
  component with k >= 2 copies gives the k-1 Helmert rows
  h_j = (e_1 + ... + e_j - j e_{j+1}) / sqrt(j (j+1)), j = 1..k-1, i.e. the
  orthonormalised redundant rows e_1 - e_j of Sec. 4.1;
* fixing dofs (3-2-1): corner (0,0,0) all three components, corner (ax,0,0)
  components y and z, corner (0,ay,0) component z;
* R columns: translations x, y, z, then rotations e_d x (X - X_centroid),
  d = x, y, z, orthonormalised by modified Gram-Schmidt in that order.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .fem import Grid, NODE_OFFSETS, face_axis_side


class Subdomain:
    def __init__(self, p, origin, dims, grid: Grid):
        self.p = p
        self.origin = tuple(int(v) for v in origin)   # element index of the lower corner
        self.dims = tuple(int(v) for v in dims)       # elements per axis
        ax, ay, az = self.dims
        self.nn_axis = (ax + 1, ay + 1, az + 1)
        self.n_nodes = (ax + 1) * (ay + 1) * (az + 1)
        self.n_dof = 3 * self.n_nodes
        self.n_elements = ax * ay * az
        li, lj, lk = np.meshgrid(np.arange(ax + 1), np.arange(ay + 1), np.arange(az + 1), indexing="ij")
        # local node order: li fastest
        li, lj, lk = (v.transpose(2, 1, 0).ravel() for v in (li, lj, lk))
        self.local_ijk = np.stack([li, lj, lk], axis=1)
        self.global_node = grid.node_id(li + self.origin[0], lj + self.origin[1], lk + self.origin[2])
        self.coords = np.stack([(self.local_ijk[:, d] + self.origin[d]) * grid.h[d] for d in range(3)], axis=1)

    def lnode(self, li, lj, lk):
        return li + self.nn_axis[0] * (lj + self.nn_axis[1] * lk)

    def element_local_nodes(self) -> np.ndarray:
        """(n_elements, 8) local node ids, elements in lexicographic order (x fastest)."""
        ax, ay, az = self.dims
        out = np.zeros((self.n_elements, 8), dtype=np.int64)
        e = 0
        for lk in range(az):
            for lj in range(ay):
                for li in range(ax):
                    for a, o in enumerate(NODE_OFFSETS):
                        out[e, a] = self.lnode(li + o[0], lj + o[1], lk + o[2])
                    e += 1
        return out

    def element_dofs(self) -> np.ndarray:
        """(n_elements, 24) local dofs."""
        ln = self.element_local_nodes()
        return (3 * ln[:, :, None] + np.arange(3)[None, None, :]).reshape(self.n_elements, 24)

    def fixing_dofs(self) -> np.ndarray:
        ax, ay, _ = self.dims
        a = self.lnode(0, 0, 0)
        b = self.lnode(ax, 0, 0)
        c = self.lnode(0, ay, 0)
        return np.array(sorted([3 * a, 3 * a + 1, 3 * a + 2, 3 * b + 1, 3 * b + 2, 3 * c + 2]))

    def rigid_modes(self) -> np.ndarray:
        """Orthonormal basis (n_dof x 6) of the rigid-body modes (kernel of K_p)."""
        X = self.coords - self.coords.mean(axis=0)
        R = np.zeros((self.n_dof, 6))
        for d in range(3):
            R[d::3, d] = 1.0
        # rotation about axis d: u = e_d x X
        e = np.eye(3)
        for d in range(3):
            u = np.cross(e[d][None, :], X)
            R[:, 3 + d] = u.ravel()
        for j in range(6):                      # modified Gram-Schmidt
            for i in range(j):
                R[:, j] -= (R[:, i] @ R[:, j]) * R[:, i]
            R[:, j] /= np.linalg.norm(R[:, j])
        return R


class Decomposition:
    """Box partition of a Grid, the orthonormal B and per-subdomain data."""

    def __init__(self, grid: Grid, cuts, dirichlet_masks):
        self.grid = grid
        self.cuts = tuple(tuple(int(v) for v in c) for c in cuts)
        self.masks = tuple(int(v) for v in dirichlet_masks)
        for d in range(3):
            c = self.cuts[d]
            if c[0] != 0 or c[-1] != grid.nel[d] or any(c[i] >= c[i + 1] for i in range(len(c) - 1)):
                raise ValueError("bad cuts")
        self.nsub_axis = tuple(len(c) - 1 for c in self.cuts)
        sx, sy, sz = self.nsub_axis
        self.subs = []
        for K in range(sz):
            for J in range(sy):
                for I in range(sx):
                    p = I + sx * (J + sy * K)
                    origin = (self.cuts[0][I], self.cuts[1][J], self.cuts[2][K])
                    dims = (self.cuts[0][I + 1] - origin[0], self.cuts[1][J + 1] - origin[1],
                            self.cuts[2][K + 1] - origin[2])
                    self.subs.append(Subdomain(p, origin, dims, grid))
        self.n_sub = len(self.subs)
        self.dof_off = np.concatenate([[0], np.cumsum([s.n_dof for s in self.subs])])
        self.elem_off = np.concatenate([[0], np.cumsum([s.n_elements for s in self.subs])])
        self.n_dof = int(self.dof_off[-1])
        self.n_gp = 8 * int(self.elem_off[-1])
        self._build_B()

    # -- copies and B -----------------------------------------------------------
    def _build_B(self):
        gnode = np.concatenate([s.global_node for s in self.subs])
        sub = np.concatenate([np.full(s.n_nodes, s.p) for s in self.subs])
        lnode = np.concatenate([np.arange(s.n_nodes) for s in self.subs])
        order = np.argsort(gnode, kind="stable")        # keeps subdomain order within a node
        gnode, sub, lnode = gnode[order], sub[order], lnode[order]
        starts = np.flatnonzero(np.r_[True, gnode[1:] != gnode[:-1]])
        ends = np.r_[starts[1:], gnode.size]
        node_mask = self.grid.node_dirichlet_mask(gnode[starts], self.masks)
        rows, cols, vals = [], [], []
        self.row_node, self.row_comp = [], []
        r = 0
        for g, (s0, s1) in enumerate(zip(starts, ends)):
            k = s1 - s0
            copies_dof = [self.dof_off[sub[t]] + 3 * lnode[t] for t in range(s0, s1)]
            for c in range(3):
                if (node_mask[g] >> c) & 1:
                    for j in range(k):            # Dirichlet: one identity row per copy
                        rows.append(r); cols.append(copies_dof[j] + c); vals.append(1.0)
                        self.row_node.append(gnode[s0]); self.row_comp.append(c)
                        r += 1
                elif k >= 2:
                    for j in range(1, k):         # Helmert rows h_j
                        s = 1.0 / np.sqrt(j * (j + 1.0))
                        for t in range(j):
                            rows.append(r); cols.append(copies_dof[t] + c); vals.append(s)
                        rows.append(r); cols.append(copies_dof[j] + c); vals.append(-j * s)
                        self.row_node.append(gnode[s0]); self.row_comp.append(c)
                        r += 1
        self.m = r
        self.B = sp.csr_matrix((vals, (rows, cols)), shape=(self.m, self.n_dof))
        self.row_node = np.array(self.row_node, dtype=np.int64)
        self.row_comp = np.array(self.row_comp, dtype=np.int64)

    def split(self, v: np.ndarray):
        """Views of a decomposed vector, one per subdomain."""
        return [v[self.dof_off[p]:self.dof_off[p + 1]] for p in range(self.n_sub)]

    def rigid_basis(self) -> sp.csr_matrix:
        """Block-diagonal R (n_dof x 6 s)."""
        return sp.block_diag([sp.csr_matrix(s.rigid_modes()) for s in self.subs], format="csr")

    def traction_load(self, face: str, t) -> np.ndarray:
        """Decomposed load of a uniform traction t on a face: each element face
        gives t * area / 4 to each of its four nodes, in the subdomain that owns
        the element (bilinear face integration, exact for a constant traction)."""
        axis, side = face_axis_side(face)
        h = self.grid.h
        area = np.prod([h[d] for d in range(3) if d != axis])
        f = np.zeros(self.n_dof)
        t = np.asarray(t, dtype=float)
        for s in self.subs:
            on_face = (s.origin[axis] == 0) if side == 0 else (s.origin[axis] + s.dims[axis] == self.grid.nel[axis])
            if not on_face:
                continue
            li = 0 if side == 0 else s.dims[axis]
            fl = f[self.dof_off[s.p]:self.dof_off[s.p + 1]]
            other = [d for d in range(3) if d != axis]
            for i0 in range(s.dims[other[0]]):
                for i1 in range(s.dims[other[1]]):
                    for o0 in range(2):
                        for o1 in range(2):
                            ijk = [0, 0, 0]
                            ijk[axis] = li
                            ijk[other[0]] = i0 + o0
                            ijk[other[1]] = i1 + o1
                            n = s.lnode(*ijk)
                            fl[3 * n:3 * n + 3] += t * area / 4.0
        return f


def band_lower(A: sp.spmatrix):
    """Lower banded form ab[k, j] = A[j + k, j] (LAPACK *pbtrf layout) and the half bandwidth."""
    A = sp.coo_matrix(A)
    low = A.row >= A.col
    r, c, v = A.row[low], A.col[low], A.data[low]
    bw = int((r - c).max()) if r.size else 0
    ab = np.zeros((bw + 1, A.shape[0]))
    np.add.at(ab, (r - c, c), v)
    return ab, bw


class FixingNodeInverse:
    """K^dagger = P^T [K_rr^{-1} 0; 0 0] P for one subdomain (Remark 1).

    K_rr is K with the fixing dofs' rows and columns removed; it is factorised
    by banded Cholesky (LAPACK dpbtrf through scipy) and applied by forward and
    backward substitution.  K K^dagger K = K holds because rank K_rr = rank K.
    """

    def __init__(self, K: sp.spmatrix, fixing: np.ndarray):
        n = K.shape[0]
        self.n = n
        self.keep = np.setdiff1d(np.arange(n), fixing)
        Krr = sp.csr_matrix(K)[self.keep][:, self.keep]
        ab, self.bw = band_lower(Krr)
        self.factor = sla.cholesky_banded(ab, lower=True)

    def apply(self, x: np.ndarray) -> np.ndarray:
        y = np.zeros(self.n)
        y[self.keep] = sla.cho_solve_banded((self.factor, True), x[self.keep])
        return y


class RegularisedInverse:
    """Alternative generalised inverse (K + rho R R^T)^{-1} = K^+ + R R^T / rho (dense; tiny cases only)."""

    def __init__(self, K: sp.spmatrix, R: np.ndarray, rho: float = 1.0):
        Kd = K.toarray() if sp.issparse(K) else np.asarray(K)
        self.M = np.linalg.inv(Kd + rho * R @ R.T)

    def apply(self, x):
        return self.M @ x
