"""Hex8 finite elements on a box grid (test infrastructure only).

Sec. 3.1 discretises with P1 tetrahedra; the workloads use trilinear 8-node
bricks with 2x2x2 Gauss quadrature instead, so |T| of eq. (F_def)/(K_def) and of
Algorithm 5 becomes the quadrature weight times det J at each Gauss point.

Conventions (defined here, independently of the CUDA path):

* global node (i, j, k) has id i + (nx+1) (j + (ny+1) k), coordinates (i hx, j hy, k hz);
* element local nodes: bottom face counter-clockwise then top face,
  offsets (0,0,0) (1,0,0) (1,1,0) (0,1,0) (0,0,1) (1,0,1) (1,1,1) (0,1,1);
* element dof 3a + c for local node a and component c;
* Gauss point g = gx + 2 gy + 4 gz at reference coordinates (2 g_d - 1)/sqrt(3), weight 1;
* strain rows in the order of eq. (stress_strain_vector):
  (e11, e22, e33, 2e12, 2e23, 2e13).
"""
from __future__ import annotations

import numpy as np

NODE_OFFSETS = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0],
                         [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]])
NODE_SIGNS = 2 * NODE_OFFSETS - 1


def gauss_points() -> np.ndarray:
    """8 x 3 reference coordinates, g = gx + 2 gy + 4 gz."""
    a = 1.0 / np.sqrt(3.0)
    pts = []
    for gz in range(2):
        for gy in range(2):
            for gx in range(2):
                pts.append([(2 * gx - 1) * a, (2 * gy - 1) * a, (2 * gz - 1) * a])
    return np.array(pts)


def shape_gradients_ref(xi: np.ndarray) -> np.ndarray:
    """dN_a/dxi_d (8 x 3) of N_a = prod_d (1 + s_ad xi_d) / 8."""
    G = np.zeros((8, 3))
    for a in range(8):
        s = NODE_SIGNS[a]
        for d in range(3):
            v = s[d] / 8.0
            for e in range(3):
                if e != d:
                    v *= 1.0 + s[e] * xi[e]
            G[a, d] = v
    return G


def strain_matrix(h, xi) -> np.ndarray:
    """6 x 24 matrix G_T R_T of eq. (stress_displ_alg) at reference point xi of a box element of size h."""
    dN = shape_gradients_ref(np.asarray(xi)) * (2.0 / np.asarray(h, dtype=float))[None, :]
    B = np.zeros((6, 24))
    for a in range(8):
        dx, dy, dz = dN[a]
        c = 3 * a
        B[0, c + 0] = dx
        B[1, c + 1] = dy
        B[2, c + 2] = dz
        B[3, c + 0] = dy   # 2 e12 = du1/dx2 + du2/dx1
        B[3, c + 1] = dx
        B[4, c + 1] = dz   # 2 e23
        B[4, c + 2] = dy
        B[5, c + 0] = dz   # 2 e13
        B[5, c + 2] = dx
    return B


def element_strain_matrices(h) -> np.ndarray:
    """(8, 6, 24): one strain matrix per Gauss point (identical for every box element of size h)."""
    return np.stack([strain_matrix(h, xi) for xi in gauss_points()])


def gauss_weight_detj(h) -> float:
    """w_g det J = hx hy hz / 8 for every Gauss point of a box element."""
    return float(h[0] * h[1] * h[2]) / 8.0


def element_stiffness(Bg: np.ndarray, D: np.ndarray, wdet: float) -> np.ndarray:
    """sum_g w_g detJ B_g^T D_g B_g for a batch: D (E, 8, 6, 6) -> (E, 24, 24).  Eq. (K_def), Algorithm 5."""
    DB = np.einsum("egij,gjb->egib", D, Bg)
    return wdet * np.einsum("gia,egib->eab", Bg, DB)


def element_internal_force(Bg: np.ndarray, dsigma: np.ndarray, wdet: float) -> np.ndarray:
    """sum_g w_g detJ B_g^T dsigma_g: dsigma (E, 8, 6) -> (E, 24).  Eq. (F_def), Algorithm 5."""
    return wdet * np.einsum("gia,egi->ea", Bg, dsigma)


class Grid:
    """Box [0,L]^3 cut into nx x ny x nz equal bricks."""

    def __init__(self, nel, length=(1.0, 1.0, 1.0)):
        self.nel = tuple(int(v) for v in nel)
        self.length = tuple(float(v) for v in length)
        self.h = tuple(self.length[d] / self.nel[d] for d in range(3))
        self.nnode_axis = tuple(v + 1 for v in self.nel)
        self.n_nodes = int(np.prod(self.nnode_axis))
        self.n_elements = int(np.prod(self.nel))

    def node_id(self, i, j, k):
        nx1, ny1, _ = self.nnode_axis
        return i + nx1 * (j + ny1 * k)

    def node_ijk(self, nid):
        nid = np.asarray(nid)
        nx1, ny1, _ = self.nnode_axis
        return nid % nx1, (nid // nx1) % ny1, nid // (nx1 * ny1)

    def element_nodes(self, ei, ej, ek) -> np.ndarray:
        """Global node ids of element (ei, ej, ek), local order NODE_OFFSETS."""
        return np.array([self.node_id(ei + o[0], ej + o[1], ek + o[2]) for o in NODE_OFFSETS])

    def node_dirichlet_mask(self, nid, masks) -> np.ndarray:
        """Union of the face masks (x0, x1, y0, y1, z0, z1) of the faces a node lies on."""
        i, j, k = self.node_ijk(nid)
        idx = (i, j, k)
        out = np.zeros(np.shape(nid), dtype=np.int64)
        for d in range(3):
            out |= np.where(idx[d] == 0, masks[2 * d], 0)
            out |= np.where(idx[d] == self.nel[d], masks[2 * d + 1], 0)
        return out


def face_axis_side(face: str):
    return "xyz".index(face[0]), int(face[1])
