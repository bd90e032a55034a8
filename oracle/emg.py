"""FP64 oracle of the fiber-to-3D coupling -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
import this module.  It shares no code with the CUDA library.

What it computes (Maier 2021):

* The prolongation P of eq:discretized_fibers_2: the transmembrane voltage on
  the fibers' points is mapped to the nodes of a structured hexahedral 3D
  mesh by the data mapping of sec:data_mapping_between_meshes,
  eq:mapping_source_target: every source point s contributes to the 8 nodes
  of the 3D element that contains it, with the value of each node's
  trilinear ansatz function at the point, and the value at a 3D node t is
  the sum of the contributions divided by the sum of its factors,
      V3D_t = sum_s phi_t(xi_s) V_s / sum_s phi_t(xi_s).
* The static first bidomain equation eq:bidomain1 discretised by linear
  (trilinear) finite elements, eq:static_bidomain_rhs /
  eq:discretized_fibers_3:
      K_(sigma_i + sigma_e) phi_e = -K_(sigma_i) V3D,
  with homogeneous Neumann boundaries for both potentials
  (eq:monodomain_bc3), so the boundary term vanishes.  K_sigma is the
  stiffness matrix of the conduction tensor sigma, assembled element by
  element with 2-point Gauss quadrature per direction (exact for these
  integrands).  sigma_i = sigma_i_f a (x) a along the fiber direction a and
  sigma_e isotropic (eq:multidomain_isotropic_e).

Readings where the thesis is silent:
* The Neumann problem fixes phi_e up to a constant; the oracle returns the
  solution with zero arithmetic mean over the 3D nodes.
* A 3D node that no source point contributes to (zero factor sum) gets the
  value 0.
* A source point on an element face belongs to the element with the lower
  index (the ansatz functions agree on shared faces, so the result does not
  depend on this choice).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Tuple

import numpy as np


@dataclass
class Mesh3D:
    """Structured hexahedral mesh: nodes origin + (i hx, j hy, k hz)."""
    nx: int
    ny: int
    nz: int
    origin: Tuple[float, float, float]
    spacing: Tuple[float, float, float]

    @property
    def n_nodes(self) -> int:
        return self.nx * self.ny * self.nz

    def index(self, i, j, k):
        """Node numbering: x fastest, then y, then z."""
        return (np.asarray(k) * self.ny + np.asarray(j)) * self.nx + np.asarray(i)


def locate(mesh: Mesh3D, pts: np.ndarray):
    """Element (ei, ej, ek) and local coordinates xi in [0, 1]^3 of each point
    (points outside the mesh are clamped onto its boundary elements)."""
    pts = np.asarray(pts, np.float64)
    out_e = np.zeros((pts.shape[0], 3), np.int64)
    out_xi = np.zeros((pts.shape[0], 3))
    for d, n in enumerate((mesh.nx, mesh.ny, mesh.nz)):
        q = (pts[:, d] - mesh.origin[d]) / mesh.spacing[d]
        e = np.clip(np.floor(q).astype(np.int64), 0, n - 2)
        out_e[:, d] = e
        out_xi[:, d] = np.clip(q - e, 0.0, 1.0)
    return out_e, out_xi


def trilinear(xi: np.ndarray) -> np.ndarray:
    """Values of the 8 trilinear ansatz functions at local coordinates xi;
    corner c = (cx, cy, cz) in {0,1}^3 is column cx + 2 cy + 4 cz."""
    out = np.ones((xi.shape[0], 8))
    for c in range(8):
        for d in range(3):
            bit = (c >> d) & 1
            out[:, c] *= xi[:, d] if bit else (1.0 - xi[:, d])
    return out


def prolongation_matrix(mesh: Mesh3D, pts: np.ndarray):
    """(P, weight_sum): P is the dense-free list form of eq:mapping_source_target
    as a scipy CSR matrix (3D nodes x points) with rows normalised by the
    factor sums; weight_sum is the factor sum of every 3D node."""
    import scipy.sparse as sp
    e, xi = locate(mesh, pts)
    phi = trilinear(xi)
    rows, cols, vals = [], [], []
    for c in range(8):
        cx, cy, cz = c & 1, (c >> 1) & 1, (c >> 2) & 1
        t = mesh.index(e[:, 0] + cx, e[:, 1] + cy, e[:, 2] + cz)
        rows.append(t)
        cols.append(np.arange(pts.shape[0]))
        vals.append(phi[:, c])
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    B_T = sp.csr_matrix((vals, (rows, cols)), shape=(mesh.n_nodes, pts.shape[0]))
    wsum = np.asarray(B_T.sum(axis=1)).ravel()
    inv = np.where(wsum > 0, 1.0 / np.where(wsum > 0, wsum, 1.0), 0.0)
    P = sp.diags(inv) @ B_T
    return P.tocsr(), wsum


def prolongate(mesh: Mesh3D, pts: np.ndarray, values: np.ndarray) -> np.ndarray:
    """V3D of eq:discretized_fibers_2 at every 3D node."""
    P, _ = prolongation_matrix(mesh, pts)
    return P @ np.asarray(values, np.float64)


def element_stiffness(spacing, sigma) -> np.ndarray:
    """8 x 8 stiffness matrix of one hexahedral element of sizes `spacing`
    for the diagonal conduction tensor diag(sigma): the integral of
    grad(phi_a) . sigma grad(phi_b) by 2 x 2 x 2 Gauss quadrature."""
    h = np.asarray(spacing, np.float64)
    s = np.asarray(sigma, np.float64)
    g = 0.5 * (1.0 + np.array([-1.0, 1.0]) / np.sqrt(3.0))  # Gauss points on [0, 1]
    Ke = np.zeros((8, 8))
    for gx in g:
        for gy in g:
            for gz in g:
                xi = np.array([gx, gy, gz])
                grad = np.zeros((8, 3))  # physical gradients of the 8 ansatz functions
                for c in range(8):
                    bits = [(c >> d) & 1 for d in range(3)]
                    f = [xi[d] if bits[d] else 1.0 - xi[d] for d in range(3)]
                    df = [1.0 if bits[d] else -1.0 for d in range(3)]
                    grad[c] = [df[0] * f[1] * f[2] / h[0], f[0] * df[1] * f[2] / h[1], f[0] * f[1] * df[2] / h[2]]
                w = 0.125 * h[0] * h[1] * h[2]  # quadrature weight x element volume
                Ke += w * (grad * s) @ grad.T
    return Ke


def stiffness(mesh: Mesh3D, sigma):
    """Global stiffness matrix K_sigma (scipy CSR), assembled element by element."""
    import scipy.sparse as sp
    Ke = element_stiffness(mesh.spacing, sigma)
    ei, ej, ek = np.meshgrid(np.arange(mesh.nx - 1), np.arange(mesh.ny - 1), np.arange(mesh.nz - 1), indexing="ij")
    ei, ej, ek = ei.ravel(), ej.ravel(), ek.ravel()
    nodes = np.stack([mesh.index(ei + (c & 1), ej + ((c >> 1) & 1), ek + ((c >> 2) & 1)) for c in range(8)], axis=1)
    rows = np.repeat(nodes, 8, axis=1).ravel()
    cols = np.tile(nodes, (1, 8)).ravel()
    vals = np.tile(Ke.ravel(), nodes.shape[0])
    return sp.csr_matrix((vals, (rows, cols)), shape=(mesh.n_nodes, mesh.n_nodes))


def conductivities(sigma_i_fiber: float, sigma_e: float, fiber_axis: int = 2):
    """(sigma_i, sigma_i + sigma_e) as diagonals: intracellular conduction
    along the fiber axis only, extracellular isotropic."""
    si = np.zeros(3)
    si[fiber_axis] = sigma_i_fiber
    return si, si + sigma_e


def phi_e(mesh: Mesh3D, v3d: np.ndarray, sigma_i_fiber: float, sigma_e: float, fiber_axis: int = 2) -> np.ndarray:
    """Solution of K_(sigma_i+sigma_e) phi_e = -K_(sigma_i) V3D with zero mean
    (direct sparse solve with node 0 pinned, then the mean removed)."""
    import scipy.sparse.linalg as spla
    si, st = conductivities(sigma_i_fiber, sigma_e, fiber_axis)
    Ki = stiffness(mesh, si)
    Kt = stiffness(mesh, st).tolil()
    rhs = -(Ki @ np.asarray(v3d, np.float64))
    Kt[0, :] = 0.0
    Kt[0, 0] = 1.0
    rhs[0] = 0.0
    x = spla.spsolve(Kt.tocsc(), rhs)
    return x - x.mean()


def fiber_points(n_nodes, fiber_xy, h: float, z0: float = 0.0) -> np.ndarray:
    """3D positions of every fiber node in ragged order: fiber f at
    (x_f, y_f), node k at z0 + k h (straight fibers along z)."""
    n_nodes = np.asarray(n_nodes, np.int64)
    xy = np.asarray(fiber_xy, np.float64)
    out = np.zeros((int(n_nodes.sum()), 3))
    o = 0
    for f, n in enumerate(n_nodes):
        out[o:o + n, 0] = xy[f, 0]
        out[o:o + n, 1] = xy[f, 1]
        out[o:o + n, 2] = z0 + h * np.arange(n)
        o += n
    return out
