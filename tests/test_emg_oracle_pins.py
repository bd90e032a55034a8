"""Pins of the FP64 fiber-to-3D coupling oracle (oracle/emg.py) against what
the mathematics fixes: textbook element matrices of trilinear hexahedra, an
independent tensor-product derivation of the stiffness matrix, exact
discrete eigenmodes of the Neumann problem, and a brute-force evaluation of
the data mapping of eq:mapping_source_target on tiny inputs."""
import itertools

import numpy as np
import pytest

from oracle import emg as E


def test_unit_cube_element_stiffness_is_the_textbook_matrix():
    # Q1 hexahedron, unit cube, sigma = I: diagonal 1/3; nodes sharing an
    # edge 0; face diagonal -1/12; space diagonal -1/12
    Ke = E.element_stiffness((1.0, 1.0, 1.0), (1.0, 1.0, 1.0))
    for a, b in itertools.product(range(8), range(8)):
        d = bin(a ^ b).count("1")
        want = {0: 1.0 / 3.0, 1: 0.0, 2: -1.0 / 12.0, 3: -1.0 / 12.0}[d]
        assert abs(Ke[a, b] - want) < 1e-14


def test_assembled_interior_stencil_is_the_27_point_q1_laplacian():
    m = E.Mesh3D(5, 5, 5, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    K = E.stiffness(m, (1.0, 1.0, 1.0)).toarray()
    c = m.index(2, 2, 2)
    for di, dj, dk in itertools.product((-1, 0, 1), repeat=3):
        d = abs(di) + abs(dj) + abs(dk)
        want = {0: 8.0 / 3.0, 1: 0.0, 2: -1.0 / 6.0, 3: -1.0 / 12.0}[d]
        assert abs(K[c, m.index(2 + di, 2 + dj, 2 + dk)] - want) < 1e-13


def test_element_stiffness_equals_the_tensor_product_of_1d_matrices():
    # independent derivation: for a diagonal tensor on a box element the Q1
    # stiffness is sx Kx(x)My(x)Mz + sy Mx(x)Ky(x)Mz + sz Mx(x)My(x)Kz
    rng = np.random.default_rng(0)
    for _ in range(5):
        h = rng.uniform(0.05, 2.0, 3)
        s = rng.uniform(0.0, 10.0, 3)
        K1 = [np.array([[1.0, -1.0], [-1.0, 1.0]]) / hh for hh in h]
        M1 = [np.array([[2.0, 1.0], [1.0, 2.0]]) * hh / 6.0 for hh in h]
        # corner index c = cx + 2 cy + 4 cz -> kron order (z, y, x)
        ref = (s[0] * np.kron(M1[2], np.kron(M1[1], K1[0])) + s[1] * np.kron(M1[2], np.kron(K1[1], M1[0]))
               + s[2] * np.kron(K1[2], np.kron(M1[1], M1[0])))
        assert np.max(np.abs(E.element_stiffness(h, s) - ref)) < 1e-12 * np.max(np.abs(ref))


def test_stiffness_annihilates_constants_and_is_symmetric_semidefinite():
    m = E.Mesh3D(4, 6, 5, (0.0, 0.0, 0.0), (0.3, 0.2, 0.5))
    K = E.stiffness(m, (6.7, 6.7, 15.63)).toarray()
    assert np.max(np.abs(K @ np.ones(m.n_nodes))) < 1e-12
    assert np.max(np.abs(K - K.T)) < 1e-13
    w = np.linalg.eigvalsh(K)
    assert w.min() > -1e-10 and np.sum(w < 1e-10) == 1  # one-dimensional null space


def _mode(m, kx, ky, kz):
    i, j, k = np.meshgrid(np.arange(m.nx), np.arange(m.ny), np.arange(m.nz), indexing="ij")
    v = (np.cos(np.pi * kx * i / (m.nx - 1)) * np.cos(np.pi * ky * j / (m.ny - 1))
         * np.cos(np.pi * kz * k / (m.nz - 1)))
    out = np.zeros(m.n_nodes)
    out[m.index(i.ravel(), j.ravel(), k.ravel())] = v.ravel()
    return out


@pytest.mark.parametrize("modes", [(1, 0, 0), (0, 0, 1), (2, 1, 3), (1, 1, 1)])
def test_phi_e_of_a_cosine_mode_has_the_closed_form_amplitude(modes):
    # Products of cosines are exact eigenvectors of the assembled 1D Neumann
    # stiffness and mass matrices (with the halved boundary rows of both), so
    # K_sigma v = sum_d s_d lam_d prod_(d' != d) mu_d' W v for every diagonal
    # sigma, and phi_e = c V with
    #   c = -sum_d si_d lam_d prod mu / sum_d (si + se)_d lam_d prod mu,
    # lam = (2/h)(1 - cos t), mu = (h/3)(2 + cos t), t = k pi / (n - 1).
    m = E.Mesh3D(7, 6, 9, (0.0, 0.0, 0.0), (0.15, 0.2, 0.37))
    si_f, se = 8.93, 6.7
    V = _mode(m, *modes)
    phi = E.phi_e(m, V, si_f, se)
    lam, mu = [], []
    for k, n, h in zip(modes, (m.nx, m.ny, m.nz), m.spacing):
        t = np.pi * k / (n - 1)
        lam.append(2.0 / h * (1.0 - np.cos(t)))
        mu.append(h / 3.0 * (2.0 + np.cos(t)))
    si = np.array([0.0, 0.0, si_f])
    st = si + se
    prod = [mu[1] * mu[2], mu[0] * mu[2], mu[0] * mu[1]]
    c = -sum(si[d] * lam[d] * prod[d] for d in range(3)) / sum(st[d] * lam[d] * prod[d] for d in range(3))
    ref = c * V
    ref -= ref.mean()
    assert np.max(np.abs(phi - ref)) <= 1e-10 * max(1.0, np.max(np.abs(ref)))


def test_phi_e_amplitude_converges_to_the_continuum_at_second_order():
    # For V = cos(pi x / Lx) cos(pi z / Lz) the continuous problem gives
    # phi_e = -(si kz^2) / (se kx^2 + (si + se) kz^2) V.  Refining the mesh
    # must bring the discrete amplitude to it at order 2.
    Lx, Lz, si, se = 1.0, 3.0, 8.93, 6.7
    kx, kz = np.pi / Lx, np.pi / Lz
    exact = -(si * kz ** 2) / (se * kx ** 2 + (si + se) * kz ** 2)
    errs = []
    for n in (5, 9, 17):
        # unequal mode angles in x and z (otherwise the discrete x and z
        # factors scale alike and the amplitude is exact at any size)
        nz = 2 * n - 1
        m = E.Mesh3D(n, 3, nz, (0.0, 0.0, 0.0), (Lx / (n - 1), 0.5, Lz / (nz - 1)))
        V = _mode(m, 1, 0, 1)
        phi = E.phi_e(m, V, si, se)
        c = phi @ V / (V @ V)
        errs.append(abs(c - exact))
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(order > 1.8) and np.all(order < 2.2)


def test_prolongation_matches_a_brute_force_evaluation():
    # tiny mesh, random points: eq:mapping_source_target evaluated with plain
    # loops over every (node, point) pair and the trilinear hat functions
    # written directly in physical coordinates
    rng = np.random.default_rng(3)
    m = E.Mesh3D(3, 4, 3, (0.5, -1.0, 2.0), (0.4, 0.3, 0.7))
    lo = np.array(m.origin)
    hi = lo + np.array(m.spacing) * (np.array([m.nx, m.ny, m.nz]) - 1)
    pts = rng.uniform(lo, hi, (40, 3))
    vals = rng.normal(size=40)
    got = E.prolongate(m, pts, vals)
    for i, j, k in itertools.product(range(m.nx), range(m.ny), range(m.nz)):
        node = lo + np.array(m.spacing) * (i, j, k)
        num = den = 0.0
        for p, v in zip(pts, vals):
            # hat function of the node at the point (non-zero only in the
            # node's 8 surrounding elements)
            w = 1.0
            for d in range(3):
                w *= max(0.0, 1.0 - abs(p[d] - node[d]) / m.spacing[d])
            num += w * v
            den += w
        want = num / den if den > 0 else 0.0
        assert abs(got[m.index(i, j, k)] - want) < 1e-12


def test_prolongation_keeps_constants_and_symmetric_linear_fields():
    # fibers on a regular grid finer than the 3D mesh and aligned with it:
    # the normalised factors average symmetrically around interior nodes
    m = E.Mesh3D(5, 5, 4, (0.0, 0.0, 0.0), (0.3, 0.3, 0.4))
    xs = np.arange(13) * 0.1
    xy = np.array([(x, y) for y in xs for x in xs])
    pts = E.fiber_points(np.full(xy.shape[0], 13), xy, 0.1)
    ones = E.prolongate(m, pts, np.ones(pts.shape[0]))
    assert np.max(np.abs(ones - 1.0)) < 1e-14
    lin = 2.0 * pts[:, 0] - 3.0 * pts[:, 1] + 0.5 * pts[:, 2] + 1.0
    v3 = E.prolongate(m, pts, lin)
    for i, j, k in itertools.product(range(1, m.nx - 1), range(1, m.ny - 1), range(1, m.nz - 1)):
        x, y, z = np.array(m.spacing) * (i, j, k)
        assert abs(v3[m.index(i, j, k)] - (2 * x - 3 * y + 0.5 * z + 1.0)) < 1e-12
