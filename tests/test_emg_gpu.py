"""GPU parity of the fiber-to-3D coupling (eq:discretized_fibers_2 and _3):
the CUDA mapping V3D and the CUDA conjugate-gradient phi_e against the FP64
oracle (oracle/emg.py, direct sparse solve) on the same fiber voltages."""
import numpy as np
import pytest

from oracle import emg as E
from paper_2107_07104_gb300 import fibers as F
from paper_2107_07104_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SIGMA_I, SIGMA_E = 8.93, 6.7  # mS/cm (eq:multidomain_isotropic_e)


def _run(w, xy, mesh, steps, rtol=1e-10):
    """Fiber V after `steps` split steps, and the library's V3D and phi_e."""
    m = F.make_mesh3d(mesh["nx"], mesh["ny"], mesh["nz"], mesh["origin"], mesh["spacing"], SIGMA_I, SIGMA_E)
    with F.Fibers.from_workload(w) as f:
        f.step(steps)
        v = f.read_vm().astype(np.float64)
        emg = F.fibers_emg_create(f.ctx, xy, 0.0, m)
        try:
            n3 = F.fibers_emg_nodes(emg)
            v3 = np.empty(n3, np.float64)
            F.fibers_emg_vm3d(emg, v3)
            phi = np.empty(n3, np.float32)
            it, res = F.fibers_emg_phi_e(emg, phi, rtol=rtol)
        finally:
            F.fibers_emg_destroy(emg)
    return v, v3, phi.astype(np.float64), it, res


def _oracle(w, xy, mesh, v):
    m = E.Mesh3D(mesh["nx"], mesh["ny"], mesh["nz"], mesh["origin"], mesh["spacing"])
    pts = E.fiber_points(w.n_nodes, xy, w.params["h"])
    v3 = E.prolongate(m, pts, v)
    return v3, E.phi_e(m, v3, SIGMA_I, SIGMA_E)


def test_small_bundle_matches_the_oracle():
    # 6 x 6 fibers of 150-200 nodes (ragged), firing at 400 Hz: after 300
    # split steps action potentials are under way; a 4 x 4 x 9 mesh
    w = W.small_ragged(seed=41, n_fibers=36, lo=150, hi=200, n_steps=300)
    xy = W.fiber_grid_xy(6, 0.05)
    mesh = W.box_mesh(xy, 2.0, 4, 9)
    v, v3, phi, it, res = _run(w, xy, mesh, 300)
    assert v.max() > 0.0  # some fibers are depolarised
    r3, rphi = _oracle(w, xy, mesh, v)
    # V3D: FP32 mapping factors (relative 6e-8) times |V| <= 130 mV
    assert np.max(np.abs(v3 - r3)) <= 1e-4
    # phi_e: FP64 CG to 1e-10 of the right-hand side, stored as float
    assert res <= 1e-10 and it > 0
    scale = np.max(np.abs(rphi))
    assert scale > 0.0
    assert np.max(np.abs(phi - rphi)) <= 1e-5 * scale
    assert abs(phi.mean()) <= 1e-6 * scale


def test_constant_voltage_gives_zero_extracellular_potential():
    # at rest every node has V = Vrest: V3D is constant, K_sigma_i V3D = 0
    w = W.small_ragged(seed=42, n_fibers=4, lo=60, hi=60, n_steps=1, v0_sigma=0.0)
    w.mu_of_fiber[:] = -1  # never stimulated
    xy = W.fiber_grid_xy(2, 0.1)
    mesh = W.box_mesh(xy, 0.59, 2, 3)
    v, v3, phi, it, res = _run(w, xy, mesh, 0)
    assert np.all(v == w.params["Vrest"])
    # the FP32 mapping factors of a node sum to 1 within rounding
    assert np.max(np.abs(v3 - w.params["Vrest"])) < 1e-4
    assert np.max(np.abs(phi)) < 1e-6


def test_fibers_outside_the_mesh_are_clamped_onto_it():
    # the mesh covers only the middle of the bundle: outer fibers and the
    # fiber ends are clamped onto boundary elements, as the oracle does
    w = W.small_ragged(seed=43, n_fibers=16, lo=120, hi=150, n_steps=250)
    xy = W.fiber_grid_xy(4, 0.1)
    mesh = dict(nx=3, ny=3, nz=5, origin=(0.05, 0.05, 0.2), spacing=(0.1, 0.1, 0.2))
    v, v3, phi, it, res = _run(w, xy, mesh, 250)
    r3, rphi = _oracle(w, xy, mesh, v)
    assert np.max(np.abs(v3 - r3)) <= 1e-4
    assert np.max(np.abs(phi - rphi)) <= 1e-5 * max(np.max(np.abs(rphi)), 1e-12)


def test_bad_meshes_are_rejected():
    w = W.small_ragged(seed=44, n_fibers=4, lo=20, hi=30, n_steps=1)
    xy = W.fiber_grid_xy(2, 0.1)
    with F.Fibers.from_workload(w) as f:
        for bad in (dict(nx=1), dict(spacing=(0.0, 0.1, 0.1)), dict(sigma_e=0.0), dict(sigma_i=-1.0)):
            kw = dict(nx=3, ny=3, nz=3, origin=(0.0, 0.0, 0.0), spacing=(0.1, 0.1, 0.1), sigma_i=8.93, sigma_e=6.7)
            kw.update(bad)
            m = F.make_mesh3d(kw["nx"], kw["ny"], kw["nz"], kw["origin"], kw["spacing"], kw["sigma_i"], kw["sigma_e"])
            with pytest.raises(F.FibersError) as ei:
                F.fibers_emg_create(f.ctx, xy, 0.0, m)
            assert ei.value.status == F.FIB_EINVAL


def test_bundle_7744_geometry_matches_the_oracle():
    # the 88 x 88 bundle at 0.05 cm spacing (4.35 cm across, 14.8 cm long)
    # with a 30 x 30 x 41 mesh (36,900 nodes), 4.5 ms into the run
    w = W.bundle_7744(seed=2, t_end_ms=20.0)
    xy = W.fiber_grid_xy(88, 0.05)
    mesh = W.box_mesh(xy, 14.8, 30, 41)
    v, v3, phi, it, res = _run(w, xy, mesh, 1500)
    r3, rphi = _oracle(w, xy, mesh, v)
    assert np.max(np.abs(v3 - r3)) <= 1e-4
    scale = np.max(np.abs(rphi))
    print(f"[emg] 36900 nodes: CG {it} iterations, residual {res:.2e}, max|phi_e| {scale:.3e} mV, "
          f"max error {np.max(np.abs(phi - rphi)):.2e} mV")
    assert scale > 0.0
    assert np.max(np.abs(phi - rphi)) <= 1e-5 * scale
