"""Host logic of the partitioned tridiagonal solve, on the CPU.

The library builds the coefficient tables of the Crank-Nicolson solve
(eq:lumping_crank_nicolson_2 with lumped linear elements and Neumann ends)
on the host.  This test takes those tables through the C ABI, runs the steps
the step kernel runs with them (chunk elimination, reduced system, PCR
levels, recovery) in FP64 with numpy, and compares the result with a direct
banded solve of the same system (scipy).  A wrong table entry, a wrong PCR
level count or a wrong truncation shows up as a solve error."""
import numpy as np
import pytest

from paper_2107_07104_gb300 import fibers as F

linalg = pytest.importorskip("scipy.linalg")


@pytest.fixture(scope="module", autouse=True)
def lib():
    try:
        return F.load()
    except OSError as e:  # the library is built by build()
        pytest.skip(f"library not built: {e}")


def cn_rhs(u, r):
    """(I + dt/2 L) u for the lumped Neumann operator: rows (1 - r, r),
    (r/2, 1 - r, r/2), (r, 1 - r)."""
    N = u.size
    if N == 1:
        return u.copy()
    d = (1 - r) * u
    d[1:-1] += 0.5 * r * (u[:-2] + u[2:])
    d[0] += r * u[1]
    d[-1] += r * u[-2]
    return d


def direct_solve(u, r):
    """Banded solve of (I - dt/2 L) x = (I + dt/2 L) u."""
    N = u.size
    if N == 1:
        return u.copy()
    ab = np.zeros((3, N))
    ab[1] = 1 + r
    ab[0, 1:] = -0.5 * r
    ab[2, :-1] = -0.5 * r
    ab[0, 1] = -r      # row 0: (1 + r, -r)
    ab[2, N - 2] = -r  # row N-1: (-r, 1 + r)
    return linalg.solve_banded((1, 1), ab, cn_rhs(u, r))


def partitioned_solve(u, r, K, tab):
    """The kernel's solve, step for step, in FP64 with the library's tables."""
    N = u.size
    r = r if N > 1 else 0.0
    Tw, L = tab["threads"], tab["levels"]
    rows, rec = tab["rows"], tab["recs"]
    Tf = (N + K - 1) // K
    U = np.zeros(Tw * K)
    U[:N] = u
    # right-hand side per node, with the ghost values the kernel uses at the
    # ends (u(-1) = u(1), u(N) = u(N-2)) and zero rows past the fiber
    um = np.concatenate([[U[1]], U[:-1]])
    up = np.concatenate([U[1:], [0.0]])
    if N > 1:
        up[N - 1] = um[N - 1]
    d = (1 - r) * U + 0.5 * r * (um + up)
    d[N:] = 0.0
    d = d.reshape(Tw, K)
    S = np.broadcast_to(rows[0], (Tw, K, 5)).copy()
    S[Tf - 1] = rows[1]
    # elimination inside every chunk
    d[:, 1] = d[:, 1] * S[:, 1, 0]
    for j in range(2, K):
        d[:, j] = d[:, j] * S[:, j, 0] - S[:, j, 1] * d[:, j - 1]
    for j in range(K - 3, 0, -1):
        d[:, j] = d[:, j] - S[:, j, 2] * d[:, j + 1]
    D = d[:, 0] - rec[:, 3] * d[:, 1]
    E = d[:, K - 1].copy()
    Dn = np.concatenate([D[1:], [0.0]])
    y = E * rec[:, 4] - rec[:, 5] * D - rec[:, 6] * Dn
    # parallel cyclic reduction over the chunks' last unknowns
    for level in range(L):
        st = 1 << level
        ym_ = np.concatenate([np.zeros(st), y[:-st]]) if st < Tw else np.zeros(Tw)
        yp_ = np.concatenate([y[st:], np.zeros(st)]) if st < Tw else np.zeros(Tw)
        lv = rec[:, 7 + 3 * level:10 + 3 * level]
        y = y * lv[:, 0] - lv[:, 1] * ym_ - lv[:, 2] * yp_
    ym = np.concatenate([[0.0], y[:-1]])
    xs = D * rec[:, 0] - rec[:, 1] * ym - rec[:, 2] * y
    out = np.empty((Tw, K))
    out[:, 0] = xs
    out[:, K - 1] = y
    for j in range(1, K - 1):
        out[:, j] = d[:, j] - S[:, j, 3] * xs - S[:, j, 4] * y
    return out.ravel()[:N]


def lengths_for(K):
    top = 256 * K  # 8 warps of K-node threads
    return sorted({1, 2, 3, 5, K - 1, K, K + 1, 2 * K + 3, 33, 100, 1481 if 1481 <= top else top - 7, top})


CASES = [(K, N, r) for K in (4, 8, 12, 16) for N in lengths_for(K) for r in (0.11484, 0.22968, 1.84, 10.0)]


@pytest.mark.parametrize("fp64", [False, True], ids=["fp32-cutoff", "fp64-cutoff"])
def test_partitioned_solve_matches_a_banded_solve(fp64):
    rng = np.random.default_rng(7)
    tol = 2e-11 if fp64 else 1e-9  # cutoffs 2^-40 and 2^-32, times the fiber's largest |u|
    worst = 0.0
    for K, N, r in CASES:
        tab = F.fibers_solver_tables(K, r if N > 1 else 0.0, N, fp64)
        chunks = -(-N // K)
        assert tab["threads"] == 32 * -(-chunks // 32)  # whole warps of K-node chunks
        u = rng.normal(0.0, 50.0, N)
        got = partitioned_solve(u, r, K, tab)
        ref = direct_solve(u, r if N > 1 else 0.0)
        err = np.max(np.abs(got - ref)) / np.max(np.abs(u))
        worst = max(worst, err)
        assert err <= tol, (K, N, r, tab["levels"], err)
    print(f"[solver tables] worst relative error {worst:.2e} over {len(CASES)} cases")


def test_pcr_levels_follow_the_cutoff():
    # The bundle's shape (K = 8, 1481 nodes, r = c dt_1D / h^2 = 0.11484):
    # the coupling left after chunk elimination is about 1e-10, between the
    # two cutoffs, so the FP32 solve keeps no PCR level and the FP64 solve one.
    assert F.fibers_solver_tables(8, 0.11484, 1481, False)["levels"] == 0
    assert F.fibers_solver_tables(8, 0.11484, 1481, True)["levels"] == 1
    # larger r couples chunks more strongly: more levels, never fewer
    prev = 0
    for r in (0.46, 1.84, 10.0, 100.0):
        lv = F.fibers_solver_tables(8, r, 1481, False)["levels"]
        assert lv >= prev
        prev = lv
    assert prev >= 3
    # a single chunk needs no reduction at all
    assert F.fibers_solver_tables(16, 10.0, 10, True)["levels"] == 0


def test_dropping_the_kept_levels_breaks_the_solve():
    # the levels the library keeps are needed: without them the solve is off
    K, N, r = 8, 1481, 10.0
    tab = F.fibers_solver_tables(K, r, N, False)
    assert tab["levels"] > 0
    u = np.random.default_rng(8).normal(0.0, 50.0, N)
    trunc = dict(tab, levels=0)
    err = np.max(np.abs(partitioned_solve(u, r, K, trunc) - direct_solve(u, r))) / np.max(np.abs(u))
    assert err > 1e-3


@pytest.mark.parametrize("args", [(5, 0.1, 100, 0), (8, 0.1, 0, 0), (8, 0.1, 2049, 0), (16, 0.1, 2**31 - 1, 0),
                                  (8, -1.0, 10, 0), (8, float("nan"), 10, 0), (8, float("inf"), 10, 1)])
def test_solver_tables_reject_bad_arguments(args):
    with pytest.raises(F.FibersError) as ei:
        F.fibers_solver_tables(*args)
    assert ei.value.status == F.FIB_EINVAL
