"""The library's host-side set-up (csrc/setup.cpp), compiled with g++ alone
and run on the CPU, against the oracle: the canonical mesh (Sec. 3), the
truncated Chebyshev coefficients of e^{tL} (Sec. 2.4) with the widest
exponential the library accepts, and the Riemann-sum shifts and weights
(Sec. 2.2).  The GPU tests reach the same code only through a context."""

import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import averaging, expo
from oracle.mesh import build_mesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
R = 6.37122e6


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = tmp_path_factory.mktemp("host_setup") / "harness"
    csrc = os.path.join(ROOT, "paper_2103_07706_gb300", "csrc")
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", os.path.join(ROOT, "include"), "-I", csrc,
                    os.path.join(ROOT, "tests", "host_setup_harness.cpp"), os.path.join(csrc, "setup.cpp"),
                    os.path.join(csrc, "sd_setup.cpp"),
                    "-o", str(exe)], check=True)
    return exe


def run(exe, *args):
    out = subprocess.run([str(exe), *map(str, args)], check=True, capture_output=True, text=True).stdout
    return out.strip().split("\n")


@pytest.mark.parametrize("r", [0, 1, 2, 3, 4, 5])
def test_mesh_matches_oracle(harness, tmp_path, r):
    V, F, E = map(int, run(harness, "mesh", r, repr(R), tmp_path / "m")[0].split())
    assert (F, E, V) == (20 * 4 ** r, 30 * 4 ** r, 10 * 4 ** r + 2)
    verts = np.fromfile(tmp_path / "m.verts", dtype=np.float64).reshape(V, 3)
    cells = np.fromfile(tmp_path / "m.cells", dtype=np.int32).reshape(F, 3)
    o = build_mesh(r, R)
    assert np.array_equal(cells, o.cells)
    assert np.abs(verts - o.verts).max() <= 1e-15 * R


@pytest.mark.parametrize("Lb", [0.0, 0.5, 3.0, 42.0, 168.0])
def test_chebyshev_coefficients_match_oracle(harness, Lb):
    out = run(harness, "cheb", repr(Lb), "1e-6")
    c = np.array([float(x) for x in out[1:1 + int(out[0])]])
    want = expo.truncated_coefficients(Lb, 1.0, 1e-6)  # lambda_max |t| = Lb
    assert len(c) == len(want)
    assert np.abs(c - want).max() <= 1e-13


@pytest.mark.parametrize("Lb", ["16384.5", "1e300", "inf", "nan", "-1"])
def test_exponentials_beyond_the_limit_are_refused(harness, Lb):
    """lambda_max |t| above 16384 (PAVG_MAX_CHEB_ARG), not finite or negative:
    an empty list, which the entry points turn into PAVG_ERR_INVAL before
    the O(N^2) transform would run."""
    assert run(harness, "cheb", Lb, "1e-6") == ["0"]


@pytest.mark.parametrize("T,M,rule", [(3600.0, 8, 0), (3600.0, 5, 0), (7200.0, 7, 1), (14400.0, 128, 0),
                                      (0.0, 4, 0), (0.0, 1, 0)])
def test_shifts_and_weights_match_oracle(harness, T, M, rule):
    """Including T = 0: every shift 0, equal weights (the average is N)."""
    out = run(harness, "shifts", repr(T), M, rule)
    assert out[0] == "0"
    sw = np.array([[float(v) for v in line.split()] for line in out[1:]])
    s, w = averaging.shifts_and_weights(T, M, rule)
    assert sw.shape == (M, 2)
    assert np.abs(sw[:, 0] - s).max() <= 1e-12 * max(T, 1.0)
    assert np.abs(sw[:, 1] - w).max() <= 1e-15


@pytest.mark.parametrize("T,M,rule", [(3600.0, 4, 1), (3600.0, 1, 1), (3600.0, 0, 0), (3600.0, 3, 7),
                                      (-1.0, 4, 0), (float("inf"), 4, 0), (float("nan"), 4, 0)])
def test_invalid_point_sets_are_refused(harness, T, M, rule):
    """The closed rule needs an odd M >= 3; M >= 1; the rule must exist; the
    window must be finite and non-negative."""
    assert run(harness, "shifts", repr(T), M, rule)[0] != "0"


@pytest.mark.parametrize("r", [1, 2])
def test_element_matrices_assemble_to_the_oracles(harness, tmp_path, r):
    """The signed, packed element matrices of M1 and C (Sec. 2.5) that the
    kernels read, placed at their global DOFs, sum to the oracle's global
    matrices; det and the metric G = J^T J match per cell.  A wrong sign on reversed edges, a transposed or negated
    Coriolis matrix, or a mis-packed triangle gives O(1) differences."""
    import scipy.sparse as sp

    from oracle.assembly import Assembly
    omega = 7.292e-5
    n, F = map(int, run(harness, "cells", r, repr(R), repr(omega), tmp_path / "c")[0].split())

    def load(k):
        rows = np.fromfile(tmp_path / f"c.{k}.row", dtype=np.int64)
        cols = np.fromfile(tmp_path / f"c.{k}.col", dtype=np.int64)
        vals = np.fromfile(tmp_path / f"c.{k}.val", dtype=np.float64)
        return sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()

    asm = Assembly(build_mesh(r, R), omega, R)
    M1, C, _, _ = asm.global_matrices()
    assert M1.shape == (n, n) and F == 20 * 4 ** r
    assert abs(load("m1") - M1).max() <= 1e-13 * abs(M1).max()
    assert abs(load("c") - C).max() <= 1e-12 * abs(C).max()
    assert np.abs(np.fromfile(tmp_path / "c.det", dtype=np.float64) - asm.det).max() <= 1e-14 * asm.det.max()
    G = np.fromfile(tmp_path / "c.g", dtype=np.float64).reshape(3, F)
    want = np.stack([asm.G[:, 0, 0], asm.G[:, 0, 1], asm.G[:, 1, 1]])
    assert np.abs(G - want).max() <= 1e-14 * np.abs(want).max()
    assert np.abs(asm.G[:, 0, 1] - asm.G[:, 1, 0]).max() == 0.0


def test_stroud_rule_matches_the_oracle(harness):
    """The library's 5 x 5 Stroud rule (Gauss-Jacobi nodes by bracketing and
    bisection) against the oracle's (scipy's Gauss-Jacobi), point by point in
    the same order."""
    from oracle.quadrature import triangle_rule
    got = np.array([list(map(float, line.split())) for line in run(harness, "stroud", 5)])
    xq, wq = triangle_rule(5)
    assert got.shape == (25, 3)
    assert np.abs(got[:, :2] - xq).max() <= 2e-16 and np.abs(got[:, 2] - wq).max() <= 1e-16


@pytest.mark.parametrize("r", [0, 1, 2, 3])
def test_cubic_cell_data_match_oracle(harness, tmp_path, r):
    """Element matrices and per-point metric of the piecewise cubic surface
    (Sec. 3): the library's cubic map (closed-form barycentric basis) against
    the oracle's (inverted Vandermonde over monomials)."""
    import scipy.sparse as sp

    from oracle.assembly import Assembly
    from oracle.elements import EDGE_DIR, EDGE_START
    from oracle.quadrature import gauss_legendre_01, triangle_rule
    omega = 7.292e-5
    n, F = map(int, run(harness, "cells", r, repr(R), repr(omega), tmp_path / "c", 3)[0].split())

    def load(k):
        rows = np.fromfile(tmp_path / f"c.{k}.row", dtype=np.int64)
        cols = np.fromfile(tmp_path / f"c.{k}.col", dtype=np.int64)
        vals = np.fromfile(tmp_path / f"c.{k}.val", dtype=np.float64)
        return sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()

    mesh = build_mesh(r, R)
    asm = Assembly(mesh, omega, R, geometry_degree=3)
    M1, C, _, M2 = asm.global_matrices()
    assert abs(load("m1") - M1).max() <= 1e-13 * abs(M1).max()
    assert abs(load("c") - C).max() <= 1e-12 * abs(C).max()
    pk = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    m2e = np.fromfile(tmp_path / "c.m2e", dtype=np.float64).reshape(6, F)
    m2i = np.fromfile(tmp_path / "c.m2i", dtype=np.float64).reshape(6, F)
    want = np.stack([asm.M2_e[:, a, b] for a, b in pk])
    assert np.abs(m2e - want).max() <= 1e-13 * np.abs(want).max()
    inv = np.linalg.inv(asm.M2_e)
    wanti = np.stack([inv[:, a, b] for a, b in pk])
    assert np.abs(m2i - wanti).max() <= 1e-11 * np.abs(wanti).max()
    # per cell point: G, w / det^2, grad det / det at the Stroud points
    xq, wq = triangle_rule(5)
    g = asm.maps.geometry(xq)
    geoc = np.fromfile(tmp_path / "c.geoc", dtype=np.float64).reshape(6, 25, F)
    wantc = np.stack([g["G"][..., 0, 0], g["G"][..., 0, 1], g["G"][..., 1, 1], wq[None, :] / g["det"] ** 2,
                      g["grad_det"][..., 0] / g["det"], g["grad_det"][..., 1] / g["det"]]).transpose(0, 2, 1)
    for k in range(4):
        assert np.abs(geoc[k] - wantc[k]).max() <= 1e-12 * np.abs(wantc[k]).max(), k
    # d ln det / d xi: a small difference of second-derivative products (the
    # cell's curvature); both sides round it at the scale of the metric's
    # unit-size reference terms
    for k in (4, 5):
        assert np.abs(geoc[k] - wantc[k]).max() <= 1e-12, k
    # per facet point: each side's G and det at its own parameter
    E = mesh.n_edges
    tau, _ = gauss_legendre_01(5)
    geof = np.fromfile(tmp_path / "c.geof", dtype=np.float64).reshape(8, 5, E)
    for side, t in ((0, tau), (1, 1.0 - tau)):
        cells, loc = mesh.edge_cells[:, side], mesh.edge_local[:, side]
        gs = [asm.maps.geometry(EDGE_START[i][None, :] + t[:, None] * EDGE_DIR[i][None, :]) for i in range(3)]
        G = np.stack([x["G"] for x in gs])[loc, cells]           # (E, 5, 2, 2)
        det = np.stack([x["det"] for x in gs])[loc, cells]
        for k, v in enumerate([G[..., 0, 0], G[..., 0, 1], G[..., 1, 1], 1.0 / det]):
            assert np.abs(geof[4 * side + k] - v.T).max() <= 1e-12 * np.abs(v).max(), (side, k)


def test_reference_tables_match_the_oracle(harness):
    """The constant-memory tables the kernels scale per cell: D-hat (the
    oracle's D_e with its orientation signs divided out, the same for every
    cell under the Piola map) and the DG1 mass M2-hat = (1 + delta_ij) / 24
    of the reference triangle, with its inverse."""
    from oracle.assembly import Assembly
    rows = [list(map(float, line.split())) for line in run(harness, "tables")]
    D, M2, M2inv = np.array(rows[:3]), np.array(rows[3:6]), np.array(rows[6:9])
    asm = Assembly(build_mesh(1, R), 7.292e-5, R)
    Dref = asm.D_e / asm.sign[:, None, :]
    assert np.abs(Dref - D[None]).max() <= 1e-13
    assert np.abs(M2 - (np.ones((3, 3)) + np.eye(3)) / 24.0).max() <= 1e-15
    assert np.abs(asm.M2_e / asm.det[:, None, None] - M2[None]).max() <= 1e-15
    assert np.abs(M2inv @ M2 - np.eye(3)).max() <= 1e-13


def test_solver_and_facet_setup(harness, tmp_path):
    """Set-up data of the mixed M1 solver and the facet kernels at r2 against
    the oracle.  Edge incidence: plus cell = the one running the edge
    low -> high, with local indices.  DOF triples: a cell's three edges and
    its interior, each triple owned by exactly one cell.  Preconditioner:
    FP32 inverses of M1's 3x3 diagonal blocks.  Jacobi diagonal.  The FP32
    matrix copies in both layouts are roundings of the FP64 element
    matrices."""
    from oracle.assembly import Assembly
    r = 2
    E, F = map(int, run(harness, "solver", r, repr(R), tmp_path / "s")[0].split())
    ld = lambda k, dt: np.fromfile(tmp_path / f"s.{k}", dtype=dt)  # noqa: E731
    mesh = build_mesh(r, R)
    # edge incidence
    assert np.array_equal(ld("eplus", np.int32), mesh.edge_cells[:, 0])
    assert np.array_equal(ld("eminus", np.int32), mesh.edge_cells[:, 1])
    lpos = ld("elpos", np.uint8).astype(np.int64)
    assert np.array_equal(lpos & 3, mesh.edge_local[:, 0]) and np.array_equal((lpos >> 2) & 3, mesh.edge_local[:, 1])
    # DOF triples and owners
    tri = ld("tri", np.int32).view(np.uint32).reshape(F, 4).astype(np.int64)
    idx, own = tri & 0x7FFFFFFF, tri >> 31
    assert np.array_equal(idx[:, :3], mesh.cell_edges) and np.array_equal(idx[:, 3], E + np.arange(F))
    assert np.array_equal(own[:, :3].astype(bool), mesh.cell_edge_aligned) and own[:, 3].all()
    assert np.array_equal(np.bincount(idx[own == 1], minlength=E + F), np.ones(E + F, dtype=np.int64))
    # preconditioner blocks and Jacobi diagonal against the oracle's M1
    M1 = Assembly(mesh, 7.292e-5, R).global_matrices()[0].toarray()
    P = ld("pinv", np.float32).reshape(E + F, 8).astype(np.float64)
    sym = np.array([[0, 1, 2], [1, 3, 4], [2, 4, 5]])
    for t in range(E + F):
        blk = M1[3 * t:3 * t + 3, 3 * t:3 * t + 3]
        assert np.abs(P[t][sym] @ blk - np.eye(3)).max() <= 1e-5
    assert np.abs(ld("dinv", np.float64) * np.diag(M1) - 1.0).max() <= 1e-14
    # FP32 copies: packed [78][F] and row blocks [36][F][4]
    m1 = ld("m1", np.float64)
    assert np.array_equal(ld("m1p", np.float32), m1.astype(np.float32))
    m1 = m1.reshape(78, F)
    full = np.zeros((F, 12, 12))
    k = 0
    for i in range(12):
        for j in range(i, 12):
            full[:, i, j] = full[:, j, i] = m1[k]
            k += 1
    m1f = ld("m1f", np.float32).reshape(36, F, 4)
    e = np.arange(36)
    for q in range(4):
        want = full[:, 3 * q + e // 12, e % 12].T.astype(np.float32)  # (36, F)
        assert np.array_equal(m1f[:, :, q], want)


def test_reference_basis_matches_the_oracle(harness):
    """The library's BDM2 basis (values and derivatives at any reference point)
    equals the oracle's: the same degrees of freedom fix the same basis."""
    from oracle.elements import BDM2
    rng = np.random.default_rng(11)
    pts = rng.random((16, 2))
    pts = np.where(pts.sum(1, keepdims=True) > 1, 1 - pts, pts)
    out = run(harness, "element", *[f"{v:.17g}" for v in pts.ravel()])
    el = BDM2()
    want_v, want_g = el.values(pts), el.grads(pts)
    for q in range(len(pts)):
        v = np.array(out[2 * q].split(), dtype=np.float64).reshape(12, 2)
        g = np.array(out[2 * q + 1].split(), dtype=np.float64).reshape(12, 2, 2)
        assert np.abs(v - want_v[q]).max() <= 1e-12
        assert np.abs(g - want_g[q]).max() <= 1e-11


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 8])
def test_gauss_legendre_on_unit_interval(harness, n):
    from scipy.special import roots_legendre
    xw = np.array([line.split() for line in run(harness, "gauss", n)], dtype=np.float64)
    x, w = roots_legendre(n)
    assert np.abs(xw[:, 0] - (x + 1) / 2).max() <= 1e-15
    assert np.abs(xw[:, 1] - w / 2).max() <= 1e-15


def test_cell_rule_of_the_nonlinear_kernels_is_degree_five(harness):
    """Every integrand of N on a flat cell has degree <= 5, so the 7-point rule
    must integrate x^a y^b exactly over the reference triangle for a + b <= 5:
    a! b! / (a + b + 2)!."""
    from math import factorial
    rows = np.array([line.split() for line in run(harness, "cellrule")], dtype=np.float64)
    w, phi = rows[:, 0], rows[:, 1:]
    assert np.abs(phi.sum(1) - 1).max() <= 1e-15
    x, y = phi[:, 1], phi[:, 2]
    for a in range(6):
        for b in range(6 - a):
            want = factorial(a) * factorial(b) / factorial(a + b + 2)
            assert abs(np.sum(w * x ** a * y ** b) - want) <= 1e-15


def test_nonlinear_kernel_tables_match_the_oracle(harness):
    """The constant tables of the nonlinear kernels are the reference basis
    sampled where the oracle samples it (Sec. 2.5).  That means the 7 cell
    points and the 4 Gauss points of each local edge: the + side at tau,
    the - side at 1 - tau (each side runs the edge its own way).  Also the
    edge directions and the basis divergences at the reference vertices."""
    from oracle.elements import BDM2, EDGE_DIR, EDGE_START, dg1_values
    from oracle.quadrature import gauss_legendre_01
    lines = run(harness, "ntables")
    arr = [np.array(line.split(), dtype=np.float64) for line in lines]
    cq_psi, cq_dpsi, fq_w, fq_psi, fq_phi, edge_dir, div_vert = arr
    rule = np.array([line.split() for line in run(harness, "cellrule")], dtype=np.float64)
    xq = rule[:, 2:4]
    el = BDM2()
    assert np.abs(cq_psi.reshape(7, 12, 2) - el.values(xq)).max() <= 1e-12
    assert np.abs(cq_dpsi.reshape(7, 12, 2, 2) - el.grads(xq)).max() <= 1e-11
    tau, wt = gauss_legendre_01(4)
    assert np.abs(fq_w - wt).max() <= 1e-15
    fq_psi, fq_phi = fq_psi.reshape(2, 3, 4, 12, 2), fq_phi.reshape(2, 3, 4, 3)
    for e in range(3):
        for side, t in ((0, tau), (1, 1.0 - tau)):
            x = EDGE_START[e][None, :] + t[:, None] * EDGE_DIR[e][None, :]
            assert np.abs(fq_psi[side, e] - el.values(x)).max() <= 1e-12
            assert np.abs(fq_phi[side, e] - dg1_values(x)).max() <= 1e-15
    assert np.array_equal(edge_dir.reshape(3, 2), EDGE_DIR)
    verts = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    assert np.abs(div_vert.reshape(12, 3) - el.divs(verts).T).max() <= 1e-11


def _read(path, dtype):
    return np.fromfile(path, dtype=dtype)


@pytest.mark.parametrize("r,P", [(2, 10), (3, 40), (4, 152), (5, 152)])
def test_subdomain_partition_reproduces_the_global_product(harness, tmp_path, r, P):
    """The subdomain solver's data flow, replayed on the CPU from the set-up
    data the kernel reads: every part multiplies its cells' element matrices
    into per-(cell, q) slots, each local triple adds its local slots and, when
    it is shared, the partner part's contribution read from the partner's send
    slot.  Every part's copy of every triple must equal the assembled M1 x,
    each triple must have exactly one owner, and at most two cells."""
    E, F = map(int, run(harness, "solver", r, repr(R), tmp_path / "s")[0].split())
    nslots, max_cells, max_lt, max_shared = map(int, run(harness, "partition", r, repr(R), P, tmp_path / "p")[0].split())
    tri = _read(tmp_path / "s.tri", np.int32).reshape(F, 4) & 0x7fffffff
    m1 = _read(tmp_path / "s.m1", np.float64).reshape(78, F)
    cell0, lt0 = _read(tmp_path / "p.cell0", np.int32), _read(tmp_path / "p.lt0", np.int32)
    gtri, slot = _read(tmp_path / "p.gtri", np.uint32), _read(tmp_path / "p.slot", np.uint32)
    recv = _read(tmp_path / "p.recv", np.int32)
    celllt = _read(tmp_path / "p.celllt", np.int32).reshape(F, 4)
    cellsend = _read(tmp_path / "p.cellsend", np.int32).reshape(F, 4)
    assert len(cell0) == P + 1 and cell0[0] == 0 and cell0[-1] == F
    assert max_cells == np.diff(cell0).max() and max_lt == np.diff(lt0).max()
    T = E + F
    # full 12 x 12 element matrices and the global product
    iu = np.triu_indices(12)
    A = np.zeros((F, 12, 12))
    A[:, iu[0], iu[1]] = m1.T
    A = A + np.transpose(A, (0, 2, 1)) - A * np.eye(12)[None]
    x = np.random.default_rng(1).standard_normal((T, 3))
    y_loc = np.einsum("fij,fj->fi", A, x[tri].reshape(F, 12)).reshape(F, 4, 3)
    want = np.zeros((T, 3))
    np.add.at(want, tri.ravel(), y_loc.reshape(-1, 3))
    # send buffer: contribution of (cell, q) at its send slot
    send = np.full((nslots, 3), np.nan)
    for c, q in zip(*np.nonzero(cellsend >= 0)):
        send[cellsend[c, q]] = y_loc[c, q]
    assert not np.isnan(send).any()
    owners = np.zeros(T, dtype=int)
    for p in range(P):
        c0, c1 = cell0[p], cell0[p + 1]
        for i in range(lt0[p], lt0[p + 1]):
            t = gtri[i] & 0x7fffffff
            owners[t] += gtri[i] >> 31
            s0, s1 = slot[i] & 0xffff, slot[i] >> 16
            assert s0 != 0xffff
            got = y_loc[c0 + s0 // 4, s0 % 4].copy()
            assert tri[c0 + s0 // 4, s0 % 4] == t and celllt[c0 + s0 // 4, s0 % 4] == i - lt0[p]
            if s1 != 0xffff:
                assert tri[c0 + s1 // 4, s1 % 4] == t and recv[i] == -1
                got += y_loc[c0 + s1 // 4, s1 % 4]
            elif recv[i] >= 0:
                got += send[recv[i]]
            assert np.abs(got - want[t]).max() <= 1e-14 * np.abs(want).max()
        assert (celllt[c0:c1] < lt0[p + 1] - lt0[p]).all()
    assert (owners == 1).all()
    assert nslots == 2 * (recv >= 0).sum() // 2 and (recv >= 0).sum() == nslots
    assert max_shared <= max_lt


def test_subdomain_spectrum_and_iteration_count(harness, tmp_path):
    """Preconditioned Lanczos bounds of P M1 against its dense eigenvalues
    (refinement 2), and the Chebyshev iteration count against the polynomial's
    closed-form error bound 2 / (c^k + c^-k)."""
    E, F = map(int, run(harness, "solver", 2, repr(R), tmp_path / "s")[0].split())
    lo, hi = map(float, run(harness, "spectrum", 2, repr(R), 40)[0].split())
    tri = _read(tmp_path / "s.tri", np.int32).reshape(F, 4) & 0x7fffffff
    m1 = _read(tmp_path / "s.m1", np.float64).reshape(78, F)
    pinv = _read(tmp_path / "s.pinv", np.float32).reshape(E + F, 8).astype(np.float64)
    n = 3 * (E + F)
    iu = np.triu_indices(12)
    A = np.zeros((F, 12, 12))
    A[:, iu[0], iu[1]] = m1.T
    A = A + np.transpose(A, (0, 2, 1)) - A * np.eye(12)[None]
    dofs = (3 * tri[:, :, None] + np.arange(3)).reshape(F, 12)
    M = np.zeros((n, n))
    np.add.at(M, (np.repeat(dofs, 12, axis=1).ravel(), np.tile(dofs, (1, 12)).ravel()), A.reshape(F, -1).ravel())
    Pm = np.zeros((n, n))
    idx = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    for t in range(E + F):
        for k, (a, b) in enumerate(idx):
            Pm[3 * t + a, 3 * t + b] = Pm[3 * t + b, 3 * t + a] = pinv[t, k]
    ev = np.sort(np.linalg.eigvals(Pm @ M).real)
    assert ev[0] <= lo <= ev[0] * 1.01 and ev[-1] * 0.99 <= hi <= ev[-1], (lo, hi, ev[0], ev[-1])
    a, b = 0.95 * lo, 1.05 * hi
    k = int(run(harness, "chebits", a, b, 1e-5)[0])
    c = (np.sqrt(b / a) + 1) / (np.sqrt(b / a) - 1)
    bound = lambda j: 2 / (c ** j + c ** -j)  # noqa: E731
    assert bound(k) <= 1e-5 < bound(k - 1)
