"""CPU tests of the library's host-side hierarchy builders (csrc/hierarchy.cpp) against the oracle.

The builders are compiled with the system C++ compiler through a small test shim (tests/host_shim.cpp)
and called with ctypes; no GPU is involved.  Each test converts what the library builds into matrices
and compares them with the oracle's element-by-element assembly and Galerkin products (Sec. 3.1's
multigrid ingredients): the stiffness stencil records, their Galerkin coarsening, the records of the
diagonal blocks M + sigma K, the Jacobi diagonals, the scaled Jacobi stencil of the finest-level
sweeps, the dense coarsest inverses, the monolithic point blocks and coupled coarse inverse, and the
3D Q1 class values with their dense coarsest inverse.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import fem, mg, rk
from oracle import tableaux as OT

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2403_08084_gb300", "csrc")

D_ = ctypes.POINTER(ctypes.c_double)


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("host") / "libhost_shim.so")
    cmd = [cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, os.path.join(ROOT, "tests", "host_shim.cpp"),
           os.path.join(CSRC, "hierarchy.cpp"), "-o", out, "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return ctypes.CDLL(out)


def ptr(a):
    return a.ctypes.data_as(D_)


def records(lib, N, kappa):
    out = np.empty((N + 1) ** 2 * 5)
    lib.shim_stiffness_records(N, ptr(kappa) if kappa is not None else None, ptr(out))
    return out


def coarsen(lib, Nf, cf):
    Nc = Nf // 2
    out = np.empty((Nc + 1) ** 2 * 5)
    lib.shim_galerkin_coarsen(Nf, ptr(cf), ptr(out))
    return out


def record_matrix(N, rec):
    """The full-grid matrix whose interior rows the records {D, E, N, NE, NW} describe: row p holds D_p,
    E_p at p + 1, E_{p-1} at p - 1, N_p at p + nx, N_{p-nx} at p - nx, NE_p at p + nx + 1, NE_{p-nx-1} at
    p - nx - 1, NW_p at p + nx - 1 and NW_{p-nx+1} at p - nx + 1; boundary rows are left empty."""
    nx = N + 1
    R = np.asarray(rec).reshape(nx * nx, 5)
    rows, cols, vals = [], [], []
    for iy in range(1, nx - 1):
        for ix in range(1, nx - 1):
            p = ix + nx * iy
            for q, v in ((p, R[p, 0]), (p + 1, R[p, 1]), (p - 1, R[p - 1, 1]), (p + nx, R[p, 2]),
                         (p - nx, R[p - nx, 2]), (p + nx + 1, R[p, 3]), (p - nx - 1, R[p - nx - 1, 3]),
                         (p + nx - 1, R[p, 4]), (p - nx + 1, R[p - nx + 1, 4])):
                rows.append(p), cols.append(q), vals.append(v)
    return sp.csr_matrix((vals, (rows, cols)), shape=(nx * nx, nx * nx))


def interior_block(N, A):
    ii = fem.interior_index(2, N)
    return A[ii][:, ii].toarray()


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


@pytest.mark.parametrize("with_kappa", [False, True])
def test_stiffness_records_match_element_assembly(lib, with_kappa):
    N = 12
    kap = W.lognormal_kappa(2, N, 0.5, seed=11) if with_kappa else None
    d = fem.Discretisation(2, N, kap)
    K = record_matrix(N, records(lib, N, kap))
    assert rel(interior_block(N, K), d.K.toarray()) < 1e-14


def test_galerkin_records_match_ptkp(lib):
    """Two coarsenings of the 32^2 records against the oracle's Galerkin products P^T K P."""
    N = 32
    kap = W.lognormal_kappa(2, N, 0.5, seed=12)
    d = fem.Discretisation(2, N, kap)
    h = mg.Hierarchy(d, 3)
    cf = records(lib, N, kap)
    for lev in (1, 2):
        cf = coarsen(lib, N >> (lev - 1), cf)
        Nl = N >> lev
        assert rel(interior_block(Nl, record_matrix(Nl, cf)), h.K[lev].toarray()) < 1e-13
        # the Galerkin mass of every level is the Q1 mass stencil of that level's spacing
        Ml, _ = fem.assemble(2, Nl)
        assert rel(interior_block(Nl, Ml), h.M[lev].toarray()) < 1e-13


def test_block_records_and_jacobi_diagonals(lib):
    N, s, omega = 16, 3, 2.0 / 3.0
    kap = W.lognormal_kappa(2, N, 0.5, seed=13)
    d = fem.Discretisation(2, N, kap)
    cf = records(lib, N, kap)
    hm = (1.0 / N) ** 2 / 36.0
    sigma = np.array([0.01, 0.2, 3.0])
    nn = (N + 1) ** 2
    rec = np.empty(nn * 5 * s)
    lib.shim_block_records(N, ptr(cf), ctypes.c_double(hm), ptr(sigma), s, ptr(rec))
    dinv = np.empty(nn * s)
    lib.shim_jacobi_inverse_diag(N, ptr(cf), ctypes.c_double(hm), ptr(sigma), s, ctypes.c_double(omega), ptr(dinv))
    ii = fem.interior_index(2, N)
    for i in range(s):
        B = (d.M + sigma[i] * d.K).toarray()
        Bi = interior_block(N, record_matrix(N, rec[i * nn * 5:(i + 1) * nn * 5]))
        assert rel(Bi, B) < 1e-14
        di = dinv.reshape(nn, s)[:, i]
        assert rel(di[ii], omega / np.diag(B)) < 1e-14
        assert np.all(np.delete(di, ii) == 0.0)


def test_scaled_jacobi_stencil_is_the_weighted_jacobi_sweep(lib):
    """x1 + sum_k c'_k x_k equals x + d (b - B x) with x1 = d b, for random x and b (zero boundary)."""
    N, omega, sig = 16, 2.0 / 3.0, np.array([0.05])
    kap = W.lognormal_kappa(2, N, 0.5, seed=14)
    d = fem.Discretisation(2, N, kap)
    cf = records(lib, N, kap)
    hm = (1.0 / N) ** 2 / 36.0
    nn = (N + 1) ** 2
    rec = np.empty(nn * 5)
    lib.shim_block_records(N, ptr(cf), ctypes.c_double(hm), ptr(sig), 1, ptr(rec))
    dinv = np.empty(nn)
    lib.shim_jacobi_inverse_diag(N, ptr(cf), ctypes.c_double(hm), ptr(sig), 1, ctypes.c_double(omega), ptr(dinv))
    srec = np.empty(9 * nn)
    lib.shim_scaled_jacobi_records(N, ptr(rec), ptr(dinv), ptr(srec))
    B = (d.M + sig[0] * d.K).toarray()
    ii = fem.interior_index(2, N)
    rng = np.random.default_rng(15)
    x, b = np.zeros(nn), np.zeros(nn)
    x[ii], b[ii] = rng.standard_normal(len(ii)), rng.standard_normal(len(ii))
    ref = x[ii] + dinv[ii] * (b[ii] - B @ x[ii])
    nx = N + 1
    offs = [0, 1, -1, nx, -nx, nx + 1, -nx - 1, nx - 1, -nx + 1]  # centre, E, W, N, S, NE, SW, NW, SE
    P = srec.reshape(9, nn)
    got = dinv[ii] * b[ii] + sum(P[k, ii] * x[ii + o] for k, o in enumerate(offs))
    assert rel(got, ref) < 1e-13
    # couplings to boundary nodes and the boundary rows are zero
    assert np.all(np.delete(P, ii, axis=1) == 0.0)


def test_dense_coarsest_inverse(lib):
    N, sigma = 8, 0.37
    kap = W.lognormal_kappa(2, N, 0.5, seed=16)
    d = fem.Discretisation(2, N, kap)
    cf = records(lib, N, kap)
    n = (N - 1) ** 2
    inv = np.empty(n * n)
    assert lib.shim_dense_block_inverse(N, ptr(cf), ctypes.c_double((1.0 / N) ** 2 / 36.0), ctypes.c_double(sigma),
                                        ptr(inv)) == 1
    B = (d.M + sigma * d.K).toarray()
    assert np.abs(inv.reshape(n, n) @ B - np.eye(n)).max() < 1e-12


def test_monolithic_point_blocks_and_coupled_coarse_inverse(lib):
    """omega (M_pp I + dt K_pp A)^{-1} per node, and the dense inverse of I (x) M + dt A (x) K with unknowns
    interleaved (row q s + i), against the oracle's Kronecker operator (Sec. 3, monolithic multigrid)."""
    N, dt, omega = 8, 1 / 16, 2.0 / 3.0
    A = OT.radau_iia(3).A
    s = A.shape[0]
    kap = W.lognormal_kappa(2, N, 0.5, seed=17)
    d = fem.Discretisation(2, N, kap)
    cf = records(lib, N, kap)
    hm = (1.0 / N) ** 2 / 36.0
    nn = (N + 1) ** 2
    Ac = np.ascontiguousarray(A)
    blk = np.empty(nn * s * s)
    assert lib.shim_mmg_block_inverses(N, ptr(cf), ctypes.c_double(hm), ptr(Ac), s, ctypes.c_double(dt),
                                       ctypes.c_double(omega), ptr(blk)) == 1
    ii = fem.interior_index(2, N)
    m, k = d.M.diagonal(), d.K.diagonal()
    D = blk.reshape(nn, s, s)
    for q, p in enumerate(ii):
        assert np.abs(D[p] @ (m[q] * np.eye(s) + dt * k[q] * A) - omega * np.eye(s)).max() < 1e-13
    n = len(ii)
    inv = np.empty((n * s) ** 2)
    assert lib.shim_mmg_coarse_inverse(N, ptr(cf), ctypes.c_double(hm), ptr(Ac), s, ctypes.c_double(dt),
                                       ptr(inv)) == 1
    S = rk.kronecker_operator(d.M, d.K, A, dt).toarray()  # stage-major: row i n + q
    perm = np.array([i * n + q for q in range(n) for i in range(s)])  # interleaved row q s + i
    Si = S[np.ix_(perm, perm)]
    assert np.abs(inv.reshape(n * s, n * s) @ Si - np.eye(n * s)).max() < 1e-11


def test_3d_q1_classes_and_coarsest_inverse(lib):
    """3D (kappa = 1): the 27-point Q1 mass and stiffness values by offset class (number of nonzero offset
    coordinates) against the oracle's assembly, and the dense inverse of M + sigma K on the interior."""
    N, sigma = 4, 0.8
    h = 1.0 / N
    mass, stiff = np.empty(4), np.empty(4)
    lib.shim_q1_classes_3d(ctypes.c_double(h), ptr(mass), ptr(stiff))
    Mf, Kf = fem.assemble(3, N)
    nx = N + 1
    p = 2 + nx * (2 + nx * 2)  # the centre node: all 26 neighbours interior
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                q = p + dx + nx * (dy + nx * dz)
                cls = abs(dx) + abs(dy) + abs(dz)
                assert abs(Mf[p, q] - mass[cls]) <= 1e-15 * abs(mass[0])
                assert abs(Kf[p, q] - stiff[cls]) <= 1e-14 * abs(stiff[0])
    n = (N - 1) ** 3
    inv = np.empty(n * n)
    assert lib.shim_dense_block_inverse_3d(N, ptr(mass), ptr(stiff), ctypes.c_double(sigma), ptr(inv)) == 1
    d = fem.Discretisation(3, N)
    B = (d.M + sigma * d.K).toarray()
    assert np.abs(inv.reshape(n, n) @ B - np.eye(n)).max() < 1e-12
