"""Pins for the oracle's Q1 assembly (Sec. 2 eq. heat / rkheat)."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import fem
from oracle import manufactured as mf


def test_element_matrices_2d_textbook():
    """Bilinear square element: K_e = [[4,-1,-1,-2],...]/6 (h-independent), M_e = h^2/36 [[4,2,2,1],...]."""
    for h in (1.0, 0.25):
        Me, Ke = fem.element_matrices(2, h)
        Kt = np.array([[4, -1, -1, -2], [-1, 4, -2, -1], [-1, -2, 4, -1], [-2, -1, -1, 4]]) / 6
        Mt = h * h / 36 * np.array([[4, 2, 2, 1], [2, 4, 1, 2], [2, 1, 4, 2], [1, 2, 2, 4]])
        assert np.allclose(Ke, Kt, atol=1e-15) and np.allclose(Me, Mt, atol=1e-16)


@pytest.mark.parametrize("dim", [2, 3])
def test_element_matrices_tensor_structure(dim):
    """Q1 element matrices are Kronecker products of the 1D linear-element ones."""
    h = 0.3
    M1 = h / 6 * np.array([[2, 1], [1, 2]])
    K1 = 1 / h * np.array([[1, -1], [-1, 1]])
    Me, Ke = fem.element_matrices(dim, h)

    def kron_list(ms):
        out = ms[0]
        for m in ms[1:]:
            out = np.kron(m, out)  # later (slower) axes on the left: x fastest
        return out

    Mt = kron_list([M1] * dim)
    Kt = sum(kron_list([K1 if a == d else M1 for a in range(dim)]) for d in range(dim))
    assert np.allclose(Me, Mt, atol=1e-15) and np.allclose(Ke, Kt, atol=1e-14)


@pytest.mark.parametrize("dim,N", [(2, 5), (3, 3)])
def test_assembly_exact_integrals(dim, N):
    """u = prod x_d is in the Q1 space: u^T M u = 3^-dim, u^T K u = dim 3^-(dim-1);
    sum(M) = volume, K 1 = 0."""
    M, K = fem.assemble(dim, N)
    xs = W.node_coords(dim, N)
    u = np.prod(np.stack(xs), axis=0)
    assert math.isclose(u @ (M @ u), 3.0**-dim, rel_tol=1e-13)
    assert math.isclose(u @ (K @ u), dim * 3.0 ** -(dim - 1), rel_tol=1e-13)
    assert math.isclose(M.sum(), 1.0, rel_tol=1e-13)
    assert np.abs(K @ np.ones(K.shape[0])).max() < 1e-13
    assert abs(K - K.T).max() < 1e-15


def _row_sums(K):
    """Exact sums (math.fsum) of the stored entries of every row."""
    K = K.tocsr()
    return np.array([math.fsum(K.data[K.indptr[i]:K.indptr[i + 1]]) for i in range(K.shape[0])])


@pytest.mark.parametrize("dim,N", [(2, 16), (2, 64), (3, 8)])
def test_stiffness_rows_sum_to_zero_exactly(dim, N):
    """The gradient of a constant vanishes, so every interior row of K sums to zero.  For kappa = 1 and h a
    power of two the stored entries must satisfy it exactly: a same-sign rounding bias in the row sums acts
    like a small reaction term, which the stiff stage systems amplify (the stiffness stencil applied to a
    smooth state cancels by a factor of order h^2)."""
    _, K = fem.assemble(dim, N)
    rs = _row_sums(K)[fem.interior_index(dim, N)]
    assert np.all(rs == 0.0)


def test_stiffness_row_sums_unbiased_for_variable_kappa():
    """With per-cell lognormal kappa the entries round independently: interior row sums average to zero
    (relative to the diagonal) far below one rounding unit, with no systematic sign."""
    N = 128
    kap = W.lognormal_kappa(2, N, 0.5, 3)
    _, K = fem.assemble(2, N, kap)
    ii = fem.interior_index(2, N)
    rs, D = _row_sums(K)[ii], K.diagonal()[ii]
    assert abs(rs.mean()) <= 1e-17 * D.mean()
    assert np.abs(rs).max() <= 4e-16 * D.max()


def test_variable_kappa_energy():
    """For u = x, u^T K(kappa) u = sum_c kappa_c |cell| (grad u = e_x on every cell)."""
    N = 6
    kap = W.lognormal_kappa(2, N, 0.5, 3)
    _, K = fem.assemble(2, N, kap)
    u = W.node_coords(2, N)[0]
    assert math.isclose(u @ (K @ u), kap.sum() / N**2, rel_tol=1e-13)


@pytest.mark.parametrize("dim,N", [(2, 32), (2, 7), (3, 6)])
def test_sine_eigenvector(dim, N):
    """K S = lam_h M S with the closed form lam_h; M S = m1^dim S."""
    d = fem.Discretisation(dim, N)
    S = d.to_interior(W.sine_initial(dim, N))
    KS, MS = d.K @ S, d.M @ S
    assert np.abs(KS - mf.lam_h(dim, N) * MS).max() < 1e-12 * np.abs(KS).max()
    assert np.abs(MS - mf.m1(N) ** dim * S).max() < 1e-14
    if (dim, N) == (2, 32):
        assert abs(mf.lam_h(2, 32) - 19.7551) < 1e-4 and abs(mf.gamma(32) - 0.0312249) < 1e-7


@pytest.mark.parametrize("dim,N", [(2, 12), (3, 5)])
def test_manufactured_load(dim, N):
    """The closed-form load recipe of the workloads module equals quadrature of f."""
    f = lambda *x: np.prod([np.sin(np.pi * xi) for xi in x], axis=0)  # noqa: E731
    Fq = fem.load_by_quadrature(dim, N, f, order=8)
    ii = fem.interior_index(dim, N)
    assert np.abs(Fq[ii] - W.sine_load_space(dim, N)[ii]).max() < 1e-16
