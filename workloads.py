"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds input recipes only (diffusivity fields, initial data, forcing
loads, random vectors, workload sizes).  It contains none of the solver's
arithmetic, so both the FP64 CPU oracle and the GPU library may be fed from it.

Vectors use the full node grid of a uniform mesh of the unit square/cube with
``N`` cells per direction: ``(N+1)**dim`` nodes, x fastest.  Boundary entries
are zero (homogeneous Dirichlet).  Stage vectors are node-major with the ``s``
stage values of a node contiguous: ``v[node*s + i]``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def n_nodes(dim: int, N: int) -> int:
    return (N + 1) ** dim


def n_cells(dim: int, N: int) -> int:
    return N**dim


def node_coords(dim: int, N: int) -> list[np.ndarray]:
    """Per-axis coordinates of every node (flattened, x fastest)."""
    x = np.arange(N + 1, dtype=np.float64) / N
    grids = np.meshgrid(*([x] * dim), indexing="ij")  # grids[d] indexed [i0, i1, ...]
    # flatten so that axis 0 (x) is fastest: transpose index order
    return [g.transpose(tuple(range(dim))[::-1]).reshape(-1) for g in grids]


def boundary_mask(dim: int, N: int) -> np.ndarray:
    idx = np.arange(N + 1)
    on = (idx == 0) | (idx == N)
    m = np.zeros([N + 1] * dim, dtype=bool)
    for d in range(dim):
        shape = [1] * dim
        shape[dim - 1 - d] = N + 1
        m |= on.reshape(shape)
    return m.reshape(-1)


def lognormal_kappa(dim: int, N: int, sigma: float = 0.5, seed: int = 0) -> np.ndarray:
    """Per-cell diffusivity with log(kappa) ~ Normal(0, sigma^2), i.i.d., cells x fastest."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.normal(0.0, sigma, n_cells(dim, N)))


def unit_directions(ncells: int, count: int, seed: int) -> np.ndarray:
    """``count`` Gaussian directions over cells, each scaled to unit Euclidean norm."""
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(count, ncells))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def random_nodal(dim: int, N: int, seed: int, s: int = 1) -> np.ndarray:
    """Random node-major vector with ``s`` values per node, zero on the boundary."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((n_nodes(dim, N), s))
    v[boundary_mask(dim, N)] = 0.0
    return v.reshape(-1) if s > 1 else v[:, 0].copy()


def sine_initial(dim: int, N: int) -> np.ndarray:
    """Nodal interpolant of prod_d sin(pi x_d) (zero on the boundary)."""
    u = np.ones(n_nodes(dim, N))
    for x in node_coords(dim, N):
        u *= np.sin(math.pi * x)
    u[boundary_mask(dim, N)] = 0.0
    return u


def sine_load_space(dim: int, N: int) -> np.ndarray:
    """Exact integral of prod_d sin(pi x_d) against each Q1 hat function.

    In 1D the integral of sin(pi x) against the hat at x_j is
    gamma * sin(pi x_j) with gamma = 2 (1 - cos(pi h)) / (pi^2 h); the Q1 hat is a
    tensor product, so the d-dimensional integral is gamma^d prod_d sin(pi x_j,d).
    """
    h = 1.0 / N
    gamma = 2.0 * (1.0 - math.cos(math.pi * h)) / (math.pi**2 * h)
    return gamma**dim * sine_initial(dim, N)


def sine_load_time(dim: int, t: float) -> float:
    """Time factor of the manufactured forcing f = (d pi^2 - 1) e^{-t} prod sin(pi x_d)."""
    return (dim * math.pi**2 - 1.0) * math.exp(-t)


def sine_exact(dim: int, N: int, t: float) -> np.ndarray:
    """u(t, x) = e^{-t} prod_d sin(pi x_d) at the nodes."""
    return math.exp(-t) * sine_initial(dim, N)


@dataclass(frozen=True)
class Workload:
    """A named heat-equation workload: mesh, tableau, step, preconditioner."""

    name: str
    dim: int
    N: int
    tableau: str
    s: int
    dt: float
    steps: int
    kappa_seed: int | None  # None: kappa = 1
    levels: int
    precond: str = "lower"
    vcycle: str = "fp64"
    rtol: float = 1e-10
    extra: dict = field(default_factory=dict)


# The five heat workloads.  Sizes follow the hot path they exercise.
WORKLOADS = {
    "heat2d-32-radau2": Workload("heat2d-32-radau2", 2, 32, "RadauIIA", 2, 1 / 32, 10, None, 1, "lower", "exact"),
    "heat2d-1024-radau3": Workload("heat2d-1024-radau3", 2, 1024, "RadauIIA", 3, 1 / 256, 20, 0, 6, "diag"),
    "heat3d-128": Workload("heat3d-128", 3, 128, "RadauIIA", 3, 1 / 64, 10, None, 5, "diag", "fp32"),
    "adjoint2d-512": Workload("adjoint2d-512", 2, 512, "RadauIIA", 3, 1 / 100, 50, 1, 6, "lower", "fp32"),
    "heat2d-2048-long": Workload("heat2d-2048-long", 2, 2048, "RadauIIA", 3, 1 / 100, 100, 0, 7, "lower"),
}
