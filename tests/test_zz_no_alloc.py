"""irk_apply_preconditioner_noalloc against irk_apply_preconditioner, through the C ABI.

The no-allocation entry point serves callers that cannot allocate device memory
while they apply the preconditioner (for example inside a CUDA-graph stream
capture, or on threads that must not touch the allocator).  It keeps its
multigrid level vectors in a static 16 MiB device array shared by all calls, so
the test checks two calls in a row, a handle of another size in between (the
array keeps earlier contents), and the size limit.  This file is collected last.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA GPU required", allow_module_level=True)

from paper_2403_08084_gb300 import Solver, _lib  # noqa: E402
from paper_2403_08084_gb300 import tableaux as PT  # noqa: E402


def noalloc(sv, v, z, transpose=False):
    return _lib.lib.irk_apply_preconditioner_noalloc(sv._h, C.c_void_p(v.data_ptr()), C.c_void_p(z.data_ptr()),
                                                     int(transpose))


def rel(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("N,levels,kind,prec", [(96, 3, "lower", "fp64"), (64, 2, "diag", "fp32"),
                                                (128, 4, "upper", "bf16")])
def test_noalloc_matches_allocating_entry_point(N, levels, kind, prec):
    s = 3
    kap = W.lognormal_kappa(2, N, 0.5, seed=21)
    v = torch.from_numpy(W.random_nodal(2, N, seed=22, s=s)).cuda()
    with Solver(N, PT.radau_iia(s), 1 / 64, kappa=kap, levels=levels, precond=kind, vcycle=prec) as sv:
        for transpose in (False, True):
            z_ref = torch.empty(sv.n_nodes * s, dtype=torch.float64, device="cuda")
            sv.apply_preconditioner(v, z_ref, transpose=transpose)
            for _ in range(2):  # two calls in a row share the static array
                z = torch.full_like(z_ref, 3.0)
                assert noalloc(sv, v, z, transpose) == 0, _lib.lib.irk_last_error().decode()
                assert rel(z, z_ref) <= 1e-12


def test_noalloc_rejects_oversize_and_host_pointers():
    s, N = 3, 512
    with Solver(N, PT.radau_iia(s), 1 / 64, levels=5, precond="lower", vcycle="fp64") as sv:
        v = torch.zeros(sv.n_nodes * s, dtype=torch.float64, device="cuda")
        z = torch.zeros_like(v)
        assert noalloc(sv, v, z) == _lib.IRK_EINVAL
        assert "scratch" in _lib.lib.irk_last_error().decode()
    with Solver(32, PT.radau_iia(s), 1 / 64, levels=2) as sv:
        vh = np.zeros(sv.n_nodes * s)
        zh = np.zeros(sv.n_nodes * s)
        rc = _lib.lib.irk_apply_preconditioner_noalloc(sv._h, C.c_void_p(vh.ctypes.data), C.c_void_p(zh.ctypes.data), 0)
        assert rc == _lib.IRK_EINVAL and "device pointers" in _lib.lib.irk_last_error().decode()
