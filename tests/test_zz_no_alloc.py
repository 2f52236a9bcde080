"""irk_apply_preconditioner_noalloc against irk_apply_preconditioner, through the C ABI.

The no-allocation entry point serves callers that cannot allocate device memory
while they apply the preconditioner: host threads that must not enter the
allocator (real-time loops) and embeddings whose device memory belongs to
another framework's fixed budget.  It keeps its multigrid level vectors in a
static 16 MiB device array shared by all calls, so the tests check two calls in
a row against the allocating entry point, handles of other sizes in between (the
array keeps the last call's contents), that the device's free memory does not
change across the calls, and the rejections (oversize handles, host pointers, a
transposed IA preconditioner).  This file is collected last, so a run that stops
at its first failure has run every other test before it.
"""
import ctypes as C
import gc

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA GPU required", allow_module_level=True)

from paper_2403_08084_gb300 import Solver, _lib  # noqa: E402
from paper_2403_08084_gb300 import tableaux as PT  # noqa: E402

TOL = 1e-12  # same V-cycle arithmetic on other buffers: agreement to rounding of the final casts


def noalloc(sv, v, z, transpose=False):
    return _lib.lib.irk_apply_preconditioner_noalloc(sv._h, C.c_void_p(v.data_ptr()), C.c_void_p(z.data_ptr()),
                                                     int(transpose))


def rel(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def solver(N, levels, kind, prec, split="ai", dim=2, seed=21):
    s = 3
    kap = W.lognormal_kappa(2, N, 0.5, seed=seed) if dim == 2 else None
    return Solver(N, PT.radau_iia(s), 1 / 64, dim=dim, kappa=kap, levels=levels, precond=kind, vcycle=prec,
                  splitting=split)


def check_two_calls(sv, transpose, seed=22):
    s = sv.s
    v = torch.from_numpy(W.random_nodal(sv.dim, sv.N, seed=seed, s=s)).cuda()
    z_ref = torch.empty(sv.n_nodes * s, dtype=torch.float64, device="cuda")
    sv.apply_preconditioner(v, z_ref, transpose=transpose)
    for _ in range(2):  # two calls in a row share the static array
        z = torch.full_like(z_ref, 3.0)
        assert noalloc(sv, v, z, transpose) == 0, _lib.lib.irk_last_error().decode()
        assert rel(z, z_ref) <= TOL
        assert float((z - z_ref).abs().max()) <= TOL * float(z_ref.abs().max())


@pytest.mark.parametrize("N,levels,kind,prec,split,dim", [
    (96, 3, "lower", "fp64", "ai", 2), (64, 2, "diag", "fp32", "ai", 2), (128, 4, "upper", "bf16", "ai", 2),
    (96, 3, "lower", "fp64", "ia", 2), (64, 3, "rana_ld", "fp32", "ia", 2), (64, 3, "monolithic", "fp32", "ai", 2),
    (64, 3, "monolithic", "fp64", "ai", 2), (32, 3, "lower", "fp32", "ai", 3), (16, 2, "lower", "fp64", "ia", 3)])
def test_noalloc_matches_allocating_entry_point(N, levels, kind, prec, split, dim):
    with solver(N, levels, kind, prec, split, dim) as sv:
        for transpose in ((False, True) if split == "ai" else (False,)):
            check_two_calls(sv, transpose)


def test_noalloc_after_larger_and_smaller_handles():
    """Large, then small, then large again: each call clears what it uses, so stale contents left by a
    handle of another size do not reach the result."""
    with solver(160, 4, "lower", "fp64") as big, solver(32, 2, "lower", "bf16", seed=5) as small:
        check_two_calls(big, False, seed=1)
        check_two_calls(small, True, seed=2)
        check_two_calls(big, True, seed=3)
        check_two_calls(small, False, seed=4)


def test_noalloc_leaves_device_memory_unchanged():
    with solver(128, 4, "lower", "fp32") as sv:
        s = sv.s
        v = torch.from_numpy(W.random_nodal(2, 128, seed=8, s=s)).cuda()
        z = torch.empty(sv.n_nodes * s, dtype=torch.float64, device="cuda")
        assert noalloc(sv, v, z) == 0  # the first call may load the library's device code
        # tensors left by earlier tests are freed first, and no collection runs during the calls
        gc.collect()
        gc.disable()
        try:
            free0, torch0 = free_bytes(), (torch.cuda.memory_allocated(), torch.cuda.memory_reserved())
            for transpose in (False, True, False):
                assert noalloc(sv, v, z, transpose) == 0, _lib.lib.irk_last_error().decode()
            free1, torch1 = free_bytes(), (torch.cuda.memory_allocated(), torch.cuda.memory_reserved())
        finally:
            gc.enable()
        assert free1 == free0
        assert torch1 == torch0


def test_noalloc_rejects_oversize_host_pointers_and_transposed_ia():
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
    with solver(32, 2, "lower", "fp64", "ia") as sv:
        v = torch.zeros(sv.n_nodes * s, dtype=torch.float64, device="cuda")
        z = torch.zeros_like(v)
        assert noalloc(sv, v, z, True) == _lib.IRK_EINVAL
        assert "AI splitting" in _lib.lib.irk_last_error().decode()
