"""The small-level tail of the block V-cycles as one cooperative launch (mg2d_tail.cuh, IRK_TAIL=1).

The persistent kernel runs the fused legs of the levels below 513 nodes per axis and the coarsest solve
with the separate kernels' tiles and summation order, so its results must equal those of the separate
launches (the default) bit for bit, so the oracle parity of those carries over; it must replace them
(one launch per V-cycle); and a grid-barrier wait that runs out (forced with a zero wait limit,
IRK_TAIL_SPIN_CYCLES=0) must come back as IRK_ECUDA with the handle and the process still usable.
"""
import os

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA GPU required", allow_module_level=True)

from paper_2403_08084_gb300 import IRKError, Solver, _lib  # noqa: E402
from paper_2403_08084_gb300 import tableaux as PT  # noqa: E402


TAIL = {"IRK_TAIL": "1"}
SEPARATE = {"IRK_TAIL": "0"}


def make(N, levels, precond, prec, split, env=None, s=3):
    """A solver created with the given environment switches (read by irk_create)."""
    saved = {k: os.environ.get(k) for k in (env or {})}
    os.environ.update(env or {})
    try:
        return Solver(N, PT.radau_iia(s), 1 / 256, kappa=W.lognormal_kappa(2, N, 0.5, 11), levels=levels,
                      precond=precond, vcycle=prec, splitting=split, rtol=1e-12)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def apply(sv, v, transpose=False):
    z = torch.empty_like(v)
    sv.apply_preconditioner(v, z, transpose=transpose)
    return z.cpu().numpy()


@pytest.mark.parametrize("N,levels", [(256, 5), (800, 5), (1088, 6)])
@pytest.mark.parametrize("precond,prec,split", [("lower", "fp64", "ia"), ("lower", "fp32", "ai"),
                                                ("diag", "fp64", "ai"), ("lower", "bf16", "ia"),
                                                ("rana_ld", "fp32", "ia")])
def test_tail_matches_separate_launches_bitwise(N, levels, precond, prec, split):
    v = torch.from_numpy(W.random_nodal(2, N, seed=12, s=3)).cuda()
    with make(N, levels, precond, prec, split, TAIL) as a, make(N, levels, precond, prec, split, SEPARATE) as b:
        for transpose in ((False, True) if split == "ai" else (False,)):
            za, zb = apply(a, v, transpose), apply(b, v, transpose)
            assert np.array_equal(za, zb), float(np.abs(za - zb).max())


def test_tail_step_matches_separate_launches_bitwise():
    """Whole time steps (FGMRES in CUDA graphs, the tail launched inside them)."""
    N, levels, dt = 512, 6, 1 / 100
    u0 = torch.from_numpy(W.sine_initial(2, N)).cuda()
    f = torch.from_numpy(W.sine_load_space(2, N)).cuda()
    out = []
    for env in (TAIL, SEPARATE):
        with make(N, levels, "lower", "fp64", "ia", env) as sv:
            u = u0.clone()
            for n in range(3):
                sv.step(u, u, f_space=f, f_coef=[W.sine_load_time(2, (n + c) * dt) for c in PT.radau_iia(3).c])
            out.append(u.cpu().numpy())
    assert np.array_equal(out[0], out[1])


def test_tail_is_one_launch_per_vcycle():
    N, levels = 256, 5  # tail: 129, 65, 33 and the 17^2 coarsest level
    v = torch.from_numpy(W.random_nodal(2, N, seed=13, s=3)).cuda()
    for env, per_cycle in ((TAIL, 1), (SEPARATE, 7), (None, 7)):
        with make(N, levels, "lower", "fp64", "ia", env) as sv:
            sv.perf_select([])
            apply(sv, v)
            p = sv.perf_read()["classes"]
            launches = p["mg_tail"]["launches"] + p["coarse"]["launches"]
            assert launches == 3 * per_cycle, (env, p["mg_tail"]["launches"], p["coarse"]["launches"])


def test_tail_barrier_timeout_is_reported_and_recovers():
    """With a zero wait limit every block except the last to arrive gives up at the first barrier: the call
    returns IRK_ECUDA, the kernel ends, and the same process then runs a normal solver correctly."""
    N, levels = 256, 5
    v = torch.from_numpy(W.random_nodal(2, N, seed=14, s=3)).cuda()
    with make(N, levels, "lower", "fp64", "ia", {"IRK_TAIL": "1", "IRK_TAIL_SPIN_CYCLES": "0"}) as bad:
        with pytest.raises(IRKError) as e:
            apply(bad, v)
        assert e.value.code == _lib.IRK_ECUDA and "grid barrier" in str(e.value)
        with pytest.raises(IRKError):  # still times out (same limit), and still reports it
            apply(bad, v)
    with make(N, levels, "lower", "fp64", "ia", TAIL) as a, make(N, levels, "lower", "fp64", "ia", SEPARATE) as b:
        assert np.array_equal(apply(a, v), apply(b, v))
