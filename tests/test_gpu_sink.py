"""FP32 / BF16 V-cycles write the FP64 stage vector from their finest up leg (ZSink in kernels.h).

The last finest-level up leg of a one-block cycle (triangular sweeps), of the batched P_D cycle and of the
monolithic cycle stores its result, rounded to the storage type, straight into the FGMRES stage vector, so no
separate scatter or cast pass runs after the cycle (on GB300 the results were compared bit for bit with the
separate passes); what remains is the cast of the input into the cycle's precision where the cycle reads it
(P_D, monolithic).  This pins the launch structure; the results of these paths are checked against the
oracle's cycles in test_gpu_parity.py, test_gpu_next.py and test_gpu_mmg.py.
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA GPU required", allow_module_level=True)

from paper_2403_08084_gb300 import Solver  # noqa: E402
from paper_2403_08084_gb300 import tableaux as PT  # noqa: E402


@pytest.mark.parametrize("precond,split,other_launches", [("lower", "ia", 0), ("upper", "ai", 0),
                                                          ("diag", "ia", 1), ("monolithic", "ai", 1)])
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_no_separate_output_pass(precond, split, other_launches, prec):
    N, levels = 128, 4
    with Solver(N, PT.radau_iia(3), 1 / 256, kappa=W.lognormal_kappa(2, N, 0.5, 41), levels=levels,
                precond=precond, vcycle=prec, splitting=split) as sv:
        v = torch.from_numpy(W.random_nodal(2, N, seed=42, s=3)).cuda()
        z = torch.empty_like(v)
        sv.apply_preconditioner(v, z)
        sv.perf_select([])
        sv.apply_preconditioner(v, z)
        p = sv.perf_read()["classes"]
        # "other": scatter / cast / scaling passes; the input cast stays for P_D and monolithic cycles
        assert p["other"]["launches"] == other_launches, p["other"]
        assert np.isfinite(z.cpu().numpy()).all()
