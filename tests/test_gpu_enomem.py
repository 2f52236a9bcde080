"""IRK_ENOMEM through the C ABI, with the allocation failures injected on the host.

IRK_FAIL_DEVICE_ALLOC=n makes every n-th device allocation of the process fail
before cudaMalloc is called, so no device memory is exhausted and nothing runs
on the GPU that could fault.  In a child process, a loop of irk_create / irk_step
(host buffers, which allocate staging memory) / irk_destroy meets failures at
many different points of set-up and of the first step: every failure must come
back as IRK_ENOMEM with its message, leave the process able to build and run the
next solver, and release what the failed call had allocated (the device's free
memory returns to its value before the loop).
"""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA GPU required", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import numpy as np, torch
torch.cuda.init()
import workloads as W
from paper_2403_08084_gb300 import IRKError, Solver, _lib
from paper_2403_08084_gb300 import tableaux as PT

N, s, dt = 64, 3, 1 / 64
kap = W.lognormal_kappa(2, N, 0.5, 7)
u0, fsp = W.sine_initial(2, N), W.sine_load_space(2, N)
coef = [W.sine_load_time(2, c * dt) for c in PT.radau_iia(s).c]

def attempt():
    sv = None
    try:
        sv = Solver(N, PT.radau_iia(s), dt, kappa=kap, levels=3, precond="lower", rtol=1e-12)
        u1 = np.empty(sv.n_nodes)
        sv.step(u0, u1, f_space=fsp, f_coef=coef)
        return ("ok", float(np.linalg.norm(u1)))
    except IRKError as e:
        return ("enomem" if e.code == _lib.IRK_ENOMEM else "other", str(e))
    finally:
        if sv is not None:
            sv.close()

for _ in range(20):  # warm the context and the device code once
    if attempt()[0] == "ok":
        break
torch.cuda.synchronize()
free0 = torch.cuda.mem_get_info()[0]
outcomes = [attempt() for _ in range(int(sys.argv[2]))]
torch.cuda.synchronize()
print(json.dumps({"outcomes": outcomes, "free_before": free0, "free_after": torch.cuda.mem_get_info()[0]}))
"""


# periods above the ~60 device allocations of one create + step, so that failures land at a different
# point of each attempt and successful attempts come between them
@pytest.mark.parametrize("period", [97, 151, 211])
def test_injected_allocation_failures(period):
    env = dict(os.environ, IRK_FAIL_DEVICE_ALLOC=str(period))
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, "24"], capture_output=True, text=True, timeout=600,
                       env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    kinds = [k for k, _ in res["outcomes"]]
    assert "other" not in kinds, res["outcomes"]
    assert kinds.count("enomem") >= 1 and kinds.count("ok") >= 1, kinds
    for k, msg in res["outcomes"]:
        if k == "enomem":
            assert "IRK_ENOMEM" in msg and "injected" in msg
    norms = {round(v, 9) for k, v in res["outcomes"] if k == "ok"}
    assert len(norms) <= 1  # every successful solver gives the same step
    assert res["free_after"] == res["free_before"]
