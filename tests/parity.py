"""Parity bounds shared by the GPU tests, and the check that prints and asserts them.

One V-cycle (or block-preconditioner) application against the oracle's sparse
restatement of the same cycle, on the same seeded input: relative L2 error and
the largest element-wise error relative to the largest reference entry.

Bounds per V-cycle storage precision, relative L2: 1e-13 (FP64), 1e-5 (FP32),
1e-2 (BF16).  Element-wise: the same for FP64 and FP32; 2e-2 for BF16, about ten
units of BF16 rounding (2^-9) of the largest entry, since every stored vector
entry of a BF16 cycle carries its own rounding.

FP64 on large meshes needs the oracle's stiffness entries to be the rounded closed-form integrals
(rows summing to zero): a same-sign rounding bias in the row sums moved the oracle's own cycle by up
to 9e-13 at 1088^2, since the stiffness stencil applied to a smooth iterate cancels by a factor of
order h^2.
"""
import numpy as np

VCYCLE_TOL = {"fp64": 1e-13, "fp32": 1e-5, "bf16": 1e-2}
ELEMENT_TOL = {"fp64": 1e-13, "fp32": 1e-5, "bf16": 2e-2}


def errors(z, z_ref):
    z, z_ref = np.ravel(np.asarray(z, dtype=np.float64)), np.ravel(np.asarray(z_ref, dtype=np.float64))
    e = z - z_ref
    rel = float(np.linalg.norm(e) / max(np.linalg.norm(z_ref), 1e-300))
    mx = float(np.abs(e).max() / max(np.abs(z_ref).max(), 1e-300))
    return rel, mx


def check_vcycle(z, z_ref, prec, label, tol=None, tol_max=None):
    """Assert relative L2 and element-wise errors within the bounds for ``prec`` (printed first)."""
    rel, mx = errors(z, z_ref)
    b_rel = VCYCLE_TOL[prec] if tol is None else tol
    b_max = ELEMENT_TOL[prec] if tol_max is None else tol_max
    print(f"PARITY {label} {prec} rel={rel:.3e} max={mx:.3e} bound={b_rel:.1e}/{b_max:.1e}")
    assert rel <= b_rel and mx <= b_max, (label, prec, rel, mx)
