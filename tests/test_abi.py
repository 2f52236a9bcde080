"""Host-side checks of the C ABI: the library loads, exports what include/irk.h
declares, and rejects bad arguments before touching the GPU; without the library the
binding fails loudly, and the package never imports the oracle."""
import ctypes as C

import numpy as np
import pytest

from oracle import tableaux as O


def test_library_exports_every_declared_symbol():
    from paper_2403_08084_gb300 import _lib as L

    declared = L.header_symbols()
    assert "irk_create" in declared and "irk_step_adjoint" in declared and len(declared) >= 10
    for name in declared:
        assert hasattr(L.lib, name), name


def test_default_options():
    from paper_2403_08084_gb300 import _lib as L

    opt = L.irk_options()
    L.lib.irk_default_options(C.byref(opt))
    assert (opt.precond, opt.vcycle_prec, opt.nu_pre, opt.nu_post, opt.restart, opt.orth) == (1, 0, 2, 2, 50, 0)
    assert abs(opt.omega - 2 / 3) < 1e-15 and opt.rtol == 1e-10
    assert (opt.solver, opt.splitting, opt.warm_start) == (0, 0, 0)


@pytest.mark.parametrize("s", [1, 2, 3, 4])
def test_product_tableaux_match_oracle(s):
    from paper_2403_08084_gb300 import tableaux as T

    for prod, ref in ((T.radau_iia(s), O.radau_iia(s)), (T.gauss_legendre(s), O.gauss_legendre(s))):
        assert np.abs(prod.A - ref.A).max() < 1e-14
        assert np.abs(prod.b - ref.b).max() < 1e-14
        assert np.abs(prod.c - ref.c).max() < 1e-14
    assert np.abs(T.alexander().A - O.alexander().A).max() < 1e-14


def _create(N=8, levels=1, A=None, s=2, dt=0.1, **opt_over):
    from paper_2403_08084_gb300 import _lib as L

    tab = O.radau_iia(s)
    A = tab.A if A is None else A
    Aa, ba, ca = L.dbl_array(np.ravel(A)), L.dbl_array(tab.b), L.dbl_array(tab.c)
    mesh = L.irk_mesh(2, N, levels, None)
    t = L.irk_tableau(s, Aa, ba, ca)
    opt = L.irk_options()
    L.lib.irk_default_options(C.byref(opt))
    for k, v in opt_over.items():
        setattr(opt, k, v)
    h = C.c_void_p()
    rc = L.lib.irk_create(C.byref(h), C.byref(mesh), C.byref(t), dt, C.byref(opt), None)
    return rc, L.lib.irk_last_error().decode()


@pytest.mark.parametrize(
    "kwargs,needle",
    [
        (dict(A=O.radau_iia(3).A.T, s=3), "transposed"),
        (dict(N=12, levels=4), "divisible"),
        (dict(N=256, levels=2), "> 64"),
        (dict(dt=-1.0), "dt"),
        (dict(nu_pre=0), "nu_pre"),
        (dict(restart=0), "restart"),
        (dict(omega=2.5), "omega"),
        (dict(precond=7), "precond"),
        (dict(orth=5), "orth"),
        (dict(solver=1), "lower-triangular"),
        (dict(warm_start=2), "warm_start"),
    ],
)
def test_create_rejects_bad_input(kwargs, needle):
    rc, msg = _create(**kwargs)
    assert rc == -1 and needle in msg


def test_null_handle_is_rejected_without_a_gpu():
    """Entry points given a NULL handle return IRK_EINVAL before touching the device."""
    from paper_2403_08084_gb300 import _lib as L

    assert L.lib.irk_reset_initial_guess(None) == L.IRK_EINVAL
    assert "null" in L.lib.irk_last_error().decode()
    assert L.lib.irk_destroy(None) == 0


def test_missing_library_fails_loudly(tmp_path):
    """Without the built library the binding raises: there is no CPU fallback."""
    from paper_2403_08084_gb300 import _lib

    with pytest.raises(ImportError, match="no fallback"):
        _lib.load(str(tmp_path / "libirk.so"))


def test_product_never_imports_the_oracle():
    """The oracle is test infrastructure: no module of the package imports it."""
    import ast
    import pathlib

    pkg = pathlib.Path(__file__).resolve().parents[1] / "paper_2403_08084_gb300"
    for py in pkg.glob("*.py"):
        tree = ast.parse(py.read_text())
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                names = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                names = [node.module or ""]
            else:
                continue
            assert not any(n == "oracle" or n.startswith("oracle.") for n in names), (py.name, names)
