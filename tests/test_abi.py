"""The C ABI library builds for sm_103a, loads, and exports every entry point
declared in include/hd.h (no GPU needed: no compute call is made)."""
import ctypes

import pytest


def test_library_exports_declared_symbols():
    from paper_1508_02897_gb300.build import build
    path = build()
    from paper_1508_02897_gb300 import _binding as B
    names = B.declared_symbols()
    assert {"hd_setup_medium", "hd_factor_subdomains", "hd_apply_precond", "hd_gmres_solve", "hd_matvec"} <= set(names)
    L = ctypes.CDLL(path)
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(B._SIGS), "every declared function has a binding"
    assert B.hd_version().startswith("hd")


def test_invalid_arguments_are_rejected_without_gpu():
    from paper_1508_02897_gb300 import _binding as B
    with pytest.raises(B.HDError) as e:
        B.hd_query_workspace(None, 1, 1)
    assert e.value.code == B.HD_ERR_INVALID
    ctx = ctypes.c_void_p()
    g = B.hd_grid(0, 0, 0, 0.0, 0.0, 20.0, 2)
    d = B.hd_decomp(1, 1, 0, None, None, 1)
    rc = B.lib().hd_setup_medium(ctypes.byref(ctx), ctypes.byref(g), ctypes.byref(d), None, 0, None)
    assert rc == B.HD_ERR_INVALID and not ctx.value
    assert "NULL" in B.hd_last_error() or "bad" in B.hd_last_error()
