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


def test_storage_flags_and_new_entry_points_validate_without_gpu():
    """Host-side checks run before any CUDA call: the tensor-core storage flag is
    refused with FP64 factors or together with symmetric storage, the split-TF32 flag
    without the tensor-core storage, an unknown flag bit is refused, and the multi-step DDM and FGMRES entry points refuse NULL
    contexts, zero steps and bad options."""
    from paper_1508_02897_gb300 import _binding as B
    L = B.lib()
    g = B.hd_grid(64, 64, 8, 1.0 / 64, 40.0, 20.0, 2)
    d = B.hd_decomp(2, 2, 4, None, None, 1)
    fake_c = ctypes.c_void_p(16)   # never dereferenced: validation fails first
    for prec in (B.HD_C128 | B.HD_TCORE, B.HD_C64 | B.HD_TCORE | B.HD_SYMMETRIC, B.HD_C64 | B.HD_TF32X3,
                 B.HD_C64 | 0x1000, 7):
        ctx = ctypes.c_void_p()
        rc = L.hd_setup_medium(ctypes.byref(ctx), ctypes.byref(g), ctypes.byref(d), fake_c, prec, None)
        assert rc == B.HD_ERR_INVALID and not ctx.value, prec
    assert "precision" in B.hd_last_error() or "HD_TCORE" in B.hd_last_error()
    p = ctypes.c_void_p(16)
    assert L.hd_apply_ddm(None, p, p, 1, 2, p, 1 << 20, p, 1 << 20, None) == B.HD_ERR_INVALID
    o = B.hd_gmres_opts(10, 100, 1e-6, 0, B.HD_ARNOLDI_DS, 0, 1, 1)
    st = (B.hd_gmres_stats * 1)()
    assert L.hd_gmres_solve(None, p, p, 1, ctypes.byref(o), p, 1 << 20, p, 1 << 20, st, None) == B.HD_ERR_INVALID


def test_restart_bound_is_enforced_without_gpu():
    """restart beyond HD_MAX_RESTART is refused by the workspace query, the solver and
    the server before any pointer is used or any CUDA call is made."""
    from paper_1508_02897_gb300 import _binding as B
    L = B.lib()
    for restart in (0, B.HD_MAX_RESTART + 1):
        with pytest.raises(B.HDError) as e:
            B.hd_query_workspace(None, 1, restart)
        assert e.value.code == B.HD_ERR_INVALID and "restart" in B.hd_last_error()
        p = ctypes.c_void_p(16)   # never dereferenced: validation fails first
        o = B.hd_gmres_opts(restart, 100, 1e-6, 0, B.HD_ARNOLDI_DS, 0, 1, 1)
        st = (B.hd_gmres_stats * 1)()
        assert L.hd_gmres_solve(p, p, p, 1, ctypes.byref(o), p, 1 << 20, p, 1 << 20, st, None) == B.HD_ERR_INVALID
        assert "bad options" in B.hd_last_error()



def test_block_solver_validates_without_gpu():
    """The block solver refuses bad block sizes, restarts and the multi-step preconditioner
    before any pointer is used or any CUDA call is made."""
    from paper_1508_02897_gb300 import _binding as B
    L = B.lib()
    p_ = ctypes.c_void_p(16)
    kb, sb = ctypes.c_size_t(), ctypes.c_size_t()
    for blk, restart in ((0, 5), (B.HD_MAX_BLOCK + 1, 5), (3, 0), (3, B.HD_MAX_RESTART + 1)):
        assert L.hd_query_block_workspace(p_, blk, restart, ctypes.byref(kb), ctypes.byref(sb)) == B.HD_ERR_INVALID
    st = (B.hd_gmres_stats * 3)()
    o = B.hd_gmres_opts(5, 100, 1e-6, 0, B.HD_ARNOLDI_FP64, 0, 0, 2)   # two preconditioner steps
    assert L.hd_block_gmres_solve(p_, p_, p_, 3, ctypes.byref(o), p_, 1 << 20, p_, 1 << 20, st, None) == B.HD_ERR_INVALID
    o = B.hd_gmres_opts(5, 100, 1e-6, 0, B.HD_ARNOLDI_FP64, 0, 0, 1)
    assert L.hd_block_gmres_solve(None, p_, p_, 3, ctypes.byref(o), p_, 1 << 20, p_, 1 << 20, st, None) == B.HD_ERR_INVALID
    assert L.hd_block_gmres_solve(p_, p_, p_, 0, ctypes.byref(o), p_, 1 << 20, p_, 1 << 20, st, None) == B.HD_ERR_INVALID
