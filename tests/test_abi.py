"""The C-ABI library builds, loads and exports every symbol of include/thc.h."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "thc.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"^(?:thc_status|const char\*|void)\s+(thc_\w+)\s*\(", text,
                                 flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    import paper_2111_11473_gb300 as pkg
    return pkg.load_library()


def test_header_declares_the_abi():
    assert _declared() == ["thc_config_default", "thc_cp_als", "thc_destroy", "thc_energy",
                           "thc_energy_noalloc", "thc_init", "thc_init_finish",
                           "thc_last_error", "thc_load_cholesky", "thc_mlp_create",
                           "thc_mlp_destroy",
                           "thc_mlp_get_params", "thc_mlp_loss_grad", "thc_mlp_num_params",
                           "thc_mlp_predict", "thc_mlp_set_params", "thc_mlp_train",
                           "thc_mp2_density", "thc_probe_alu", "thc_probe_gemm",
                           "thc_profile_enable", "thc_profile_read",
                           "thc_residual", "thc_selftest_bounded_wait", "thc_selftest_gemm", "thc_selftest_gemm_f64",
                           "thc_solve",
                           "thc_solve_opts_default", "thc_solve_pairs", "thc_solve_state_load",
                           "thc_solve_state_save", "thc_solve_state_size", "thc_step_name"]


def test_library_exports_every_declared_symbol(lib):
    import paper_2111_11473_gb300 as pkg
    out = subprocess.run(["nm", "-D", "--defined-only", pkg.binding.LIB_PATH],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(thc_\w+)", out))
    for name in _declared():
        assert name in exported, name
        assert hasattr(lib, name)
    assert set(pkg.exported_symbols()) <= exported


def test_config_defaults_and_argument_errors(lib):
    import ctypes as C
    from paper_2111_11473_gb300.binding import ThcConfig, ThcSolveOpts
    cfg = ThcConfig()
    assert lib.thc_config_default(C.byref(cfg), 5, 20, 60, 120, 60) == 0
    assert cfg.precision == 0 and cfg.lsq_rel_cutoff == 1e-10
    assert lib.thc_config_default(C.byref(cfg), 0, 20, 60, 120, 60) == 1
    opts = ThcSolveOpts()
    assert lib.thc_solve_opts_default(C.byref(opts)) == 0
    assert opts.r_tol == 1e-8 and opts.diis_n == 8
    # NULL arguments are rejected before any device work.
    h = C.c_void_p()
    assert lib.thc_init(None, None, None, None, None, None, None, None, C.byref(h)) == 1
    assert lib.thc_last_error(None).decode() != ""
    assert lib.thc_residual(None, None, None, None, None, None) == 1
    assert lib.thc_load_cholesky(None, 0, 1, None) == 1
    assert lib.thc_init_finish(None) == 1
    lib.thc_destroy(None)


def test_missing_library_fails_loudly(tmp_path):
    from paper_2111_11473_gb300 import binding
    with pytest.raises(RuntimeError, match="not built"):
        saved = binding._LIB
        binding._LIB = None
        try:
            binding.load_library(str(tmp_path / "libthc.so"))
        finally:
            binding._LIB = saved
