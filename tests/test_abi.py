"""The C-ABI library loads and exports every symbol include/*.h declares;
host-only entry points validate their arguments (CPU only)."""

import ctypes
import os
import re

import pytest

from paper_1907_07774_gb300 import build
from paper_1907_07774_gb300 import rd as R

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return R.lib()


def declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            names |= set(re.findall(r"\b(r[dg]_[a-z_]+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert "rd_gradient" in names and "rd_hessvec" in names
    assert "rg_gradient" in names and "rg_hessvec" in names and "rg_project" in names
    for name in names:
        assert hasattr(lib, name), name


def test_config_default_and_workspace_size(lib):
    cfg = R.rd_config()
    assert lib.rd_config_default(ctypes.byref(cfg)) == 0
    assert list(cfg.n) == [64, 64, 64] and cfg.nt == 16 and cfg.prec == R.RD_FP64
    nb = ctypes.c_size_t()
    assert lib.rd_workspace_size(ctypes.byref(cfg), 8, ctypes.byref(nb)) == 0
    fields = 23 + 16      # working fields + one checkpoint slot per step
    assert nb.value >= fields * 64 ** 3 * 8 and nb.value < (fields + 8) * 64 ** 3 * 8
    cfg.prec = R.RD_MIXED
    nb32 = ctypes.c_size_t()
    assert lib.rd_workspace_size(ctypes.byref(cfg), 8, ctypes.byref(nb32)) == 0
    assert nb32.value < nb.value
    cfg.ckpt_stride = 4   # 4 stored states + 4 segment slots instead of 16
    nbs = ctypes.c_size_t()
    assert lib.rd_workspace_size(ctypes.byref(cfg), 8, ctypes.byref(nbs)) == 0
    assert nbs.value < nb32.value


def test_invalid_arguments_are_rejected(lib):
    cfg = R.rd_config()
    lib.rd_config_default(ctypes.byref(cfg))
    nb = ctypes.c_size_t()
    cfg.n[1] = 48
    assert lib.rd_workspace_size(ctypes.byref(cfg), 8, ctypes.byref(nb)) == 2   # RD_ERR_SHAPE
    cfg.n[1] = 64
    cfg.nt = 0
    assert lib.rd_workspace_size(ctypes.byref(cfg), 8, ctypes.byref(nb)) == 1   # RD_ERR_ARG
    cfg.nt = 4
    assert lib.rd_workspace_size(ctypes.byref(cfg), 0, ctypes.byref(nb)) == 1
    assert lib.rd_gradient(None, None, 0.0, 0.0, None, None) == 1
    assert lib.rd_last_pcg_iters(None) == 0


def test_state_solve_guesses_default_on_and_range_checked(lib):
    """rd_config.guess_restart: 0 by default (extrapolated guesses, restarted
    only at step 0 and at checkpoint segment starts), -1 turns them off,
    anything below -1 is an argument error; the setting does not change the
    workspace size."""
    cfg = R.rd_config()
    lib.rd_config_default(ctypes.byref(cfg))
    assert cfg.guess_restart == 0
    sizes = []
    for g in (0, -1, 5):
        cfg.guess_restart = g
        nb = ctypes.c_size_t()
        assert lib.rd_workspace_size(ctypes.byref(cfg), 8, ctypes.byref(nb)) == 0
        sizes.append(nb.value)
    assert sizes[0] == sizes[1] == sizes[2]
    cfg.guess_restart = -2
    assert lib.rd_workspace_size(ctypes.byref(cfg), 8, ctypes.byref(ctypes.c_size_t())) == 1


def test_registration_config_and_argument_checks(lib):
    from paper_1907_07774_gb300 import rg as G
    L = G.lib()
    cfg = G.rg_config()
    assert L.rg_config_default(ctypes.byref(cfg)) == 0
    assert list(cfg.n) == [64, 64, 64] and cfg.nt == 8 and cfg.prec == G.RD_FP64 and cfg.beta_v == 1e-2
    h = ctypes.c_void_p()
    cfg.n[2] = 40
    assert L.rg_create(ctypes.byref(h), ctypes.byref(cfg), None) == 2        # RD_ERR_SHAPE
    cfg.n[2] = 64
    cfg.nt = 0
    assert L.rg_create(ctypes.byref(h), ctypes.byref(cfg), None) == 1        # RD_ERR_ARG
    cfg.nt = 8
    cfg.beta_v = 0.0
    assert L.rg_create(ctypes.byref(h), ctypes.byref(cfg), None) == 1
    assert not h.value
    assert L.rg_gradient(None, None, None, None) == 1


def test_argument_checks_of_the_context_free_entry_points(lib):
    """Both context-free entry points reject bad arguments before touching a
    device (no GPU needed)."""
    assert lib.rd_selftest_bounded_wait(100, 0, None, None, None) == 1        # no status buffer
    assert lib.rd_selftest_bounded_wait(0, 0, None, 16, None) == 1            # zero polls
    assert lib.rd_selftest_bounded_wait(100, 0, None, 18, None) == 1          # status misaligned
    assert lib.rd_selftest_bounded_wait(100, 1, 24, 16, None) == 1            # source misaligned
    assert lib.rd_selftest_bounded_wait(1 << 27, 0, None, 16, None) == 1      # above the passes' limit
    dims = (ctypes.c_int * 3)(8, 8, 8)
    assert lib.rd_apply_precond_static(dims, 0.1, None, None, None) == 1
    assert lib.rd_apply_precond_static(dims, float("inf"), 16, 32, None) == 1
    assert lib.rd_apply_precond_static(dims, 0.1, 8, 32, None) == 1          # 16-byte alignment
