"""The C-ABI library loads without a GPU, exports every entry point declared in
include/nrc.h, and rejects bad arguments on the host before touching CUDA."""
import ctypes
import os
import subprocess

import pytest

from paper_2106_12372_gb300 import nrc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2106_12372_gb300 import build

    build.build()
    return nrc.lib()


def test_header_declares_the_boundary():
    names = nrc.declared_functions()
    for n in ("nrc_create", "nrc_encode", "nrc_infer", "nrc_train_step", "nrc_destroy", "nrc_gather",
              "nrc_frame", "nrc_frame_host", "nrc_get_state", "nrc_set_state", "nrc_check_error"):
        assert n in names


def test_library_exports_every_declared_symbol(L):
    for name in nrc.declared_functions():
        assert hasattr(L, name), name


def test_exported_symbols_are_only_the_abi(L):
    out = subprocess.run(["nm", "-D", "--defined-only", nrc.LIB_PATH], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert set(nrc.declared_functions()) <= exported
    assert not [s for s in exported if s.startswith("oracle_")]


def test_default_config(L):
    cfg = nrc.default_config()
    assert (cfg.width, cfg.hidden_layers, cfg.dtype, cfg.pad_value) == (64, 5, nrc.FP16, 1.0)
    assert abs(cfg.lr - 1e-2) < 1e-9 and abs(cfg.beta2 - 0.99) < 1e-7 and abs(cfg.loss_eps - 0.01) < 1e-9


def test_bad_arguments_fail_on_the_host(L):
    # checks that run before any CUDA call
    h = ctypes.c_void_p()
    bad = nrc.default_config(hidden_layers=0)
    assert L.nrc_create(ctypes.byref(bad), None, ctypes.byref(h)) == nrc.NRC_ERR_INVALID_ARG
    assert b"hidden_layers" in L.nrc_last_error_string()
    assert L.nrc_create(ctypes.byref(nrc.default_config(width=96)), None, ctypes.byref(h)) == nrc.NRC_ERR_UNSUPPORTED
    assert L.nrc_create(ctypes.byref(nrc.default_config(dtype=7)), None, ctypes.byref(h)) == nrc.NRC_ERR_INVALID_ARG
    assert L.nrc_create(None, None, ctypes.byref(h)) == nrc.NRC_ERR_INVALID_ARG
    assert L.nrc_infer(None, None, 10, None, None) == nrc.NRC_ERR_INVALID_ARG
    assert L.nrc_train_step(None, None, None, 10, 10, 0, 0, None, None) == nrc.NRC_ERR_INVALID_ARG
    assert L.nrc_gather(None, None, 100, -1, 0, 0, None, None, None) == nrc.NRC_ERR_INVALID_ARG
    assert L.nrc_gather(None, None, 100, 60, 0, 1, None, None, None) == nrc.NRC_ERR_INVALID_ARG  # 2*60 > 100
    assert L.nrc_gather(None, None, 100, 10, 0, 0, None, None, None) == nrc.NRC_ERR_INVALID_ARG  # NULL pool
    assert L.nrc_gather(None, None, 100, 0, 0, 0, None, None, None) == nrc.NRC_OK  # empty batch: no-op
    assert L.nrc_destroy(None) == nrc.NRC_OK
    assert L.nrc_param_count(None) == 0


def test_path_tiling_helpers_on_the_host():
    from paper_2106_12372_gb300 import build, nrc

    build.build()
    assert nrc.paths_tile_count(1920, 1080, 8) == 240 * 135
    assert nrc.paths_tile_count(37, 21, 8) == 5 * 3
    assert nrc.paths_tile_count(0, 21, 8) == 0
    # records scale with the number of tiles ~ 1 / tile^2: four times the target doubles the side
    assert nrc.paths_adapt_tile(8, 4 * 65536, 65536) == 16
    assert nrc.paths_adapt_tile(8, 65536 // 4, 65536) == 4
    assert nrc.paths_adapt_tile(8, 65536, 65536) == 8
    assert nrc.paths_adapt_tile(1, 1, 10 ** 9) == 1 and nrc.paths_adapt_tile(200, 10 ** 9, 1) == 256
    # the records scan's scratch: the offsets plus one block total per 2048 tiles
    assert nrc.paths_offsets_count(0) == 0
    assert nrc.paths_offsets_count(1) == 2
    assert nrc.paths_offsets_count(2048) == 2049
    assert nrc.paths_offsets_count(2049) == 2051
    assert nrc.paths_offsets_count(32400) == 32400 + 16
