"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/idl.h declares (no compute calls: CPU only)."""
import ctypes

import paper_1901_10559_gb300 as idl


def test_header_declares_the_pipeline_and_stage_calls():
    names = idl.header_symbols()
    for n in ["id_matrix", "id_matrix_csr", "id_cp_tensor", "idl_create", "idl_destroy", "idl_sync",
              "idl_draw_countsketch", "idl_draw_gaussian", "idl_bucket_offsets", "idl_countsketch_dense",
              "idl_countsketch_csr", "idl_tensorsketch", "idl_gaussian_stage", "idl_cpqr", "idl_t_solve",
              "idl_lambda_hat"]:
        assert n in names, n


def test_library_exports_every_declared_symbol(built_lib):
    L = ctypes.CDLL(built_lib)
    missing = [n for n in idl.header_symbols() if not hasattr(L, n)]
    assert not missing, missing
    assert idl.lib().idl_version() >= 100


def test_binding_signatures_cover_the_header():
    declared = set(idl.header_symbols())
    bound = set(idl._SIGS)
    assert declared <= bound, declared - bound


def test_params_struct_layout_matches_header():
    # idl_params: 2 x int64, 2 x int32, uint64, 2 x int32, 4 x int64 = 72 bytes
    assert ctypes.sizeof(idl.Params) == 72
    assert ctypes.sizeof(idl.Info) == 40


def test_create_without_gpu_fails_cleanly(built_lib):
    import torch
    if torch.cuda.is_available():
        return
    p = ctypes.c_void_p()
    assert idl.lib().idl_create(ctypes.byref(p), 0) == idl.IDL_ECUDA
