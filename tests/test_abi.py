"""The C ABI library without a GPU: it builds, loads, exports every declared
symbol, and rejects invalid arguments with status codes (no compute calls)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1504_05046_gb300 as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(bsmm_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    L = P.lib()
    decl = declared_functions()
    assert len(decl) >= 10
    for name in decl:
        assert hasattr(L, name), name
    assert sorted(P.EXPORTED) == sorted(n for n in decl if n in P.EXPORTED)
    assert set(decl) <= set(P.EXPORTED)


def test_options_default():
    o = P.bsmm_options_default()
    assert (o.mode, o.nslices, o.schedule, o.max_ctas) == (P.BSMM_FP64, 6, P.BSMM_SCHED_FLOPS, 0)


def test_invalid_arguments_return_status():
    L = P.lib()
    r = np.array([4, -1], np.int32)
    m = np.ones((2, 2), np.uint8)
    with pytest.raises(P.BsmmError) as ei:
        P.bsmm_plan(r, r, r, m, m)
    assert ei.value.status == 1 and "negative" in str(ei.value)
    with pytest.raises(P.BsmmError) as ei:
        P.bsmm_plan([4], [4], [4], [[1]], [[1]], mode=7)
    assert ei.value.status == 1
    with pytest.raises(P.BsmmError) as ei:
        P.bsmm_plan([4], [4], [4], [[1]], [[1]], mode=P.BSMM_SPLIT_BF16, nslices=9)
    assert ei.value.status == 1
    # NULL handles are rejected, never dereferenced
    assert L.bsmm_plan_query(None, None, None, None, None, None) == 1
    assert L.bsmm_execute(None, 1.0, None, None, None, None, 0.0, None, None, None) == 1
    assert L.bsmm_status_device(None, None) == 1
    L.bsmm_destroy(None)
    assert "NULL" in P.bsmm_last_error() or P.bsmm_last_error() != ""
    # the entry points added for split k, element types and batches reject NULL handles
    assert L.bsmm_execute_f32(None, 1.0, None, None, None, None, 0.0, None, None, None) == 1
    assert L.bsmm_plan_ksplit(None, None, None, None) == 1
    n = ctypes.c_int32()
    assert L.bsmm_batch_kernels(None, ctypes.byref(n)) == 1
    # the wait self-test rejects a limit out of range before touching the device
    assert L.bsmm_selftest_wait(10, None) == 1
    assert L.bsmm_selftest_wait(10 ** 10, None) == 1


def test_plan_without_gpu_reports_cuda_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(P.BsmmError) as ei:
        P.bsmm_plan([4], [4], [4], [[1]], [[1]])
    assert ei.value.status == 2


def test_tune_space_lists_fitting_candidates():
    """The autotuner's candidate list is host logic: FP64 tries both sub-tile edges;
    the split modes try every cluster size with every ring depth that fits 227 KB next to
    the C staging buffer, each in both kernel forms (without and with C store warps)."""
    import paper_1504_05046_gb300 as P
    assert P.bsmm_tune_space(P.BSMM_FP64) == [{"cluster": 0, "stages": 0, "fp64_tile": 32, "store_warps": 0},
                                               {"cluster": 0, "stages": 0, "fp64_tile": 64, "store_warps": 0}]
    s6 = P.bsmm_tune_space(P.BSMM_SPLIT_BF16, 6)
    assert [(c["cluster"], c["stages"], c["store_warps"]) for c in s6] == \
        [(cl, st, sw) for cl in (1, 2, 4) for st in (2, 3) for sw in (1, 2)]
    s3 = P.bsmm_tune_space(P.BSMM_SPLIT_FP16, 3)
    assert [(c["cluster"], c["stages"], c["store_warps"]) for c in s3] == \
        [(cl, st, sw) for cl in (1, 2, 4) for st in range(2, 7) for sw in (1, 2)]
    with pytest.raises(P.BsmmError):
        P.bsmm_tune_space(P.BSMM_SPLIT_BF16, 7)


def _model_file(path, version=1, feature_version=P.BSMM_FEATURE_VERSION, F=12, H=32, corrupt=False):
    """A cost-model file laid out as include/bsmm.h states (written here byte by byte)."""
    import struct
    NP = H * F + H + H * H + H + H + 1
    body = b"BSMMMLP\0" + struct.pack("<5I", version, feature_version, F, H, NP)
    body += struct.pack(f"<{NP}f", *([0.01] * NP)) + struct.pack(f"<{F}f", *([0.0] * F))
    body += struct.pack(f"<{F}f", *([1.0] * F)) + struct.pack("<2f", 0.0, 1.0)
    h = 1469598103934665603
    for c in body:
        h = ((h ^ c) * 1099511628211) & (2 ** 64 - 1)
    if corrupt:
        h ^= 1
    with open(path, "wb") as f:
        f.write(body + struct.pack("<Q", h))


def test_cost_model_file_checks_before_any_device_work(tmp_path):
    """bsmm_mlp_load refuses a missing file, a bad checksum, another format or feature
    version and another shape with BSMM_ERR_INVALID, before creating a model (no GPU
    needed); a well-formed file passes the checks and only then needs the device."""
    import torch
    L = P.lib()
    with pytest.raises(P.BsmmError) as ei:
        P.bsmm_mlp_load(tmp_path / "missing.bin")
    assert ei.value.status == 1
    for kw in (dict(corrupt=True), dict(version=2), dict(feature_version=9), dict(feature_version=1), dict(H=16)):
        _model_file(tmp_path / "m.bin", **kw)
        with pytest.raises(P.BsmmError) as ei:
            P.bsmm_mlp_load(tmp_path / "m.bin")
        assert ei.value.status == 1, kw
    (tmp_path / "short.bin").write_bytes(b"BSMMMLP\0")
    with pytest.raises(P.BsmmError) as ei:
        P.bsmm_mlp_load(tmp_path / "short.bin")
    assert ei.value.status == 1
    if not torch.cuda.is_available():
        _model_file(tmp_path / "good.bin")
        with pytest.raises(P.BsmmError) as ei:
            P.bsmm_mlp_load(tmp_path / "good.bin")
        assert ei.value.status == 2  # the file was accepted; creating the model needs a GPU
    assert L.bsmm_mlp_save(None, b"x") == 1
    assert L.bsmm_plan_cost_source(None, None) == 1


def test_execute_batch_rejects_null_arguments():
    L = P.lib()
    assert L.bsmm_execute_batch(0, None, None, None, None, None, None, None, None, None, None) == 1
    one = (ctypes.c_void_p * 1)(None)
    d = (ctypes.c_double * 1)(1.0)
    assert L.bsmm_execute_batch(1, one, d, one, one, one, one, d, one, one, None) == 1
    assert L.bsmm_measure_rates(None, None) == 1


def test_host_products_reject_null_arguments():
    L = P.lib()
    assert L.bsmm_plan_form(None, None, None, None, None, None) == 1
    assert L.bsmm_execute_host_async(None, 1.0, None, 0, None, None, 0, None, 0.0, None, 0, None, None) == 1
    assert L.bsmm_host_wait(None) == 1
    assert "NULL" in P.bsmm_last_error()
