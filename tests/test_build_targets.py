"""What the sm_103a toolchain offers the split method (no GPU needed): the tensor-core
kinds it accepts. The split path multiplies 7-bit integer slices held exactly in bf16 or
fp16 (kind::f16); an INT8 form of the method would need tcgen05.mma kind::i8, which the
assembler refuses for sm_103a (it accepts it for sm_100a), so the only INT8 tensor path
on this GPU is the legacy mma.sync one (its rate: bsmm_measure_rates)."""
import shutil

import pytest

from paper_1504_05046_gb300 import build as B

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not __import__("os").path.exists(
    "/usr/local/cuda/bin/nvcc"), reason="needs nvcc")


def test_f16_kind_is_accepted():
    ok, msg = B.tcgen05_kind_supported("f16")
    assert ok, msg


def test_i8_kind_is_refused_on_sm_103a():
    ok, msg = B.tcgen05_kind_supported("i8")
    assert not ok
    assert "i8" in msg and "103" in msg, msg
