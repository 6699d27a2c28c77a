"""The benchmark's host-side bookkeeping, without a GPU: the recorded DRAM traffic of the
contraction kernel is reported only while the kernel's source is the one it was measured
on (comments and blank space aside)."""
import importlib.util
import os
import shutil

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
REPO = os.path.dirname(HERE)


@pytest.fixture()
def bench(tmp_path):
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(REPO, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    src = tmp_path / "paper_1504_05046_gb300" / "csrc"
    src.mkdir(parents=True)
    for f in ("split.cu", "bsmm_internal.h"):
        shutil.copy(os.path.join(REPO, "paper_1504_05046_gb300", "csrc", f), src / f)
    (tmp_path / "profiles").mkdir()
    mod.ROOT = str(tmp_path)
    mod.PROFILE_FILE = str(tmp_path / "profiles" / "p.txt")
    return mod, src


def _write_profile(mod, h, nbytes):
    with open(mod.PROFILE_FILE, "w") as f:
        f.write(f"a summary line: with a colon\nkernel_source_hash: {h}\ndram_bytes_per_full_launch: {nbytes}\n")


def test_comment_and_space_edits_keep_the_hash(bench):
    mod, src = bench
    h0 = mod.kernel_source_hash()
    p = src / "split.cu"
    text = p.read_text()
    p.write_text("// a new line comment\n/* a block\n   comment */\n" + text.replace("\n", "\n\n", 5))
    assert mod.kernel_source_hash() == h0


def test_code_edit_changes_the_hash_and_drops_the_traffic(bench):
    mod, src = bench
    _write_profile(mod, mod.kernel_source_hash(), 123000000000)
    assert mod.profiled_traffic() == 123e9
    p = src / "bsmm_internal.h"
    p.write_text(p.read_text() + "\nconstexpr int kAnotherConstant = 1;\n")
    assert mod.profiled_traffic() is None


def test_missing_or_malformed_profile_gives_no_traffic(bench):
    mod, _ = bench
    assert mod.profiled_traffic() is None
    _write_profile(mod, mod.kernel_source_hash(), "not-a-number")
    assert mod.profiled_traffic() is None

