"""Host-side helpers of bench.py (CPU only)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_kernel_hash_ignores_comments(tmp_path, monkeypatch):
    a = tmp_path / "a.cuh"
    b = tmp_path / "b.cuh"
    a.write_text("int f(int x)\n{\n    return x + 1;  // one more\n}\n")
    b.write_text("// a comment\nint f(int x)\n{\n\n    return x + 1;\n}\n")
    monkeypatch.setattr(bench, "KERNEL_SRC", str(a))
    ha = bench.kernel_hash()
    monkeypatch.setattr(bench, "KERNEL_SRC", str(b))
    assert bench.kernel_hash() == ha
    b.write_text("int f(int x)\n{\n    return x + 2;\n}\n")
    assert bench.kernel_hash() != ha


@pytest.mark.parametrize("storage,pattern", [("f32", "ab"), ("f16", "ab"), ("f16s", "ab"), ("bf16s", "ab"),
                                             ("f32", "aa"), ("f16", "aa")])
def test_committed_ncu_summaries_belong_to_the_current_kernel(storage, pattern):
    """The traffic figure bench.py reports comes from a capture of the kernel code as it is
    (the AA pattern's FP16 buffer partly stays in L2, hence the lower bound)."""
    t = bench.ncu_traffic(storage, "jet4096x1024", pattern)
    assert t is not None and 0.9 * bench.bytes_per_lup(storage) * 4096 * 1024 < t


def test_committed_batch_summary_belongs_to_the_current_kernel():
    """The ensemble's traffic figure: DRAM bytes per step of the 256-jet batch in moment-split
    storage, from a capture of the kernel code as it is."""
    t = bench.ncu_traffic("f16s", "ensemble256", kernel="batch")
    nodes = 23162880  # the seeded 256-jet ensemble
    assert t is not None and bench.bytes_per_lup("f16s") * nodes < t
    assert bench.ncu_traffic("f16", "ensemble256", kernel="batch") is None  # no summary: null


def test_kernel_hash_of_the_aa_pattern_covers_its_own_source():
    assert bench.kernel_hash("aa") != bench.kernel_hash("ab")


def test_step_launch_counts():
    class L:
        def __init__(self, nx, nr):
            self.nx, self.nr = nx, nr

    # one lattice: one launch unless the work counter would pass 2^31
    assert bench.step_launches([L(4096, 1024)], "f32", (6, 1, 2432), 20000) == 1
    assert bench.step_launches([L(4096, 1024)], "f32", (6, 1, 2432), 200000) == 3
    # a batch: graph replays of 64 steps plus one launch for the rest, each with its advance
    ls = [L(128, 64), L(256, 128)]
    assert bench.step_launches(ls, "f32", (16, 1, 0), 128) == 4
    assert bench.step_launches(ls, "f32", (16, 1, 0), 130) == 6
