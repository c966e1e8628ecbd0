"""Host-side pins of the double-float arithmetic the FP32-iterate checks use
(csrc/lpb_df.h): error-free TwoSum / TwoProd, df add / mul / FMA-accumulate
against FP64, and the handling of infinite bounds.  Built with nvcc for the
host; runs without a GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_double_float_helpers(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "df_host_test"
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2601_21990_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "native", "df_host_test.cu"), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip().endswith("ok"), out.stdout[-2000:]


def test_graph_key_changes_with_every_baked_input(tmp_path):
    """A captured interval graph is replayed only while its key holds; the key
    must change with every pointer, size and launch shape the graph bakes in
    (lane buffers and leading dimension, check workspace, long-row lists)."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "graph_key_test"
    subprocess.check_call([nvcc, "-O1", "-std=c++17", "-I", os.path.join(ROOT, "paper_2601_21990_gb300", "csrc"),
                           "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "native", "graph_key_test.cu"), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip().endswith("ok"), out.stdout[-2000:]


def test_joint_launch_grid_covers_each_part_once(tmp_path):
    """The flattened grid of a joint step launch (several matrices in one
    launch): every block falls in one part's own grid, every place of every
    part is taken exactly once, in k_step's block order, and a grid past
    INT_MAX blocks is rejected (seeded random mixes of up to 8 parts)."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "joint_grid_test"
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2601_21990_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "native", "joint_grid_test.cu"), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip().endswith("ok"), out.stdout[-2000:]
