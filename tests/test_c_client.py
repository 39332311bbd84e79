"""The library used from plain C: tests/c_client.c is compiled with gcc
against include/bf.h and linked with libbf.so.  Without a GPU it must build,
link and fail cleanly at bf_init; on the GPU it runs a search, a control and
a served request with closed-form checks."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1802_01685_gb300")


def build_client(tmp_path):
    import __graft_entry__
    __graft_entry__.build()
    if shutil.which("gcc") is None:
        pytest.skip("gcc not found")
    exe = tmp_path / "c_client"
    cmd = ["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c_client.c"), "-o", str(exe), "-L", PKG, "-lbf",
           "-Wl,-rpath," + PKG, "-lm"]
    subprocess.run(cmd, check=True)
    return exe


def gpu_present():
    try:
        import torch
        return torch.cuda.is_available()
    except ImportError:
        return False


def test_c_client_builds_and_fails_cleanly_without_gpu(tmp_path):
    if gpu_present():
        pytest.skip("a GPU is present: the GPU test runs the client")
    exe = build_client(tmp_path)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 77, (r.returncode, r.stdout, r.stderr)
    assert "no GPU" in r.stderr


@pytest.mark.gpu
def test_c_client_runs_on_the_gpu(tmp_path):
    exe = build_client(tmp_path)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    print(r.stdout)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.strip().endswith("OK")
