"""The C-ABI from plain C: tests/c_consumer.c compiles as C99 against include/seg.h and links
against libseg.so (no GPU needed); on a GPU it runs one job through the ABI."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BUILD = os.path.join(ROOT, "paper_1403_0240_gb300", "_build")


def _compile(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_1403_0240_gb300 import seg
    seg.lib()                                          # builds libseg.so when it is missing
    exe = str(tmp_path / "c_consumer")
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c_consumer.c"), "-L", BUILD, "-lseg", f"-Wl,-rpath,{BUILD}", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_consumer_compiles_and_links(tmp_path):
    assert os.path.exists(_compile(tmp_path))


@pytest.mark.gpu
def test_c_consumer_runs_a_job(tmp_path):
    exe = _compile(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    ok, particles, accepted, fg = r.stdout.split()
    assert ok == "ok" and int(particles) > 0 and int(accepted) > 0
    assert 24 * 24 < int(fg) <= 40 * 40 + 4 * 40     # the label grows towards the bright square
