"""The join kernels' key check of one row word (dpg::pk_word_ok, a masked
compare of two 64-bit halves) against its byte-by-byte definition: the
header compiled for the host by nvcc and run over every word size and every
word that overlaps the key.  No GPU is used."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    pytest.skip("nvcc not found")


def test_pk_word_ok_matches_byte_definition(tmp_path):
    exe = tmp_path / "pk_word_check"
    src = os.path.join(ROOT, "tests", "native", "pk_word_check.cu")
    inc = os.path.join(ROOT, "paper_cs_0308004_gb300", "csrc")
    subprocess.run([nvcc(), "-std=c++17", "-O2", "-I", inc, "-o", str(exe), src], check=True, capture_output=True)
    res = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert res.returncode == 0, res.stdout + res.stderr
    lines = res.stdout.strip().splitlines()
    assert len(lines) == 5 and all(l.endswith("mismatches=0") for l in lines), res.stdout
