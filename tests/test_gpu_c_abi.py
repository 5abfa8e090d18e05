"""The C ABI from C: a C11 program (tests/c_abi_oscillator.c) compiled by gcc
with -std=c11 -pedantic against include/kv.h and linked with libkv.so runs the
paper's oscillator example (Sec. 2.2).  Its checks are the paper's printed
values: first violation at step 3 (t = 3 pi/4), the basis entries 0.707 and
3.54 there (Fig. 2), and the Krylov dimensions 2 (generator) and 4 (fixed
column, Sec. 4.2: the happy breakdown)."""
import json
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLD = json.load(open(os.path.join(ROOT, "tests", "golden", "oscillator.json")))


@pytest.mark.gpu
def test_c11_client_runs_the_oscillator(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_1804_01583_gb300 import build as kvbuild
    lib = kvbuild.build()
    exe = str(tmp_path / "c_abi_oscillator")
    cmd = ["gcc", "-std=c11", "-pedantic", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c_abi_oscillator.c"), "-o", exe, "-L", os.path.dirname(lib), "-lkv",
           "-Wl,-rpath," + os.path.dirname(lib), "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    kvs = dict(tok.split("=", 1) for tok in r.stdout.split())
    tol = GOLD["printed_digits_tol"]
    assert int(kvs["violation_step"]) == GOLD["violation_step"]
    assert int(kvs["violation_row"]) == 0
    k = GOLD["violation_step"]
    assert abs(float(kvs[f"basis_gen_{k}"]) - GOLD["basis_at_violation"]["i_y"]) <= tol
    assert abs(float(kvs[f"basis_fix_{k}"]) - GOLD["basis_at_violation"]["i_f"]) <= tol
    assert int(kvs["m_used_gen"]) == GOLD["krylov_dim_generator"]
    assert int(kvs["m_used_fix"]) == GOLD["krylov_dim_fixed_column"]
    for s in GOLD["no_violation_steps"]:
        assert float(kvs[f"basis_fix_{s}"]) + max(float(kvs[f"basis_gen_{s}"]), 0.0) < 4.0
