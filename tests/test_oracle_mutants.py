"""The oracle's pins must catch plausible mistakes.

Each case below compiles a copy of the oracle with one deliberate error planted in
its source (on the CPU, in a temporary directory) and re-runs test_oracle.py against
that copy in a subprocess. The run must fail. An unmodified copy must pass, which
shows that the harness itself works.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BODY = "ksort_ref_body.h"

MUTANTS = {
    # Step 3: ties sent left instead of right.
    "ties_left": ("if (key <= a[p]) {", "if (key < a[p]) {"),
    # Step 4: the saved temp is never written back.
    "drop_temp": ("        a[i + 1] = temp;\n", "        ;\n"),
    # Step 3.1: temp saved but flag never raised.
    "no_flag": ("temp = a[p];\n                flag = 1;", "temp = a[p];"),
    # Step 6 as printed ("left > i+1"): right parts are never sorted.
    "step6_as_printed": ("if (right > i + 1) {", "if (left > i + 1) {"),
    # Step 5 off by one: two-element left parts are left unsorted.
    "step5_off_by_one": ("if (left < i - 1) {", "if (left < i - 2) {"),
    # Step 3.2 without k = k + 1: the scan re-reads one position.
    "no_k_increment": ("            k = k + 1;\n", ""),
    # Step 1 with j = right: the last element is never classified.
    "j_init_right": ("int64_t j = right + 1;", "int64_t j = right;"),
    # Steps 5/6 order swapped (right part first): same sorted output, wrong call order.
    "right_part_first": (
        "        /* Step 6 (pushed first, so it runs after everything Step 5 starts). */\n"
        "        if (right > i + 1) {\n"
        "            lo_s[top] = i + 1; hi_s[top] = right; depth_s[top] = depth + 1; top++;\n"
        "        }\n"
        "        /* Step 5. */\n"
        "        if (left < i - 1) {\n"
        "            lo_s[top] = left; hi_s[top] = i - 1; depth_s[top] = depth + 1; top++;\n"
        "        }\n",
        "        if (left < i - 1) {\n"
        "            lo_s[top] = left; hi_s[top] = i - 1; depth_s[top] = depth + 1; top++;\n"
        "        }\n"
        "        if (right > i + 1) {\n"
        "            lo_s[top] = i + 1; hi_s[top] = right; depth_s[top] = depth + 1; top++;\n"
        "        }\n"),
}


def _build_copy(tmp_path, name, mutation):
    src = os.path.join(ROOT, "oracle")
    dst = tmp_path / name
    dst.mkdir()
    for f in ("ksort_ref.c", "ksort_ref.h", BODY):
        shutil.copy(os.path.join(src, f), dst / f)
    if mutation is not None:
        old, new = mutation
        text = (dst / BODY).read_text()
        assert text.count(old) == 1, f"mutation anchor for {name} not found exactly once"
        (dst / BODY).write_text(text.replace(old, new))
    so = dst / "libksort_ref_mut.so"
    subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", str(dst / "ksort_ref.c"),
                    "-o", str(so)], check=True)
    return str(so)


def _run_pins(so):
    env = dict(os.environ, KSORT_ORACLE_SO=so, PYTHONPATH=ROOT)
    cmd = [sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle.py"),
           "-x", "-q", "-p", "no:cacheprovider"]
    try:
        r = subprocess.run(cmd, env=env, cwd=ROOT, capture_output=True, text=True, timeout=300)
    except subprocess.TimeoutExpired:
        return None
    return r.returncode


def test_unmodified_copy_passes(tmp_path):
    assert _run_pins(_build_copy(tmp_path, "control", None)) == 0


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    rc = _run_pins(_build_copy(tmp_path, name, MUTANTS[name]))
    assert rc != 0, f"pins did not catch mutant {name}"
