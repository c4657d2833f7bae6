"""The C ABI from a plain C program (no Python, no torch).

A C99 program is compiled with gcc against ``include/stiles.h`` alone and
linked to the built library. It calls the host-only entry points (plan
statistics, host validation, error strings) and tries to create a handle:
without a CUDA device that must fail with STILES_ERR_CUDA (no CPU fallback);
with one, the handle is created and destroyed. Its output is checked against
the closed-form flop count and the paper's GEMM-count table."""
import json
import os
import shutil
import subprocess

import pytest

from oracle import flops as F

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BUILD = os.path.join(ROOT, "paper_2504_19171_gb300", "_build")

PROGRAM = r"""
#include <stdio.h>
#include "stiles.h"

int main(void) {
  long long st[10];
  /* the n = 1040 configuration: nt 16, b 64, w 1, a 16 (fused plan) */
  int rc = stiles_plan_stats(16, 64, 1, 16, 2, 152, st);
  printf("stats %d %lld %lld %lld %lld\n", rc, st[0], st[4], st[5], st[9]);
  /* phase-2 tile GEMMs of an arrowhead of N = 6 tiles (5 band tile columns
     and the arrow; selinv plan) with lower tile bandwidth w = 0 and w = 1 */
  rc = stiles_plan_stats(5, 8, 0, 8, 1, 16, st);
  printf("gemms_w0 %d %lld\n", rc, st[5]);
  rc = stiles_plan_stats(5, 8, 1, 8, 1, 16, st);
  printf("gemms_w1 %d %lld\n", rc, st[5]);
  printf("validate %d\n", stiles_debug_validate(16, 64, 1, 16, 2));
  printf("invalid %d\n", stiles_plan_stats(0, 64, 1, 16, 2, 152, st));
  printf("strerror %s\n", stiles_strerror(STILES_ERR_NOT_SPD));
  stiles_t h = NULL;
  rc = stiles_create(16, 64, 1, 16, STILES_FP64, &h);
  printf("create %d %d\n", rc, h != NULL);
  if (rc == STILES_OK) stiles_destroy(h);
  return 0;
}
"""


@pytest.fixture(scope="module")
def program(tmp_path_factory):
    lib = os.path.join(BUILD, "libstiles.so")
    if not os.path.exists(lib):
        pytest.fail(f"{lib} is missing: build the library first")
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    d = tmp_path_factory.mktemp("cabi")
    src, exe = d / "consumer.c", d / "consumer"
    src.write_text(PROGRAM)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe), "-L", BUILD, "-lstiles", f"-Wl,-rpath,{BUILD}"], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return dict(line.split(" ", 1) for line in out.strip().splitlines())


def test_plan_statistics_from_c(program):
    rc, tasks, flops, gemms, edges = (int(x) for x in program["stats"].split())
    assert rc == 0 and tasks > 0 and gemms > 0 and 0 < edges < 8 * tasks
    assert flops == round(F.flops(16, 64, 1, 16, "fused"))


def test_gemm_count_from_c_matches_paper_table(program):
    """The GEMM-count table of Sec. III-E (tests/golden/gemm_counts.json) at
    N = 6 tiles: 10 tile GEMMs for B = 1 and 26 for B = 2, B counting the band
    tiles including the diagonal (w = B - 1)."""
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "gemm_counts.json")))
    want = {row["B"]: row["gemm"] for row in g["table"] if row["N"] == 6}
    for key, B in (("gemms_w0", 1), ("gemms_w1", 2)):
        rc, gemms = (int(x) for x in program[key].split())
        assert rc == 0 and gemms == want[B], (key, gemms, want[B])


def test_host_validation_and_errors_from_c(program):
    assert int(program["validate"]) == 0
    assert int(program["invalid"]) == -1            # STILES_ERR_INVALID_ARG
    assert "SPD" in program["strerror"] or "positive" in program["strerror"].lower()


def test_create_without_fallback(program):
    rc, got = (int(x) for x in program["create"].split())
    import torch
    if torch.cuda.is_available():
        assert rc == 0 and got == 1
    else:
        assert rc == -4 and got == 0                # STILES_ERR_CUDA: no device, no CPU path
