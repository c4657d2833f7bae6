"""Host-side checks of the C ABI library (no GPU needed): it loads, exports
every function include/stiles.h declares, and its task planner reproduces the
paper's GEMM counts and rejects corrupted dependency tables."""
import ctypes
import json
import os
import re

import pytest

from paper_2504_19171_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def S():
    B.build()
    from paper_2504_19171_gb300 import stiles
    return stiles


def declared_functions():
    text = open(os.path.join(ROOT, "include", "stiles.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(stiles_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(S):
    lib = ctypes.CDLL(S.LIB_PATH)
    names = declared_functions()
    assert "stiles_create" in names and "stiles_selinv" in names
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(S.EXPORTS) == names


def n_gemm_formula(N, B):
    return (N - B) * B + B * (B - 1) // 2 + B * B * (N - B - 1) + B * (B + 1) * (2 * B + 1) // 6


def test_plan_gemm_counts_match_paper_table(S):
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "gemm_counts.json")))
    for row in g["table"]:
        N, Bw = row["N"], row["B"]
        for which in (S.PLAN_SELINV, S.PLAN_FUSED):
            st = S.stiles_plan_stats(N - 1, 8, Bw - 1, 3, which, workers=4)
            assert st["tile_gemms"] == row["gemm"], (row, which)


@pytest.mark.parametrize("N", [2, 3, 5, 8, 13])
def test_plan_gemm_counts_match_formula(S, N):
    for Bw in range(1, N + 1):
        st = S.stiles_plan_stats(N - 1, 5, Bw - 1, 2, S.PLAN_SELINV, workers=8)
        assert st["tile_gemms"] == n_gemm_formula(N, Bw)


def test_plan_flops_split(S):
    # factor + selinv flops add up to the fused plan's
    for shape in [(16, 64, 1, 16), (7, 100, 3, 37), (5, 10, 0, 0)]:
        f = S.stiles_plan_stats(*shape, S.PLAN_FACTOR)["flops"]
        s = S.stiles_plan_stats(*shape, S.PLAN_SELINV)["flops"]
        u = S.stiles_plan_stats(*shape, S.PLAN_FUSED)["flops"]
        assert abs(f + s - u) <= 2


def test_plan_schedule_bounds(S):
    st = S.stiles_plan_stats(16, 64, 1, 16, S.PLAN_FUSED, workers=152)
    assert st["tasks"] > 0 and st["critical_path_ns"] > 0
    assert st["makespan_ns"] >= st["critical_path_ns"]


@pytest.mark.parametrize("mode", [1, 2, 3])
@pytest.mark.parametrize("which", [0, 1, 2])
def test_corrupted_tables_are_rejected(S, mode, which):
    assert S.stiles_debug_check_corrupted(6, 70, 2, 9, which, mode) == S.STILES_ERR_PLAN


def test_invalid_shapes(S):
    for shape in [(0, 4, 1, 1), (3, 0, 1, 1), (3, 4, -1, 1), (3, 4, 1, -2)]:
        with pytest.raises(S.StilesError) as e:
            S.stiles_plan_stats(*shape, 0)
        assert e.value.code == S.STILES_ERR_INVALID_ARG


def test_packed_layout_roundtrip(S):
    import numpy as np
    from paper_2504_19171_gb300 import workloads as W
    M = W.random_arrowhead(5, 7, 2, 3, seed=1)
    lay = S.PackedLayout(5, 7, 2, 3)
    flat = lay.pack(M.tiles, np.full(lay.doubles, np.nan))
    back = lay.unpack(flat)
    for key, T in M.tiles.items():
        assert np.array_equal(back[key], T)
    # column-major inside a tile, fixed column stride
    assert lay.offset(1, 0) == 49 and lay.offset(5, 0) == 3 * 49 and lay.offset(1, 1) == lay.colstride
    assert flat[1] == M.tiles[(0, 0)][1, 0]


VALIDATE_SHAPES = [(16, 64, 1, 16), (5, 100, 2, 37), (9, 130, 1, 70), (4, 3, 1, 2), (1, 50, 0, 5), (6, 64, 0, 0),
                   (7, 40, 4, 0), (3, 200, 2, 1), (12, 64, 3, 64), (30, 1, 1, 0), (10, 2, 3, 1), (6, 100, 1, 9)]


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("which", [0, 1, 2])
def test_plans_validate_on_host(S, which, precision):
    """Host emulation of one launch: in-bounds accesses of every task part,
    queue capacities, every task released once."""
    for shape in VALIDATE_SHAPES:
        assert S.stiles_debug_validate(*shape, which, precision) == S.STILES_OK, shape
