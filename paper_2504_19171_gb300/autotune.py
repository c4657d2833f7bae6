"""Autotuner of the plan tuning code (``stiles_create_tuned`` /
``stiles_batch_create``) and of the workers per SM (``STILES_OPT_GRID``).

The planner cuts the work into tasks in several legal ways (tuning code bit
fields, see include/stiles.h): how many source block columns one factor
update task applies, and into how many CTA parts phase-2 and factor update
blocks are split. Which cut is fastest depends on the tile order b, the
bandwidth w, the number of arrow block rows, the precision -- and on the
regime the matrix runs in:

* ``batch``: many matrices in one launch (the batched and served forms). The
  probe is several copies of a short matrix of the key in one launch, so that
  the GPU is as loaded as in a real batch; tuned: the plan code.
* ``single``: one long matrix alone on the GPU (a long band chain whose
  factorization is one critical path). The probe is one matrix of
  ``nt_single`` tile columns launched alone; tuned: the plan code and the
  persistent CTAs per SM (two, or one so that each worker has its SM's FP64
  pipe to itself).

Each batch key keeps the fastest candidate on its probe; a single key keeps
the defaults unless a candidate beats them by SINGLE_MARGIN. Results are
cached in a JSON file, keyed ``b:w:arrow_blocks:precision`` (batch) or
``b:w:arrow_blocks:precision:single``.
"""
from __future__ import annotations

import json
import os
from typing import Dict, Iterable, Optional, Tuple

from . import stiles as S
from . import workloads as W

# chunk of old update terms (bits 0-1) x phase-2 split (bits 2-3) x newest-update split (bits 4-5)
CANDIDATES = (0, 1, 2, 4, 8, 16, 4 + 16, 2 + 8 + 16)
GRID_PER_SM = (2, 1)  # persistent CTAs per SM tried in the single regime
FB = 64
# A short probe stands in for a long matrix only roughly: in the single
# regime a candidate replaces the defaults (code 0, two CTAs per SM) only if
# it beats them on the probe by more than this fraction (measured repeat
# spread of the probe is below 1 %; picks within 0.3 % of the default were
# 7 % slower on the n = 204,864 matrix).
SINGLE_MARGIN = 0.03


def default_cache_path() -> str:
    """The tuning file shipped with the package (codes measured on GB300),
    used as the starting cache; keys it lacks are tuned and added."""
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_gb300.json")


def key_of(b: int, w: int, a: int, precision: int, regime: str = "batch") -> str:
    base = f"{b}:{w}:{(a + FB - 1) // FB}:{precision}"
    return base if regime == "batch" else f"{base}:{regime}"


class Autotuner:
    def __init__(self, cache_path: Optional[str] = None, nt_probe: int = 12, copies: int = 8, reps: int = 2,
                 candidates: Iterable[int] = CANDIDATES, device: str = "cuda", nt_single: int = 24):
        self.cache_path = cache_path
        self.nt_probe, self.copies, self.reps = nt_probe, copies, reps
        self.nt_single = nt_single
        self.candidates = tuple(candidates)
        self.device = device
        self.cache: Dict[str, dict] = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                self.cache = json.load(f)

    def save(self) -> None:
        if self.cache_path:
            tmp = self.cache_path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.cache, f, indent=1, sort_keys=True)
            os.replace(tmp, self.cache_path)

    def best(self, b: int, w: int, a: int, precision: int = S.STILES_FP64) -> int:
        """Plan code for a matrix of this key in a batch."""
        k = key_of(b, w, a, precision)
        if k not in self.cache:
            code, times = self.tune(b, w, a, precision)
            self.cache[k] = {"code": code, "seconds": {str(c): t for c, t in times.items()}}
            self.save()
        return int(self.cache[k]["code"])

    def codes_for(self, shapes, precision: int = S.STILES_FP64):
        return [self.best(b, w, a, precision) for (_, b, w, a) in shapes]

    def best_single(self, b: int, w: int, a: int, precision: int = S.STILES_FP64) -> Tuple[int, int]:
        """(plan code, CTAs per SM) for one long matrix of this key alone."""
        k = key_of(b, w, a, precision, "single")
        if k not in self.cache:
            (code, grid), times = self.tune_single(b, w, a, precision)
            self.cache[k] = {"code": code, "grid_per_sm": grid,
                             "seconds": {f"{c}/{g}": t for (c, g), t in times.items()}}
            self.save()
        e = self.cache[k]
        return int(e["code"]), int(e.get("grid_per_sm", 2))

    def cached(self, b: int, w: int, a: int, precision: int, regime: str = "batch"):
        """The cached entry of a key, or None (no tuning run)."""
        return self.cache.get(key_of(b, w, a, precision, regime))

    def tune(self, b: int, w: int, a: int, precision: int) -> Tuple[int, Dict[int, float]]:
        """Time every candidate code on the probe batch; returns (best code,
        {code: seconds per launch})."""
        import torch

        nt = max(self.nt_probe, w + 1)
        shapes = [(nt, b, w, a)] * self.copies
        A = None
        times: Dict[int, float] = {}
        for code in self.candidates:
            bt = S.StilesBatch(shapes, device=self.device, precision=precision, tuning=[code] * self.copies)
            try:
                if A is None:
                    A = torch.empty(bt.doubles, dtype=torch.float64, device=bt.device)
                    for m in range(self.copies):
                        lay = bt.layouts[m]
                        W.random_arrowhead_packed(nt, b, w, a, 500 + m, A[bt.off[m]:bt.off[m] + lay.doubles])
                bt.A = A
                bt.factor_selinv()  # warm-up (and the graph build)
                torch.cuda.synchronize(bt.device)
                if any(bt.status(m)[0] != S.STILES_OK for m in range(self.copies)):
                    raise RuntimeError(f"autotune probe failed for code {code}")
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(self.reps):
                    bt.factor_selinv()
                e1.record()
                torch.cuda.synchronize(bt.device)
                times[code] = e0.elapsed_time(e1) / 1e3 / self.reps
            finally:
                bt.A = None
                bt.close()
        best = min(times, key=times.get)
        return best, times

    @staticmethod
    def pick_single(times: Dict[Tuple[int, int], float]) -> Tuple[int, int]:
        """The fastest (code, CTAs per SM), unless the defaults are within
        SINGLE_MARGIN of it."""
        best = min(times, key=times.get)
        default = times.get((0, 2))
        if default is not None and times[best] > (1.0 - SINGLE_MARGIN) * default:
            return (0, 2)
        return best

    def tune_single(self, b: int, w: int, a: int, precision: int) -> Tuple[Tuple[int, int], Dict]:
        """Time every (code, CTAs per SM) on one matrix of nt_single tile
        columns launched alone; returns ((code, grid per SM), {(code, grid):
        seconds per launch})."""
        import torch

        nt = max(self.nt_single, w + 1)
        M = None
        A = None
        times: Dict[Tuple[int, int], float] = {}
        for code in self.candidates:
            st = S.Stiles(nt, b, w, a, device=self.device, precision=precision, tuning=code)
            try:
                if A is None:
                    M = W.random_arrowhead(nt, b, w, a, seed=700)
                    A = st.upload(M).A
                else:
                    st.A = A
                sms = torch.cuda.get_device_properties(st.device).multi_processor_count
                for g in GRID_PER_SM:
                    S.stiles_set_option(st.h, S.STILES_OPT_GRID, g * sms)
                    st.factor_selinv()
                    torch.cuda.synchronize(st.device)
                    if st.status()[0] != S.STILES_OK:
                        raise RuntimeError(f"autotune probe failed for code {code}, {g} CTAs per SM")
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    for _ in range(self.reps):
                        st.factor_selinv()
                    e1.record()
                    torch.cuda.synchronize(st.device)
                    times[(code, g)] = e0.elapsed_time(e1) / 1e3 / self.reps
            finally:
                st.A = None
                st.close()
        return self.pick_single(times), times
