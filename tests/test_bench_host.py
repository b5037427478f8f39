"""Host-side helpers of bench.py that need no GPU: the 4-thread oracle sample
run in a child process, and its failure path (the headline line never depends
on it)."""
from __future__ import annotations

import os
import sys
from types import SimpleNamespace

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

D200 = SimpleNamespace(nocc=380, nvir=1520, naux_k=100)


def test_four_thread_oracle_sample_runs_in_a_child():
    r = bench.cpu_baseline_threads(4, D200, 259.0, budget_s=1.0)
    assert "unavailable" not in r, r
    assert r["cores"] == 4 and r["kind"] == "oracle" and r["unit"] == "matvecs/s"
    assert r["value"] > 0.0 and r["s_per_step_extrapolated"] > 0.0


def test_failing_child_reports_unavailable():
    # dimensions the sample cannot use: the child fails, the helper returns a note
    r = bench.cpu_baseline_threads(4, SimpleNamespace(nocc=0, nvir=0, naux_k=0), 259.0, budget_s=1.0,
                                   timeout_s=120.0)
    assert set(r) == {"unavailable"}


def test_child_sample_uses_the_parents_case():
    # the 100-atom profiling case (50 heavy + 50 H, nao 950, nocc 190): the child
    # must build that molecule, not the 200-atom one, for these dimensions to fit
    r = bench.cpu_baseline_threads(4, SimpleNamespace(nocc=190, nvir=760, naux_k=50), 100.0, budget_s=1.0,
                                   case="small")
    assert "unavailable" not in r, r
    assert "of the 50 heavy atoms" in r["sample"]
