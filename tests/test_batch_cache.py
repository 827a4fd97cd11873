"""CPU checks of the batch autotuner's cache: a choice stored for (device, p, m, precision,
batch size) is returned from the JSON file without timing anything (no GPU needed), and
entries of an older two-field form are not taken as choices."""
import json

import pytest

torch = pytest.importorskip("torch")

from paper_2009_01499_gb300 import batch, iga2l  # noqa: E402


def test_cached_choice_is_returned_without_timing(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    key = batch._key(3, 64, iga2l.MIXED_FP32, 6)
    choice = [iga2l.SCHED_TILE, 2, iga2l.SWEEP_WORK_LIST]
    path.write_text(json.dumps({key: choice}))
    monkeypatch.setattr(batch, "_cache", {})

    def no_solver(*a, **k):
        raise AssertionError("the autotuner timed a candidate although the choice was cached")

    monkeypatch.setattr(iga2l, "Solver", no_solver)
    assert batch.autotune_schedule(3, 64, iga2l.MIXED_FP32, cache_path=str(path), nbatch=6) == choice
    # a different batch size is a different key
    assert batch._key(3, 64, iga2l.MIXED_FP32, 6) != batch._key(3, 64, iga2l.MIXED_FP32, 1)


def test_old_two_field_entries_are_not_choices(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    key = batch._key(2, 128, iga2l.FP64, 1)
    path.write_text(json.dumps({key: [iga2l.SCHED_LATTICE, 0]}))
    monkeypatch.setattr(batch, "_cache", {})
    calls = []

    def record(*a, **k):
        calls.append(k)
        raise RuntimeError("stop before any GPU work")

    monkeypatch.setattr(iga2l, "Solver", record)
    with pytest.raises(RuntimeError):
        batch.autotune_schedule(2, 128, iga2l.FP64, cache_path=str(path))
    assert calls   # the stale entry was not returned: the autotuner went on to time candidates


def test_candidates_cover_the_documented_forms():
    forms = set(batch.CANDIDATES)
    assert (iga2l.SCHED_LATTICE, 0, iga2l.SWEEP_AUTO) in forms
    for groups in (1, 2, 4):
        for sweep in (iga2l.SWEEP_AUTO, iga2l.SWEEP_WORK_LIST):
            assert (iga2l.SCHED_TILE, groups, sweep) in forms
    assert len(forms) == len(batch.CANDIDATES) == 7
