"""Host logic of the batch autotuner (no GPU): the size classes, the coordinate
descent over launch choices against synthetic timings, and the committed choice
file against the 256-instance workload it was measured on."""
import json
import math
from types import SimpleNamespace

import pytest

import pdhg_workloads as W
from paper_2207_07234_gb300 import autotune as A


def _smallest_pow2_log(v):
    r = 0
    while (1 << r) < v:
        r += 1
    return r


@pytest.mark.parametrize("nx", [256, 257, 300, 511, 512, 513, 1000, 1024, 2047, 2048, 2049, 3000, 4095, 4096])
def test_size_class_is_row_transform_log2_minus_8(nx):
    # the row transform of a 1D finite-difference instance: Bluestein of length
    # 2^ceil(log2(2 nx - 1)) for nx not a power of two, else the packed real FFT of nx/2
    p = SimpleNamespace(nx=nx, nmodes=1)
    pow2 = nx & (nx - 1) == 0
    L = _smallest_pow2_log(2 * nx - 1) if not pow2 else _smallest_pow2_log(nx // 2)
    assert A.size_class(p) == min(7, max(0, L - 8))
    if pow2:
        assert 1 << (A.size_class(p) + 8) == max(nx // 2, 256)


def test_size_class_dg_uses_the_packed_length():
    # DG instances take power-of-two cell counts only; their class follows nx/2
    assert A.size_class(SimpleNamespace(nx=512, nmodes=3)) == 0
    assert A.size_class(SimpleNamespace(nx=4096, nmodes=2)) == 3


def _surface(per_stage, persistent_base, tile_gain, unsupported_bps=()):
    """ms = per_stage for the per-stage launches; persistent: base[(order, bps)] minus
    tile_gain[class][tile] summed over classes (a separable synthetic surface)."""
    calls = []

    def measure(persistent, bps, order, tiles):
        calls.append((persistent, bps, order, tuple(tiles)))
        if not persistent:
            return per_stage
        if bps in unsupported_bps:
            raise RuntimeError("does not fit")
        ms = persistent_base[(order, bps)]
        for c, g in enumerate(tiles):
            ms -= tile_gain.get(c, {}).get(g, 0.0)
        return ms
    return measure, calls


def test_search_finds_the_separable_minimum():
    base = {(o, b): 30.0 - 2 * b - 0.5 * o for o in (0, 1) for b in (0, 1, 2, 3)}      # best: order 1, 3 blocks
    gain = {2: {4: 3.0, 8: 1.0}, 5: {2: 0.5, 8: 2.5}, 6: {8: 9.0}}                     # class 6 absent
    measure, calls = _surface(40.0, base, gain)
    res = A.search(measure, present=[2, 3, 5])
    assert (res["order"], res["blocks_per_sm"]) == (1, 3)
    assert res["tiles"] == [1, 1, 4, 1, 1, 8, 1, 1]
    assert math.isclose(res["persistent_ms"], 30.0 - 6 - 0.5 - 3.0 - 2.5)
    assert res["persistent"] is True and res["per_stage_ms"] == 40.0
    # one per-stage timing, 8 (order, blocks) timings, 3 tiles tried per present class
    assert len(calls) == 1 + 8 + 3 * 3
    assert all(t[6] == 1 for (_, _, _, t) in calls)                                    # absent class untouched


def test_search_keeps_the_per_stage_launches_when_faster():
    base = {(o, b): 20.0 for o in (0, 1) for b in (0, 1, 2, 3)}
    measure, _ = _surface(16.4, base, {3: {8: 1.0}})
    res = A.search(measure, present=[3])
    assert res["persistent"] is False
    assert res["tiles"][3] == 8 and math.isclose(res["persistent_ms"], 19.0)


def test_search_skips_choices_that_do_not_fit():
    base = {(o, b): 25.0 - b for o in (0, 1) for b in (0, 1, 2, 3)}
    measure, calls = _surface(30.0, base, {}, unsupported_bps=(3,))
    res = A.search(measure, present=[], unsupported=(RuntimeError,))
    assert res["blocks_per_sm"] == 2 and res["persistent_ms"] == 23.0 and res["persistent"]
    with pytest.raises(RuntimeError):                                                   # not listed: propagates
        A.search(measure, present=[])


def test_search_when_no_persistent_form_fits():
    base = {(o, b): 1.0 for o in (0, 1) for b in (0, 1, 2, 3)}
    measure, _ = _surface(12.0, base, {}, unsupported_bps=(0, 1, 2, 3))
    res = A.search(measure, present=[4], unsupported=(RuntimeError,))
    assert res["persistent"] is False and res["persistent_ms"] is None and res["per_stage_ms"] == 12.0
    assert res["tiles"] == [1] * 8


def test_committed_choice_matches_its_workload():
    with open(A.TILES_FILE) as f:
        cfg = json.load(f)
    assert len(cfg["tiles"]) == 8 and all(int(g) in (1, 2, 4, 8) for g in cfg["tiles"])
    assert cfg["order"] in (0, 1) and 0 <= cfg["blocks_per_sm"] <= 3
    assert cfg["persistent"] == (cfg["persistent_ms"] < cfg["per_stage_ms"])
    present = sorted({A.size_class(p) for p in W.batch_instances()})
    assert cfg["classes_present"] == present
    # the recorded timings hold the chosen persistent form at the reported time
    chosen = [t for t in cfg["timings"] if t["persistent"] and t["blocks_per_sm"] == cfg["blocks_per_sm"]
              and t["order"] == cfg["order"] and t["tiles"] == cfg["tiles"]]
    assert chosen and math.isclose(min(t["ms"] for t in chosen), cfg["persistent_ms"])
    assert math.isclose(min(t["ms"] for t in cfg["timings"] if t["persistent"]), cfg["persistent_ms"])
