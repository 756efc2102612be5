"""Host checks of bench.py's roofline bookkeeping (no GPU): the algorithmic bytes per
stage on the benchmark workload, the 32 B per cell-iteration of one pass of the path,
and the lookup of the committed ncu DRAM counters, which must refuse counters taken on
another version of the kernel source."""
import hashlib
import json
import os
import shutil

import pytest

import bench
import pdhg_workloads as W


def test_fused_stage_bytes_on_the_benchmark_workload():
    p = bench.workload("burgers2d")
    assert (p.nx, p.ny, p.nt) == (1024, 1024, 256)
    sb = bench.stage_bytes(p, 4)
    cells = p.cells_per_iter
    # counted by hand from the array shapes: u has nt + 1 slices, phi and phit nt, the
    # half spectrum nx/2 + 1 complex float32 values per row of every slice
    u, f = (p.nt + 1) * p.ndof * 4, p.nt * p.ndof * 4
    spec = p.nt * p.ny * (p.nx // 2 + 1) * 8
    assert sb["primal"] == 2 * u + f + 5 * p.ndof * 4
    assert sb["fused_rows"] == u + spec
    assert sb["fused_cols"] == 4 * spec
    assert sb["dual"] == spec + 3 * f
    per_cell = sum(sb[k] for k in ("primal", "fused_rows", "fused_cols", "dual")) / cells
    assert 52.0 <= per_cell <= 52.0 * 1.005, per_cell        # 12 + 8 + 16 + 16, plus O(1/nt, 1/nx)


def test_one_pass_of_the_path_is_32_bytes_per_cell_in_float32():
    # u read and written, phit read (primal); the spill of the t-solve written and read
    # back; phi read and written, phit written (dual): 3 + 2 + 3 words per cell-iteration
    assert bench.ALG_BYTES_PER_CELL[4] == (3 + 2 + 3) * 4
    assert bench.ALG_BYTES_PER_CELL[8] == (3 + 2 + 3) * 8


def test_plain_stage_bytes_cover_every_stage():
    p = W.burgers_2d(n=64, nt=8)
    sb = bench.stage_bytes(p, 8)
    for k in ("primal", "residual_fft", "fft_y", "tsolve", "dual"):
        assert sb[k] > 0
    assert sb["tsolve"] == 2 * sb["fft_y"]


def test_traffic_lookup_follows_the_kernel_source(tmp_path, monkeypatch):
    with open(os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")) as fh:
        db = json.load(fh)
    name = "burgers2d_1024x1024x256"
    for stage, ent in db[name].items():
        src = os.path.join(bench.ROOT, "paper_2207_07234_gb300", "csrc", bench.FUSED_SOURCES[stage])
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        got = bench.traffic_for(stage, name, fused=True)
        assert got == (ent["dram_bytes_per_launch"] if ent["src_sha"] == sha else None)
    assert bench.traffic_for("fused_cols", "no_such_workload", fused=True) is None
    # a copy of the tree whose kernel source differs by one byte: counters refused
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    csrc = root / "paper_2207_07234_gb300" / "csrc"
    csrc.mkdir(parents=True)
    shutil.copy(os.path.join(bench.ROOT, "profiles", "ncu_traffic.json"), root / "profiles")
    for fn in set(bench.FUSED_SOURCES.values()):
        shutil.copy(os.path.join(bench.ROOT, "paper_2207_07234_gb300", "csrc", fn), csrc / fn)
    monkeypatch.setattr(bench, "ROOT", str(root))
    same = {s: bench.traffic_for(s, name, fused=True) for s in db[name]}
    with open(csrc / "kernels_fused2d.cu", "ab") as fh:
        fh.write(b"\n")
    for s in db[name]:
        assert bench.traffic_for(s, name, fused=True) is None
        if same[s] is not None:
            assert same[s] == db[name][s]["dram_bytes_per_launch"]


def test_a_failing_optional_leg_is_recorded_not_raised(capsys):
    assert bench.optional_leg("ok", lambda: {"value": 1.0}) == {"value": 1.0}

    def broken():
        raise RuntimeError("device lost")
    out = bench.optional_leg("batch", broken)
    assert out == {"error": "RuntimeError: device lost"}
    assert "batch leg failed" in capsys.readouterr().err
    # the result line keeps such an entry (a dict with content is truthy)
    assert out
