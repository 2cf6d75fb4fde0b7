"""Host-side parts of bench.py, on the CPU: the committed sweep capture still
describes the sweep sources (so the bench's `traffic` is not null), the job
value and environment helpers, and the oracle timings that the stage reports
carry (run here on a small synthetic field with the same structure as the
bench's).
"""
import importlib.util
import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_sweep_capture_matches_sources(bench):
    # a change to the sweep's sources needs a new ncu capture of its traffic
    per_node, src = bench.profiled_traffic(-1)
    assert per_node is not None, src
    assert 8.0 < per_node < 10.0  # 8 B of psi per node plus halo, overlap and records
    assert bench.profiled_traffic(0)[0] is None  # no capture of the nibble sweep


def test_job_value_and_env(bench, monkeypatch):
    # all ranks' grid points over the slowest rank's time
    assert bench.job_value(4, 512 ** 3, 10, 2.0) == pytest.approx(4 * 512 ** 3 * 10 / 2e-3)
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (1, 0, 0)
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench.dist_env() == (2, 1, 1)


def test_stage_baselines_on_a_small_field(bench):
    shape = (40, 96, 96)
    psi = synth.random_waves_numpy(shape, synth.wave_spec(7, 1024))
    w, _ = oracle.identify(psi)
    ids, wn = oracle.face_list(w)
    xyz = oracle.localize(psi, ids, wn)["xyz"]
    F = len(ids)
    out = bench.oracle_stage_baselines(
        torch.from_numpy(psi), torch.from_numpy(ids.view(np.int64).copy()),
        torch.from_numpy(wn.copy()), torch.from_numpy(xyz.astype(np.float32)), F,
        planes=16, nref=500)
    assert set(out) == {"node_form", "refine", "face_graph", "lines"}
    for v in out.values():
        assert v["kind"] == "oracle" and v["value"] > 0 and v["cores"] >= 1 and v["sample"]
    # the refinement sample stays inside the slab: centres of the first 12 planes
    assert "of the first 12 planes" in out["refine"]["sample"]
