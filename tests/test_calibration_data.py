"""The committed calibration against its tables (CPU only).

The fitted parameter files, the measured tables and the reports are records
of GPU runs; these checks tie them together with the FP64 oracle, so a
parameter file that no longer matches its table, or a report that was not
written from that table and file, fails here:
  * the committed theta reproduces the report's per-family MAE on the table
    it was fitted on (the GPU model matches the oracle to 1e-5 relative, far
    below the 0.05-point tolerance);
  * it predicts the second table, measured on another box with the same
    kernels, about as well (the reproducibility claim of the calibration).
"""
import json
import os

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DATA = os.path.join(ROOT, "paper_2605_04178_gb300", "data")
N_SM = 152
FIELDS = ("M", "N", "K", "BM", "BN", "BK", "stages", "cta_group", "dtype", "kind", "tmem_a")


def _load(name):
    with open(os.path.join(DATA, name)) as f:
        return json.load(f)


def _theta(reading=O.READING_MEASURED):
    name = "theta_gb300.json" if reading == O.READING_MEASURED else "theta_gb300_literal.json"
    with open(os.path.join(ROOT, "paper_2605_04178_gb300", name)) as f:
        meta = json.load(f)
    assert meta["reading"] == reading
    th = np.array(meta["theta"], dtype=np.float64)
    assert th.size == O.N_PARAMS
    return th


def _family(r):
    if "launch" in r and "G" in r:
        return "grouped"
    if r["kind"] in (O.KIND_COPY, O.KIND_TRIAD):
        return "stream"
    if r["kind"] == O.KIND_TMA2D:
        return "tma"
    fam = {O.DT_FP32: "fp32", O.DT_BF16: "bf16", O.DT_FP8: "fp8"}[int(r["dtype"])]
    return fam + "_tmemB" if r.get("tmem_a", 0) else fam


def _mae_by_family(table, th):
    rows = table["rows"]
    cols = {f: np.array([r.get(f, 0) for r in rows], dtype=np.int32) for f in FIELDS}
    pred = list(O.model_batch(cols, th, N_SM))
    fams = [_family(r) for r in rows]
    t = [r["t"] for r in rows]
    for r in table.get("grouped", []):
        pred.append(O.grouped_predict(r["M"], r["N"], r["K"], r["bm"], r["bn"], *r["launch"], O.DT_BF16, th, N_SM))
        fams.append("grouped")
        t.append(r["t"])
    ape = np.abs(np.array(pred) - np.array(t)) / np.array(t) * 100.0
    fams = np.array(fams)
    out = {f: float(ape[fams == f].mean()) for f in sorted(set(fams))}
    out["all"] = float(ape.mean())
    return out


@pytest.fixture(scope="module")
def measured_reading():
    prev = O.reading()
    O.set_reading(O.READING_MEASURED)
    yield
    O.set_reading(prev)


def test_theta_reproduces_its_report(measured_reading):
    th = _theta()
    report = _load("calib_report_gb300.json")
    assert report["reading"] == O.READING_MEASURED
    assert np.allclose(report["theta"], th, rtol=1e-12, atol=0)
    got = _mae_by_family(_load("sweep_gb300.json"), th)
    for fam, v in report["mae_all"].items():
        assert got[fam] == pytest.approx(v["mae_pct"], abs=0.05), fam


def test_theta_predicts_the_second_box(measured_reading):
    th = _theta()
    own = _mae_by_family(_load("sweep_gb300.json"), th)
    other = _mae_by_family(_load("sweep_gb300_second_box.json"), th)
    assert other["all"] <= 6.5
    for fam in own:
        assert abs(other[fam] - own[fam]) <= 1.0, (fam, own[fam], other[fam])


def test_literal_theta_reproduces_its_report():
    prev = O.reading()
    O.set_reading(O.READING_LITERAL)
    try:
        th = _theta(O.READING_LITERAL)
        report = _load("calib_report_gb300_literal.json")
        assert report["reading"] == O.READING_LITERAL
        assert np.allclose(report["theta"], th, rtol=1e-12, atol=0)
        got = _mae_by_family(_load("sweep_gb300.json"), th)
        for fam, v in report["mae_all"].items():
            assert got[fam] == pytest.approx(v["mae_pct"], abs=0.05), fam
    finally:
        O.set_reading(prev)
