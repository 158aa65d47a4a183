"""Checkpoint files on the host: the CSR matrix and the commissioning tables
survive a round trip unchanged, and malformed files are refused."""
import json

import numpy as np
import pytest

from paper_1103_1164_gb300 import checkpoint as ck, synth


def test_csr_round_trip(tmp_path):
    rng = np.random.default_rng(0)
    counts = rng.integers(0, 5, 50)
    rowptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    nnz = int(rowptr[-1])
    cols = rng.integers(0, 30, nnz).astype(np.int32)
    for vals in (rng.uniform(0, 1, nnz).astype(np.float32), rng.integers(0, 65535, nnz).astype(np.uint16)):
        path = str(tmp_path / "m.npz")
        ck.save_csr(path, rowptr, np.concatenate([cols, [7, 7]]), np.concatenate([vals, vals[:2]]), 30,
                    meta={"plan": "test"})
        r, c, v, h = ck.load_csr(path)
        assert np.array_equal(r, rowptr) and np.array_equal(c, cols) and np.array_equal(v, vals)
        assert v.dtype == vals.dtype and h["cols"] == 30 and h["meta"] == {"plan": "test"}


def test_commissioning_round_trip_and_refusals(tmp_path):
    cm = synth.make_commissioning(5, roi_radius=2.5, smooth_sigma=0.4)
    path = str(tmp_path / "c.npz")
    ck.save_commissioning(path, cm)
    back = ck.load_commissioning(path)
    for k in ("A", "water", "dens"):
        assert np.array_equal(getattr(back, k), getattr(cm, k))
    for k in ("a_dt", "a_dtheta", "w_dt", "f_rho0", "f_drho", "roi_radius", "smooth_sigma", "rho_surface",
              "density_correction"):
        assert getattr(back, k) == getattr(cm, k)
    with pytest.raises(ValueError):
        ck.load_csr(path)                                    # another format
    bad = str(tmp_path / "bad.npz")
    np.savez(bad, header=json.dumps({"format": ck.CSR_FORMAT, "rows": 3, "cols": 2, "nnz": 5, "values": "f32"}),
             rowptr=np.array([0, 1, 2, 3], np.int64), cols=np.zeros(3, np.int32), vals=np.zeros(3, np.float32))
    with pytest.raises(ValueError):
        ck.load_csr(bad)                                     # arrays disagree with the header
