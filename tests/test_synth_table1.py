"""The synthetic Table 1 cases follow the table's case dimensions (host only)."""
import os

import numpy as np
import pytest

from paper_1103_1164_gb300 import synth

TESTS = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(TESTS, "golden")


def _tsv(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_table1_constants_match_the_printed_table():
    printed = {r[0]: (int(r[1]), bool(int(r[2])), int(r[3]), (int(r[4]), int(r[5]), int(r[6])))
               for r in _tsv("table1_cases.tsv")}
    assert set(printed) == {c[0] for c in synth.TABLE1}
    for name, _, nb, noncop, n_bl, nz, _ in synth.TABLE1:
        assert printed[name] == (nb, noncop, n_bl, (128, 128, nz)), name


def test_table4_times_in_the_bench_match_the_printed_table():
    import sys
    sys.path.insert(0, os.path.dirname(TESTS))
    import bench
    printed = {r[0]: float(r[1]) for r in _tsv("table4_tgpu.tsv")}
    assert bench.TABLE4_TGPU_S == printed


@pytest.mark.parametrize("row", synth.TABLE1, ids=[r[0] for r in synth.TABLE1])
def test_case_matches_table1_dimensions(row):
    name, _, n_beams, noncop, n_beamlets, nz, tumour = row
    p = synth.table1_case(name)
    assert (p.grid.nx, p.grid.ny, p.grid.nz) == (128, 128, nz)
    assert (p.grid.dx, p.grid.dy, p.grid.dz) == synth.TABLE1_VOXEL
    assert (p.beamlet_x, p.beamlet_y) == synth.TABLE1_BEAMLET
    assert len(p.beams) == n_beams
    # beamlet count within 3 beamlets (0.5 %) of the table's
    assert abs(p.n_beamlets - n_beamlets) <= 3
    couches = [b.couch_deg for b in p.beams]
    assert any(c != 0.0 for c in couches) == noncop
    for b in p.beams:
        assert tuple(b.iso) == tumour
        nx, ny = b.field_x / p.beamlet_x, b.field_y / p.beamlet_y
        assert abs(nx - round(nx)) < 1e-9 and abs(ny - round(ny)) < 1e-9
    assert p.rho.shape == (nz, 128, 128) and p.rho.dtype == np.float32
    assert p.fluence.shape == (p.n_beamlets,)
    assert float(p.rho.min()) > 0.0


def test_cases_are_seeded():
    a, b = synth.table1_case("H2"), synth.table1_case("H2")
    assert np.array_equal(a.rho, b.rho) and np.array_equal(a.fluence, b.fluence)
    assert a.beams == b.beams


def test_lung_tumour_is_water_in_lung():
    p = synth.table1_case("L5")
    g = p.grid
    x, y, z = synth.TABLE1[9][6]
    i, j, k = (int(round((x - g.ox) / g.dx)), int(round((y - g.oy) / g.dy)),
               int(round((z - g.oz) / g.dz)))
    assert p.rho[k, j, i] == 1.0
    # lung tissue 2.5 cm further out along x
    assert p.rho[k, j, i + int(round(2.5 / g.dx))] < 0.4
