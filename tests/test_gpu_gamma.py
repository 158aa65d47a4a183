"""GPU gamma index (dc_gamma_index, through the C ABI) against the FP64 oracle
(oracle/gamma.py).  The kernel evaluates the same minimum over the same
whole-voxel offsets in FP32, so gamma agrees to about 1e-5; the statistics use
the same 50 % isodose set (exactly), and a pass decision may flip only for a
voxel whose gamma lies within that rounding of 1."""
import numpy as np
import pytest

from oracle import gamma as og
from paper_1103_1164_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1103_1164_gb300 import build, dc_fspb
    build.build()
    dc_fspb.load()
    return dc_fspb


def _fields(shape, seed):
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(*(np.linspace(0, 1, n) for n in shape), indexing="ij")
    ref = np.exp(-((x - 0.5) ** 2 + (y - 0.4) ** 2) / 0.08) * (1.2 - 0.4 * z) + 0.02
    ev = 1.02 * np.roll(ref, 1, axis=2) + rng.normal(0, 0.01, shape)
    return ref.astype(np.float32), ev.astype(np.float32)


def _check(gamma, st, ref, ev, spacing, pct, dta, radius):
    want = og.gamma_index(ref, ev, spacing, pct=pct, dta=dta, radius=radius)
    assert np.abs(gamma - want).max() < 2e-5 + 1e-5 * want.max()
    gmax, gavg, p50, n50 = og.gamma_stats(want, ref)
    assert st["n50"] == n50
    assert abs(st["gamma_max"] - gmax) < 1e-4
    assert abs(st["gamma_avg50"] - gavg) < 1e-5
    near = int((np.abs(want.ravel()[ref.ravel() >= 0.5 * ref.max()] - 1.0) < 1e-4).sum())
    assert abs(st["pass50_pct"] - p50) <= 100.0 * near / max(n50, 1) + 1e-9


@pytest.mark.parametrize("shape,vox,pct,dta,radius", [((12, 14, 16), 0.25, 3.0, 0.3, 1.5),
                                                      ((9, 17, 23), 0.2, 2.0, 0.2, 0.7),
                                                      ((1, 1, 40), 0.25, 3.0, 0.3, 0.3),
                                                      ((20, 3, 5), 0.3, 5.0, 0.5, 2.5)])
def test_gamma_matches_oracle(dc, shape, vox, pct, dta, radius):
    ref, ev = _fields(shape, seed=sum(shape))
    g = synth.centred_grid(shape[2], shape[1], shape[0], vox)
    gamma, st = dc.dc_gamma_index(ref, ev, g, pct=pct, dta=dta, search=radius)
    _check(gamma, st, ref, ev, (vox, vox, vox), pct, dta, radius)


def test_gamma_fspb_against_dc_fspb_and_device_buffers(dc):
    # the density correction's effect on a small slab plan, measured by gamma
    import torch
    p = synth.small_plan(7, n=(24, 20, 16), vox=0.25, n_beams=2, phantom="slab", roi=1.5, field=3.0)
    q = synth.small_plan(7, n=(24, 20, 16), vox=0.25, n_beams=2, phantom="slab", roi=1.5, field=3.0,
                         density_correction=0)
    ref = dc.dc_fspb_dose(dc.dc_fspb_create_from(p), p.fluence).astype(np.float32)
    ev = dc.dc_fspb_dose(dc.dc_fspb_create_from(q), q.fluence).astype(np.float32)
    gamma, st = dc.dc_gamma_index(ref, ev, p.grid)
    _check(gamma, st, ref, ev, (0.25, 0.25, 0.25), 3.0, 0.3, 1.5)
    gd, sd = dc.dc_gamma_index(torch.from_numpy(ref).cuda(), torch.from_numpy(ev).cuda(), p.grid)
    assert np.array_equal(gd.cpu().numpy(), gamma) and sd == st


def test_gamma_full_size_sampled(dc):
    # DC-FSPB against FSPB on the 128 x 128 x 96 thorax plan; the oracle on
    # seeded voxels (half of them inside the 50 % isodose)
    import torch
    p = synth.config2()
    ref = torch.empty(p.grid.shape, device="cuda")
    ev = torch.empty(p.grid.shape, device="cuda")
    dc.dc_fspb_dose(dc.dc_fspb_create_from(p), torch.from_numpy(p.fluence).cuda(), ref)
    p.comm.density_correction = 0
    dc.dc_fspb_dose(dc.dc_fspb_create_from(p), torch.from_numpy(p.fluence).cuda(), ev)
    gamma, st = dc.dc_gamma_index(ref, ev, p.grid)
    r, e, gm = ref.cpu().numpy(), ev.cpu().numpy(), gamma.cpu().numpy()
    rng = np.random.default_rng(8)
    hot = np.flatnonzero(r.ravel() >= 0.5 * r.max())
    vox = np.unique(np.concatenate([rng.integers(0, r.size, 600), rng.choice(hot, 600)]))
    want = og.gamma_at(r, e, (0.25, 0.25, 0.25), vox)
    assert np.abs(gm.ravel()[vox] - want).max() < 5e-5
    assert st["gamma_max"] == pytest.approx(float(gm.max()), abs=1e-6)
    assert st["n50"] == hot.size


def test_gamma_rejects_bad_arguments(dc):
    ref, ev = _fields((4, 5, 6), 1)
    g = synth.centred_grid(6, 5, 4, 0.25)
    with pytest.raises(dc.DcError):
        dc.dc_gamma_index(np.zeros_like(ref), ev, g)               # zero reference
    with pytest.raises(dc.DcError):
        dc.dc_gamma_index(ref, ev, g, dta=0.3, search=0.2)          # search < dta
    with pytest.raises(dc.DcError):
        dc.dc_gamma_index(ref, ev, g, dta=0.3, search=20.0)         # > 64 voxels
