"""Host side of the commissioning fit: the tables' Jacobian with respect to
the model parameters (used to carry the kernels' table gradients to the
parameters) against central finite differences of the tables themselves."""
import numpy as np

from paper_1103_1164_gb300 import commission as cmn, synth


def test_table_jacobian_matches_finite_differences():
    cm = synth.make_commissioning()
    th = synth.model_params()
    _, _, jw, jd = cmn.tables_and_jacobian(th, cm)
    w_n, f_n = cm.water.shape[1], cm.dens.shape[1]
    for k in cmn.PARAMS:
        if k in ("beta1", "beta2"):
            continue            # b enters the fit through the kernels' scale gradient
        h = 1e-6 * max(abs(th[k]), 1e-3)
        up, dn = dict(th), dict(th)
        up[k] += h
        dn[k] -= h
        wu, du = synth.model_tables(up, cm.w_dt, w_n, cm.f_rho0, cm.f_drho, f_n)
        wd, dd = synth.model_tables(dn, cm.w_dt, w_n, cm.f_rho0, cm.f_drho, f_n)
        fw, fd = (wu - wd) / (2 * h), (du[:4] - dd[:4]) / (2 * h)
        assert np.allclose(jw[k], fw, rtol=1e-6, atol=1e-7 * max(1.0, np.abs(fw).max())), k
        assert np.allclose(jd[k], fd, rtol=1e-6, atol=1e-7 * max(1.0, np.abs(fd).max())), k


def test_model_tables_reproduce_the_commissioning():
    cm = synth.make_commissioning()
    w, d = synth.model_tables(synth.model_params(), cm.w_dt, cm.water.shape[1], cm.f_rho0, cm.f_drho,
                              cm.dens.shape[1])
    assert np.array_equal(w.astype(np.float32), cm.water)
    assert np.array_equal(d.astype(np.float32), cm.dens)


def test_slab_phantom_follows_the_commissioning_geometry():
    # Section 2.1: 30 cm cube, a 15 cm slab 8 cm below the surface, 10 x 10 cm2
    # field, SAD 100 cm, SSD 90 cm
    p = cmn.slab_phantom(0.3)
    g = p.grid
    assert (g.nx, g.ny, g.nz) == (60, 60, 60) and g.dx == 0.5
    y = g.oy + g.dy * np.arange(g.ny) - (g.oy - 0.5 * g.dy)      # depth of each voxel row
    col = p.rho[g.nz // 2, :, g.nx // 2]
    assert np.all(col[(y >= 8.0) & (y < 23.0)] == np.float32(0.3))
    assert np.all(col[(y < 8.0) | (y >= 23.0)] == 1.0)
    b = p.beams[0]
    src_y = b.iso[1] - b.sad
    assert abs((g.oy - 0.5 * g.dy) - src_y - 90.0) < 1e-9
    assert p.n_beamlets == 400
