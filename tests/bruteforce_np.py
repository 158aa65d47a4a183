"""Independent float64 NumPy restatement of DC-FSPB, for tiny grids only.

It exists to pin the C oracle (oracle/oracle.c) and shares no code with it.
Every step is computed by a different route from the oracle's:

* beam frame: explicit 3x3 rotation matrices instead of in-place rotations;
* ray path lengths (Algorithm A1 steps 4-6): the ray is intersected with every
  voxel box separately (slab method, brute force over all voxels) instead of
  Siddon's merged plane crossings;
* smoothing (step 1): scipy.ndimage separable correlation with 'nearest'
  boundaries instead of the oracle's 3-D triple sum;
* lookups (steps 9-10): numpy.interp and scipy's RegularGridInterpolator;
* eq. (4): the paper's printed sinh/cosh form instead of the oracle's
  exponential-difference form;
* the axis-stencil lateral form (lateral_mode = 1): all 48 taps of every
  voxel at once through scipy.ndimage.map_coordinates (order 1, edge clamp)
  and a matrix product with the normalised Gaussian weights, instead of the
  oracle's per-tap trilinear loop.
The readings of the paper are the same as the oracle's (they are the
definition under test); the arithmetic route is not.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import ndimage
from scipy.interpolate import RegularGridInterpolator


def rotation_z(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def rotation_y(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def beam_axes(beam):
    Rm = rotation_y(math.radians(beam.couch_deg)) @ rotation_z(math.radians(beam.gantry_deg))
    ex, ey, ez = Rm @ np.array([1.0, 0, 0]), Rm @ np.array([0, 0, 1.0]), Rm @ np.array([0, 1.0, 0])
    k = math.radians(beam.coll_deg)
    ex, ey = math.cos(k) * ex + math.sin(k) * ey, -math.sin(k) * ex + math.cos(k) * ey
    return ex, ey, ez


def beamlets(plan):
    """Per beamlet: source, unit direction n, lateral axes, theta, beam index."""
    out = []
    for b, beam in enumerate(plan.beams):
        ex, ey, ez = beam_axes(beam)
        iso = np.asarray(beam.iso, float)
        src = iso - beam.sad * ez
        M = int(round(beam.field_x / plan.beamlet_x))
        N = int(round(beam.field_y / plan.beamlet_y))
        for n in range(N):
            for m in range(M):
                a = -beam.field_x / 2 + (m + 0.5) * plan.beamlet_x
                c = -beam.field_y / 2 + (n + 0.5) * plan.beamlet_y
                target = iso + a * ex + c * ey
                nv = (target - src) / np.linalg.norm(target - src)
                theta = math.acos(min(1.0, float(nv @ ez)))
                exx = ex - (ex @ nv) * nv
                exx /= np.linalg.norm(exx)
                eyy = np.cross(exx, nv)
                out.append(dict(src=src, n=nv, ex=exx, ey=eyy, theta=theta, sad=beam.sad, beam=b))
    return out


def voxel_boxes(g):
    x, y, z = g.centres()
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    c = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    h = 0.5 * np.array([g.dx, g.dy, g.dz])
    return c - h, c + h


def ray_voxel_intervals(g, src, n):
    """[enter, exit] of the ray s + a n (a >= 0) in every voxel box (slab method)."""
    lo, hi = voxel_boxes(g)
    with np.errstate(divide="ignore", invalid="ignore"):
        t0 = (lo - src) / n
        t1 = (hi - src) / n
    tmin = np.minimum(t0, t1)
    tmax = np.maximum(t0, t1)
    for a in range(3):
        if abs(n[a]) < 1e-15:
            inside = (src[a] > lo[:, a]) & (src[a] < hi[:, a])
            tmin[:, a] = np.where(inside, -np.inf, np.inf)
            tmax[:, a] = np.where(inside, np.inf, -np.inf)
    enter = np.maximum(tmin.max(1), 0.0)
    exit_ = tmax.min(1)
    return enter, exit_


def tables(plan, g, rho, src, n, d):
    """Entry/exit and exact samples of int rho and int b_i(rho) at t = k d."""
    cm = plan.comm
    enter, exit_ = ray_voxel_intervals(g, src, n)
    seglen = np.maximum(exit_ - enter, 0.0)
    hit = (seglen > 0) & (rho.ravel() > cm.rho_surface)
    if not hit.any():
        return None
    L_in, L_out = enter[hit].min(), exit_[hit].max()
    K = max(2, int(math.ceil((L_out - L_in) / d)) + 1)
    rr = rho.ravel().astype(float)
    rho_dom = cm.f_rho0 + cm.f_drho * np.arange(cm.dens.shape[1])
    b1 = np.interp(rr, rho_dom, cm.dens[4].astype(float))
    b2 = np.interp(rr, rho_dom, cm.dens[5].astype(float))
    sel = seglen > 0
    e, x = enter[sel], exit_[sel]
    T, W1, W2 = np.zeros(K), np.zeros(K), np.zeros(K)
    for k in range(K):
        hi = L_in + k * d
        ov = np.clip(np.minimum(x, hi) - np.maximum(e, L_in), 0.0, None)
        T[k] = ov @ rr[sel]
        W1[k] = ov @ b1[sel]
        W2[k] = ov @ b2[sel]
    return dict(L_in=L_in, L_out=L_out, K=K, T=T, W1=W1, W2=W2)


def smooth(rho, g, sigma):
    out = np.asarray(rho, float)
    for axis, delta in ((2, g.dx), (1, g.dy), (0, g.dz)):
        r = int(math.ceil(3 * sigma / delta)) if sigma > 0 else 0
        j = np.arange(-r, r + 1)
        w = np.exp(-(j * delta) ** 2 / (2 * sigma ** 2)) if sigma > 0 else np.ones(1)
        out = ndimage.correlate1d(out, w / w.sum(), axis=axis, mode="nearest")
    return out


def p_paper(x, u, x0):
    """Eq. (4) exactly as printed (sinh/cosh form)."""
    x = np.asarray(x, float)
    u = np.broadcast_to(np.asarray(u, float), x.shape)
    out = 1.0 - np.cosh(u * x) * np.exp(-u * x0)
    left, right = x < -x0, x > x0
    out = np.where(left, np.sinh(u * x0) * np.exp(u * x), out)
    out = np.where(right, np.sinh(u * x0) * np.exp(-u * x), out)
    return out


def axis_densities(plan, beam, d):
    """Per voxel of the grid, the three densities of the axis-stencil form.

    16 taps at (j - 7.5) d, j = 0..15, along each of the beam's axes e_x', e_y',
    e_z' through the voxel centre; trilinear density with clamp-to-edge; each
    axis averaged with Gaussian weights exp(-s^2 / 2 sigma^2) normalised to
    one.  Returns (mean of the three averages, e_x' average, e_y' average),
    the densities at which f_omega, f_u2 along x and f_u2 along y are read.
    """
    g, cm = plan.grid, plan.comm
    x, y, z = g.centres()
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    r = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    s = (np.arange(16) - 7.5) * d
    sig = cm.smooth_sigma
    wts = np.exp(-s * s / (2 * sig * sig)) if sig > 0 else np.ones(16)
    wts = wts / wts.sum()
    org = np.array([g.ox, g.oy, g.oz])
    dlt = np.array([g.dx, g.dy, g.dz])
    hi = np.array([g.nx, g.ny, g.nz], float) - 1
    rho = plan.rho.astype(float)
    avgs = []
    for ax in beam_axes(beam):
        pts = r[:, None, :] + s[None, :, None] * ax[None, None, :]      # (V, 16, 3)
        idx = np.clip((pts - org) / dlt, 0.0, hi).reshape(-1, 3)
        taps = ndimage.map_coordinates(rho, idx[:, ::-1].T, order=1, mode="nearest")
        avgs.append(taps.reshape(-1, 16) @ wts)
    return (avgs[0] + avgs[1] + avgs[2]) / 3.0, avgs[0], avgs[1]


def dose(plan, fluence=None, density_correction=None, lateral_mode=0):
    """Eq. (1) on every voxel, vectorised over voxels for each beamlet.

    lateral_mode 0: u_2 and omega at rho_hat(r) of the voxel, u_x = u_y (the
    paper's form).  lateral_mode 1: the axis-stencil form (axis_densities):
    u_2 along x at the e_x' average, along y at the e_y' average, omega at the
    mean of the three averages; u_1 stays at rho(r).
    """
    g, cm = plan.grid, plan.comm
    dc = cm.density_correction if density_correction is None else density_correction
    f = plan.fluence if fluence is None else fluence
    rho = plan.rho.astype(float)
    rhos = smooth(rho, g, cm.smooth_sigma)
    d = 0.5 * min(g.dx, g.dy, g.dz)
    x, y, z = g.centres()
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    r = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    wt = cm.water.astype(float)
    tw = cm.w_dt * np.arange(wt.shape[1])
    rho_dom = cm.f_rho0 + cm.f_drho * np.arange(cm.dens.shape[1])
    fac = [np.interp(rho.ravel() if q == 0 else rhos.ravel(), rho_dom, cm.dens[q].astype(float))
           for q in range(4)]
    fu2 = lambda dens: np.interp(dens, rho_dom, cm.dens[1].astype(float))
    # per beam: (f_u2 along x, f_u2 along y, f_omega1, f_omega2) of every voxel
    lat = []
    for beam in plan.beams:
        if lateral_mode == 1:
            rw, rx, ry = axis_densities(plan, beam, d)
            lat.append((fu2(rx), fu2(ry), np.interp(rw, rho_dom, cm.dens[2].astype(float)),
                        np.interp(rw, rho_dom, cm.dens[3].astype(float))))
        else:
            lat.append((fac[1], fac[1], fac[2], fac[3]))
    A = cm.A.astype(float)
    Aint = RegularGridInterpolator((cm.a_dtheta * np.arange(A.shape[0]), cm.a_dt * np.arange(A.shape[1])), A)
    out = np.zeros(g.n_voxels)
    for i, bl in enumerate(beamlets(plan)):
        tab = tables(plan, g, plan.rho, bl["src"], bl["n"], d)
        if tab is None or f[i] == 0:
            continue
        v = r - bl["src"]
        L = v @ bl["n"]
        perp = v - L[:, None] * bl["n"]
        q2 = (perp ** 2).sum(1)
        t = L - tab["L_in"]
        m = (q2 <= cm.roi_radius ** 2) & (t >= 0) & (t <= tab["L_out"] - tab["L_in"])
        if not m.any():
            continue
        t, L, perp = t[m], L[m], perp[m]
        xs = (perp @ bl["ex"]) * bl["sad"] / L
        ys = (perp @ bl["ey"]) * bl["sad"] / L
        tk = d * np.arange(tab["K"])
        teq = np.interp(t, tk, tab["T"])
        c1, c2 = np.interp(t, tk, tab["W1"]), np.interp(t, tk, tab["W2"])
        u1w, u2w, w1w, w2w = (np.interp(t, tw, wt[q]) for q in range(4))
        th = np.clip(np.full_like(teq, bl["theta"]), 0, cm.a_dtheta * (A.shape[0] - 1))
        Av = Aint(np.stack([th, np.clip(teq, 0, cm.a_dt * (A.shape[1] - 1))], 1))
        if dc:
            fx, fy, fw1, fw2 = lat[bl["beam"]]
            u1 = fac[0][m] * u1w
            u2x, u2y = fx[m] * u2w, fy[m] * u2w
            w1 = np.maximum(fw1[m] * (w1w + c1), 0.0)
            w2 = np.maximum(fw2[m] * (w2w + c2), 0.0)
        else:
            u1, u2x, u2y, w1, w2 = u1w, u2w, u2w, w1w, w2w
        x0, y0 = plan.beamlet_x / 2, plan.beamlet_y / 2
        F = w1 * p_paper(xs, u1, x0) * p_paper(ys, u1, y0) + w2 * p_paper(xs, u2x, x0) * p_paper(ys, u2y, y0)
        out[m] += f[i] * F * Av * (bl["sad"] / L) ** 2
    return out.reshape(g.shape)
