"""FP64 NumPy oracle of the 3-D gamma index (dose difference and distance to
agreement) used to compare dose distributions.

TEST INFRASTRUCTURE ONLY (tests and the benchmark's CPU legs).

The paper evaluates its doses with a 3-D gamma index at 3 %-3 mm, the 3 % taken
of the reference's maximum dose, and reports gamma_max over the distribution,
the mean gamma inside the reference's 50 % isodose line and the percentage of
voxels there with gamma < 1 (Section 3, accuracy evaluation; Tables 2-3).  It
does not say how the evaluated distribution is searched; the reading here:

    gamma(r) = min( R / dta,  min over offsets o with |o| <= R and r + o in the grid of
                    sqrt(|o|^2 / dta^2 + (D_eval(r + o) - D_ref(r))^2 / dD^2) )

with r a reference voxel centre, o a whole-voxel offset (so r + o is a voxel
centre of the evaluated distribution, on the same grid), dD = pct/100 * max D_ref
and R the search radius (gamma is capped at R / dta: every point farther than R
has a distance term above it).
"""
import numpy as np


def offsets(spacing, radius):
    """Whole-voxel offsets (i, j, k) with |(i dx, j dy, k dz)| <= radius, as an
    int array [n, 3] and their squared lengths [n] (cm^2)."""
    dx, dy, dz = (float(s) for s in spacing)
    ni, nj, nk = (int(np.floor(radius / s + 1e-9)) for s in (dx, dy, dz))
    i, j, k = np.meshgrid(np.arange(-ni, ni + 1), np.arange(-nj, nj + 1), np.arange(-nk, nk + 1), indexing="ij")
    o = np.stack([i.ravel(), j.ravel(), k.ravel()], 1)
    d2 = (o[:, 0] * dx) ** 2 + (o[:, 1] * dy) ** 2 + (o[:, 2] * dz) ** 2
    keep = d2 <= radius * radius * (1 + 1e-12)
    return o[keep], d2[keep]


def gamma_index(ref, ev, spacing, pct=3.0, dta=0.3, radius=None):
    """gamma for every voxel of ref [nz, ny, nx] against ev (same grid)."""
    ref = np.asarray(ref, np.float64)
    ev = np.asarray(ev, np.float64)
    radius = 5.0 * dta if radius is None else float(radius)
    dD = pct / 100.0 * float(ref.max())
    cap2 = (radius / dta) ** 2
    best = np.full(ref.shape, cap2)
    nz, ny, nx = ref.shape
    offs, d2 = offsets(spacing, radius)
    for (i, j, k), dd in zip(offs, d2):
        # reference voxels whose neighbour (x + i, y + j, z + k) is inside the grid
        xs = slice(max(0, -i), min(nx, nx - i))
        ys = slice(max(0, -j), min(ny, ny - j))
        zs = slice(max(0, -k), min(nz, nz - k))
        xe = slice(xs.start + i, xs.stop + i)
        ye = slice(ys.start + j, ys.stop + j)
        ze = slice(zs.start + k, zs.stop + k)
        if xs.start >= xs.stop or ys.start >= ys.stop or zs.start >= zs.stop:
            continue
        g2 = dd / dta ** 2 + (ev[ze, ye, xe] - ref[zs, ys, xs]) ** 2 / dD ** 2
        np.minimum(best[zs, ys, xs], g2, out=best[zs, ys, xs])
    return np.sqrt(best)


def gamma_stats(gamma, ref):
    """(gamma_max, mean gamma inside the 50 % isodose of ref, % of those voxels
    with gamma < 1, their number)."""
    g = np.asarray(gamma, np.float64).ravel()
    r = np.asarray(ref, np.float64).ravel()
    m = r >= 0.5 * r.max()
    return float(g.max()), float(g[m].mean()), float(100.0 * (g[m] < 1.0).mean()), int(m.sum())


def gamma_at(ref, ev, spacing, voxels, pct=3.0, dta=0.3, radius=None):
    """gamma_index at the flat voxel indices `voxels` only (for large grids)."""
    ref = np.asarray(ref, np.float64)
    ev = np.asarray(ev, np.float64)
    radius = 5.0 * dta if radius is None else float(radius)
    dD = pct / 100.0 * float(ref.max())
    nz, ny, nx = ref.shape
    offs, d2 = offsets(spacing, radius)
    out = np.empty(len(voxels))
    for n, v in enumerate(np.asarray(voxels, np.int64)):
        z, y, x = v // (nx * ny), (v // nx) % ny, v % nx
        xx, yy, zz = x + offs[:, 0], y + offs[:, 1], z + offs[:, 2]
        inside = (xx >= 0) & (xx < nx) & (yy >= 0) & (yy < ny) & (zz >= 0) & (zz < nz)
        g2 = d2[inside] / dta ** 2 + (ev[zz[inside], yy[inside], xx[inside]] - ref.flat[v]) ** 2 / dD ** 2
        out[n] = np.sqrt(min((radius / dta) ** 2, g2.min() if g2.size else np.inf))
    return out
