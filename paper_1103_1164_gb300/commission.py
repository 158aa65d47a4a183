"""Commissioning fit of the beam model (Section 2.1).

Section 2.1 obtains the model's parameters (u, omega, f(.), b(.)) by fitting
the DC-FSPB dose to reference doses of a slab phantom: a 30 x 30 x 30 cm^3
water cube with a 15 cm slab inserted 8 cm below the surface, slab densities
0.1-2.0 g/cm^3, a 10 x 10 cm^2 field at SAD 100 cm and SSD 90 cm.

This module is orchestration: the dose and its gradient with respect to the
tables come from the library's kernels (dc_fspb_dose, dc_fspb_dose_vjp);
here the tables are written from a parameter vector (the synthetic model
family of synth.model_tables), the gradient is carried from the tables to the
parameters (the tables' closed-form Jacobian), and Adam, or Levenberg-Marquardt
with a Gauss-Newton matrix from forward differences of the doses, takes the
steps.
Positive parameters are optimised in log space; k1 and k2 (which may be 0) in
linear space.  b_1 and b_2 are linear in the density with coefficients beta1
and beta2, so d loss / d log(beta_i) is exactly the gradient with respect to a
common scale of b_i, which dc_fspb_dose_vjp returns.
"""
from __future__ import annotations

import dataclasses
from typing import List, Sequence

import numpy as np

from . import dc_fspb, synth

PARAMS = synth.MODEL_PARAMS
LINEAR = ("k1", "k2")                       # optimised as they are; the others in log space
LIN_SCALE = 0.01                            # step scale of the linear ones


def slab_phantom(slab_rho: float, vox: float = 0.5, side: float = 30.0, depth0: float = 8.0,
                 thick: float = 15.0, ssd: float = 90.0, field: float = 10.0, beamlet: float = 0.5,
                 comm=None, roi: float = 5.0) -> synth.Plan:
    """The commissioning phantom: a water cube of `side` cm with a slab of
    density slab_rho from depth0 to depth0 + thick below the beam's entry face;
    one beam at gantry 0 (travelling +y), SSD `ssd`, a square field of `field`
    cm in beamlets of `beamlet` cm, unit fluence."""
    n = int(round(side / vox))
    g = synth.centred_grid(n, n, n, vox)
    y_face = g.oy - 0.5 * vox
    rho = synth.slab_phantom(g, (depth0, depth0 + thick), slab_rho)
    iso_y = y_face + (100.0 - ssd)
    cm = comm if comm is not None else synth.make_commissioning(roi_radius=roi)
    beam = synth.Beam(0.0, 100.0, (0.0, iso_y, 0.0), field, field)
    p = synth.Plan(f"commission{slab_rho:g}", g, rho, [beam], beamlet, beamlet, cm, np.zeros(0, np.float32))
    p.fluence = np.ones(p.n_beamlets, np.float32)
    return p


def tables_and_jacobian(theta: dict, cm):
    """Water [4, w_n] and density functions [6, f_n] for the parameters, and
    their derivatives with respect to each parameter: jw[name] [4, w_n],
    jd[name] [4, f_n] (the four density functions the dose reads directly)."""
    w_n, f_n = cm.water.shape[1], cm.dens.shape[1]
    water, dens = synth.model_tables(theta, cm.w_dt, w_n, cm.f_rho0, cm.f_drho, f_n)
    t = cm.w_dt * np.arange(w_n)
    r = cm.f_rho0 + cm.f_drho * np.arange(f_n)
    lr = np.log(r)
    z = lambda: np.zeros((4, w_n))
    jw = {k: z() for k in PARAMS}
    jd = {k: np.zeros((4, f_n)) for k in PARAMS}
    jw["u10"][0] = 1.0 / (1.0 + theta["k1"] * t)
    jw["k1"][0] = -theta["u10"] * t / (1.0 + theta["k1"] * t) ** 2
    jw["u20"][1] = 1.0 / (1.0 + theta["k2"] * t)
    jw["k2"][1] = -theta["u20"] * t / (1.0 + theta["k2"] * t) ** 2
    e = np.exp(-t / theta["tau"])
    for name, dw2 in (("w20", np.ones_like(t)), ("w21", 1.0 - e),
                      ("tau", -theta["w21"] * e * t / theta["tau"] ** 2)):
        jw[name][2] = -dw2                 # omega_1^w = 1 - omega_2^w
        jw[name][3] = dw2
    jd["a1"][0] = dens[0] * lr
    jd["a2"][1] = dens[1] * lr
    jd["gam"][3] = dens[3] * lr
    return water, dens, jw, jd


@dataclasses.dataclass
class FitResult:
    theta: dict
    loss: List[float]
    iterations: int


class CommissioningFit:
    """Least-squares fit of the model parameters to reference doses.

    plans_in: synth.Plan inputs (all with the same commissioning sampling);
    ref: reference doses, one [V] array per plan.  The loss is the mean over
    all voxels of (D - D_ref)^2 / max(D_ref)^2."""

    def __init__(self, plans_in: Sequence[synth.Plan], ref: Sequence[np.ndarray], stream=None):
        self.inputs = list(plans_in)
        self.cm = self.inputs[0].comm
        self.plans = [dc_fspb.dc_fspb_create_from(p, stream=stream) for p in self.inputs]
        self.ref = [np.asarray(r, np.float64).reshape(-1) for r in ref]
        self.scale = max(float(r.max()) for r in self.ref)
        self.nvox = sum(r.size for r in self.ref)
        self.w_n, self.f_n = self.cm.water.shape[1], self.cm.dens.shape[1]

    def set_theta(self, theta: dict):
        water, dens, _, _ = tables_and_jacobian(theta, self.cm)
        for pl in self.plans:
            dc_fspb.dc_fspb_set_tables(pl, water.astype(np.float32), dens.astype(np.float32))

    def doses(self, theta: dict) -> List[np.ndarray]:
        self.set_theta(theta)
        return [dc_fspb.dc_fspb_dose(pl, p.fluence).astype(np.float64).reshape(-1)
                for pl, p in zip(self.plans, self.inputs)]

    def loss_grad(self, theta: dict):
        """(loss, d loss / d parameter as a dict) at theta."""
        water, dens, jw, jd = tables_and_jacobian(theta, self.cm)
        gw = np.zeros((4, self.w_n))
        gd = np.zeros((4, self.f_n))
        gc = np.zeros(2)
        loss = 0.0
        norm = 1.0 / (self.nvox * self.scale ** 2)
        for pl, p, ref in zip(self.plans, self.inputs, self.ref):
            dc_fspb.dc_fspb_set_tables(pl, water.astype(np.float32), dens.astype(np.float32))
            d = dc_fspb.dc_fspb_dose(pl, p.fluence).astype(np.float64).reshape(-1)
            res = d - ref
            loss += norm * float(res @ res)
            w = (2.0 * norm * res).astype(np.float32)
            g1, g2, g3 = dc_fspb.dc_fspb_dose_vjp(pl, p.fluence, w, self.w_n, self.f_n)
            gw += g1
            gd += g2
            gc += g3
        grad = {k: float((gw * jw[k]).sum() + (gd * jd[k]).sum()) for k in PARAMS}
        # b_i = beta_i g_i(rho): d loss / d beta_i = (scale gradient) / beta_i
        grad["beta1"] = float(gc[0]) / theta["beta1"]
        grad["beta2"] = float(gc[1]) / theta["beta2"]
        return loss, grad

    @staticmethod
    def to_z(th: dict) -> np.ndarray:
        """Optimisation coordinates: log of the positive parameters, k / LIN_SCALE for the linear ones."""
        return np.array([th[k] / LIN_SCALE if k in LINEAR else np.log(th[k]) for k in PARAMS])

    @staticmethod
    def from_z(z: np.ndarray) -> dict:
        th = {k: (float(z[i]) * LIN_SCALE if k in LINEAR else float(np.exp(z[i]))) for i, k in enumerate(PARAMS)}
        for k in LINEAR:
            th[k] = max(th[k], 0.0)
        return th

    def residuals(self, theta: dict) -> np.ndarray:
        """r with loss = r . r: every plan's (D - D_ref) / (max D_ref sqrt(voxels)), concatenated."""
        c = 1.0 / (self.scale * np.sqrt(self.nvox))
        return np.concatenate([(d - ref) * c for d, ref in zip(self.doses(theta), self.ref)])

    def fit_lm(self, theta0: dict, iterations: int = 30, h: float = 1e-3, lam: float = 1e-3,
               tol: float = 0.0) -> FitResult:
        """Levenberg-Marquardt in the optimisation coordinates of fit(): the
        gradient 2 J^T r from the backward-pass kernel (loss_grad), the
        Gauss-Newton matrix J^T J from forward differences of the doses along
        each coordinate (one set of doses per parameter and iteration), and
        a damping lam diag(J^T J) that shrinks after an accepted step and
        grows after a rejected one."""
        names = list(PARAMS)
        z = self.to_z(theta0)
        hist = []
        it = 0
        for it in range(1, iterations + 1):
            th = self.from_z(z)
            loss, g = self.loss_grad(th)
            hist.append(loss)
            if loss <= tol:
                break
            gz = np.array([g[k] * LIN_SCALE if k in LINEAR else g[k] * th[k] for k in names])
            r0 = self.residuals(th)
            J = np.empty((r0.size, len(names)))
            for i in range(len(names)):
                zi = z.copy()
                zi[i] += h
                J[:, i] = (self.residuals(self.from_z(zi)) - r0) / h
            A = J.T @ J
            d = np.diag(A).copy()
            d[d <= 0] = 1.0
            for _ in range(12):
                step = np.linalg.solve(A + lam * np.diag(d), -0.5 * gz)
                trial = self.from_z(z + step)
                r1 = self.residuals(trial)
                if float(r1 @ r1) < loss:
                    z = z + step
                    lam = max(lam / 3.0, 1e-9)
                    break
                lam *= 4.0
            else:
                break                       # no descent along any damped step
        return FitResult(self.from_z(z), hist, it)

    def fit(self, theta0: dict, iterations: int = 300, lr: float = 0.02, tol: float = 0.0) -> FitResult:
        """Adam in the optimisation coordinates (log of the positive
        parameters, k / LIN_SCALE for the linear ones)."""
        names = list(PARAMS)
        from_z = self.from_z
        z = self.to_z(theta0)
        m = np.zeros_like(z)
        v = np.zeros_like(z)
        b1, b2, eps = 0.9, 0.999, 1e-12
        hist = []
        it = 0
        for it in range(1, iterations + 1):
            th = from_z(z)
            loss, g = self.loss_grad(th)
            hist.append(loss)
            if loss <= tol:
                break
            gz = np.array([g[k] * LIN_SCALE if k in LINEAR else g[k] * th[k] for k in names])
            m = b1 * m + (1 - b1) * gz
            v = b2 * v + (1 - b2) * gz * gz
            mh = m / (1 - b1 ** it)
            vh = v / (1 - b2 ** it)
            z = z - lr * mh / (np.sqrt(vh) + eps)
        return FitResult(from_z(z), hist, it)

    def destroy(self):
        for pl in self.plans:
            dc_fspb.dc_fspb_destroy(pl)
        self.plans = []
