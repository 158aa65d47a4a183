"""Checkpoint and resume: files for the surrogate trainer, the dose-deposition
matrix and the commissioning tables.

Each file is a NumPy .npz archive holding the arrays and one JSON header
(`header`, a string) with the format name and version, the shapes and what the
arrays mean, so a reader can check a file before using it.  The trainer file
holds everything training continues from (parameters, both Adam moments, the
step count): a trainer resumed from it takes the same steps, bit for bit, as
the one it was saved from.
"""
from __future__ import annotations

import json

import numpy as np

from . import dc_fspb, synth

MLP_FORMAT = "dc_fspb.mlp_trainer/1"
CSR_FORMAT = "dc_fspb.csr/1"
COMM_FORMAT = "dc_fspb.commissioning/1"


def _header(z):
    return json.loads(str(z["header"]))


def _check(h, fmt, path):
    if h.get("format") != fmt:
        raise ValueError(f"{path}: format {h.get('format')!r}, expected {fmt!r}")


def save_trainer(path: str, trainer: "dc_fspb.Mlp", extra: dict | None = None) -> None:
    """The trainer's parameters, Adam moments and step count."""
    theta, m1, m2, step = trainer.state()
    h = {"format": MLP_FORMAT, "params": dc_fspb.MLP_PARAMS, "layers": [48, 64, 64, 3], "activation": "SiLU",
         "optimizer": "Adam(0.9, 0.999, 1e-8)", "step": int(step), "extra": extra or {}}
    np.savez(path, header=json.dumps(h), theta=theta, m1=m1, m2=m2)


def load_trainer(path: str, stream=None) -> "dc_fspb.Mlp":
    """A new trainer in the saved state."""
    with np.load(path) as z:
        h = _header(z)
        _check(h, MLP_FORMAT, path)
        if h["params"] != dc_fspb.MLP_PARAMS:
            raise ValueError(f"{path}: {h['params']} parameters, the network has {dc_fspb.MLP_PARAMS}")
        t = dc_fspb.Mlp(z["theta"], stream=stream)
        t.set_state(z["theta"], z["m1"], z["m2"], h["step"])
    return t


def save_csr(path: str, rowptr, cols, vals, n_cols: int, meta: dict | None = None) -> None:
    """A dose-deposition matrix (rows = voxels, columns = beamlets): int64
    row pointers, int32 columns, float32 or BF16 (uint16 bits) values."""
    rowptr = np.asarray(rowptr, np.int64)
    nnz = int(rowptr[-1])
    cols = np.asarray(cols, np.int32)[:nnz]
    vals = np.asarray(vals)[:nnz]
    if vals.dtype not in (np.float32, np.uint16):
        raise ValueError("values must be float32 or BF16 bits (uint16)")
    h = {"format": CSR_FORMAT, "rows": int(rowptr.size - 1), "cols": int(n_cols), "nnz": nnz,
         "values": "f32" if vals.dtype == np.float32 else "bf16", "meta": meta or {}}
    np.savez(path, header=json.dumps(h), rowptr=rowptr, cols=cols, vals=vals)


def load_csr(path: str):
    """(rowptr, cols, vals, header) of a saved matrix."""
    with np.load(path) as z:
        h = _header(z)
        _check(h, CSR_FORMAT, path)
        rowptr, cols, vals = z["rowptr"], z["cols"], z["vals"]
    if rowptr.size != h["rows"] + 1 or cols.size != h["nnz"] or vals.size != h["nnz"] or rowptr[-1] != h["nnz"]:
        raise ValueError(f"{path}: arrays do not match the header")
    return rowptr, cols, vals, h


def save_commissioning(path: str, cm: synth.Commissioning) -> None:
    """The commissioning tables and scalars, so that several programs read
    identical inputs."""
    scal = {k: getattr(cm, k) for k in ("a_dt", "a_dtheta", "w_dt", "f_rho0", "f_drho", "roi_radius",
                                        "smooth_sigma", "rho_surface", "density_correction")}
    h = {"format": COMM_FORMAT, "A": list(cm.A.shape), "water": list(cm.water.shape), "dens": list(cm.dens.shape),
         **{k: float(v) if k != "density_correction" else int(v) for k, v in scal.items()}}
    np.savez(path, header=json.dumps(h), A=cm.A.astype(np.float32), water=cm.water.astype(np.float32),
             dens=cm.dens.astype(np.float32))


def load_commissioning(path: str) -> synth.Commissioning:
    with np.load(path) as z:
        h = _header(z)
        _check(h, COMM_FORMAT, path)
        A, water, dens = z["A"], z["water"], z["dens"]
    return synth.Commissioning(A, h["a_dt"], h["a_dtheta"], water, h["w_dt"], dens, h["f_rho0"], h["f_drho"],
                               h["roi_radius"], h["smooth_sigma"], h["rho_surface"], h["density_correction"])
