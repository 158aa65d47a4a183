"""Training pipeline of the lateral-correction surrogate network.

Orchestration only: samples come from the library's plain axis-stencil kernel
(dc_fspb_stencils) on seeded random slab/sphere phantoms, and the network is
trained by the library's forward/backward/Adam kernels (dc_fspb.Mlp; FP32, or
BF16 tensor-core products with FP32 master parameters).
Network: 48 nearest-voxel density taps -> 64 -> 64 (SiLU) -> 3 effective
densities (omega, u_2 along x, u_2 along y), 7491 parameters.
"""
from __future__ import annotations

import numpy as np

from . import dc_fspb, synth

RHO_LO, RHO_HI = 0.05, 2.0      # density range of the training phantoms


def init_params(seed: int = 17) -> np.ndarray:
    """Uniform fan-in initialisation of the 7491 parameters (biases zero)."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, fan_out in ((48, 64), (64, 64), (64, 3)):
        lim = np.sqrt(3.0 / fan_in)
        parts.append(rng.uniform(-lim, lim, (fan_in, fan_out)).ravel())
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)


def sample_plan(rng: np.random.Generator, n=48, vox=0.25, n_beams=8):
    """A random slab/sphere phantom with beams of random gantry and couch angles."""
    g = synth.centred_grid(n, n, n, vox)
    rho = synth.random_slab_sphere_phantom(g, rng)
    beams = [synth.Beam(float(rng.uniform(0, 360)), 100.0, (0.0, 0.0, 0.0), 0.5, 0.5,
                        float(rng.uniform(-60, 60)), float(rng.uniform(0, 90))) for _ in range(n_beams)]
    cm = synth.make_commissioning(roi_radius=1.0)
    return synth.Plan("train", g, rho, beams, 0.5, 0.5, cm, np.ones(n_beams, np.float32))


def generate_samples(n_phantoms: int = 200, per_phantom: int = 10000, seed: int = 2024):
    """(X [N, 48], T [N, 3]) from the plain axis-stencil computation on random phantoms."""
    rng = np.random.default_rng(seed)
    Xs, Ts = [], []
    for _ in range(n_phantoms):
        p = sample_plan(rng)
        plan = dc_fspb.dc_fspb_create_from(p)
        vox = rng.integers(0, plan.n_voxels, per_phantom).astype(np.int32)
        beam = rng.integers(0, len(p.beams), per_phantom).astype(np.int32)
        X, T = dc_fspb.dc_fspb_stencils(plan, vox, beam)
        Xs.append(X)
        Ts.append(T)
        dc_fspb.dc_fspb_destroy(plan)
    return np.concatenate(Xs), np.concatenate(Ts)


def train(X, T, epochs: int = 8, batch: int = 4096, lr: float = 2e-3, seed: int = 17, params=None,
          precision: int = dc_fspb.DC_PRECISION_FP32):
    """Trains on a seeded shuffle of (X, T); returns (parameters, final loss).
    precision: the gradient kernel's arithmetic (FP32, or BF16 tensor-core
    products with FP32 master parameters)."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(X.shape[0])
    net = dc_fspb.Mlp(init_params(seed) if params is None else params, precision=precision)
    loss = net.train(X[perm], T[perm], batch=batch, epochs=epochs, lr=lr)
    return net.params(), loss


def save(path: str, params: np.ndarray) -> None:
    np.save(path, np.asarray(params, np.float32))


def load(path: str) -> np.ndarray:
    p = np.load(path)
    assert p.size == dc_fspb.MLP_PARAMS
    return p.astype(np.float32)
