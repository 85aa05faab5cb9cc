"""Seeded synthetic inputs for the matrix-free H*psi workloads.

This module holds input recipes only -- random state vectors, the initial
wavepacket and the list of batched problems -- and none of the operator's
arithmetic.  Both the CUDA path's tests/benchmark and the CPU oracle receive
the same arrays from here.

Recipes:
  * random state:   numpy default_rng(seed), real and imaginary parts standard
                    normal, each of the nvec columns normalised to unit 2-norm;
  * wavepacket:     psi0(x_i) = exp(-(x_i - x0)^2 / 2) on the grid
                    x_i = -L + i * 2L/(D-1), normalised on the grid (a coherent
                    state of the unit harmonic oscillator, zero mean momentum);
  * batch:          D_p = round(exp(U[ln 1024, ln 32768])) rounded to a multiple
                    of 128, nvec_p uniform in 1..16, seeds 0..n-1, drawn by
                    default_rng(12345).
"""
import numpy as np


def dvr_default_L(D: int) -> float:
    """Half-width of the DVR grid used by the workloads: L = 0.9 sqrt(2D)."""
    return 0.9 * np.sqrt(2.0 * float(D))


def random_state(D: int, nvec: int = 1, seed: int = 1) -> np.ndarray:
    """[D, nvec] complex128 with unit-norm columns ([D] when nvec == 1)."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((D, nvec)) + 1j * rng.standard_normal((D, nvec))
    x /= np.linalg.norm(x, axis=0, keepdims=True)
    return x[:, 0].copy() if nvec == 1 else x


def wavepacket(D: int, L: float = None, x0: float = 2.0) -> np.ndarray:
    if L is None:
        L = dvr_default_L(D)
    x = -L + (2.0 * L / (D - 1)) * np.arange(D, dtype=np.float64)
    psi = np.exp(-0.5 * (x - x0) ** 2).astype(np.complex128)
    return psi / np.linalg.norm(psi)


def batch_problems(n: int = 256, seed: int = 12345):
    """List of (D_p, nvec_p, seed_p) for the batched uneven-problem workload."""
    rng = np.random.default_rng(seed)
    lnD = rng.uniform(np.log(1024.0), np.log(32768.0), n)
    D = np.maximum(128, np.round(np.exp(lnD) / 128.0).astype(np.int64) * 128)
    nv = rng.integers(1, 17, n)
    return [(int(D[i]), int(nv[i]), i) for i in range(n)]
