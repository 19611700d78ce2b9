"""Seeded walker positions and imaginary times for replay-mode evaluation.

Replay mode feeds the same host-drawn samples to the library and to the
oracle.  Any positions and any positive times are valid inputs for that
comparison; these draws only mimic the spread of a Metropolis walk around
the atomic centres (electron pairs scattered about the nuclei) and an
exponential imaginary-time distribution.
"""
from __future__ import annotations

import numpy as np


def walker_positions(centres: np.ndarray, n_steps: int, m: int, seed: int,
                     sigma: float = 1.2) -> np.ndarray:
    """Positions [n_steps, m, 2, 3] float64: each electron near a random centre."""
    rng = np.random.default_rng(seed)
    centres = np.asarray(centres, dtype=np.float64)
    idx = rng.integers(0, len(centres), size=(n_steps, m, 2))
    scale = sigma * rng.uniform(0.3, 1.5, size=(n_steps, m, 2, 1))
    r = centres[idx] + scale * rng.standard_normal((n_steps, m, 2, 3))
    return np.ascontiguousarray(r)


def imaginary_times(rate: float, n_steps: int, n_tau: int, seed: int) -> np.ndarray:
    """Times [n_steps, n_tau] float64 drawn from an exponential law of the given rate."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.exponential(1.0 / rate, size=(n_steps, n_tau)))
