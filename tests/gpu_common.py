"""Helpers shared by the GPU parity tests (inputs and comparisons only)."""
import numpy as np


def zero_slots(px, py):
    """Zero the structural slots of a vector field (x: last column, y: last row)."""
    px = np.array(px, dtype=np.float32)
    py = np.array(py, dtype=np.float32)
    px[:, -1] = 0.0
    py[-1, :] = 0.0
    return px, py


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def random_unit_field(N, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    px = rng.uniform(-1, 1, (N, N)) * scale
    py = rng.uniform(-1, 1, (N, N)) * scale
    n = np.maximum(1.0, np.hypot(px, py))
    return zero_slots(px / n, py / n)
