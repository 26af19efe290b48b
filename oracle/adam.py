"""Adam in float64 (oracle; test infrastructure only).

The paper (Sec. 4.1) trains with the standard 3D Gaussian splatting optimiser settings: Adam
with one learning rate per parameter group (position learning rate 1e-5).  This is Adam with
bias correction written out step by step in numpy.
"""
from __future__ import annotations

import numpy as np


def adam_step(p: np.ndarray, g: np.ndarray, m: np.ndarray, v: np.ndarray, lr, step: int,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-15):
    """One Adam step on float64 copies; lr is a scalar or an array broadcast against p.

    m <- b1 m + (1 - b1) g;  v <- b2 v + (1 - b2) g^2;
    p <- p - lr * (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
    Returns (p, m, v) as new float64 arrays.
    """
    p = np.asarray(p, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** step)
    v_hat = v / (1.0 - beta2 ** step)
    p = p - np.asarray(lr, dtype=np.float64) * m_hat / (np.sqrt(v_hat) + eps)
    return p, m, v
