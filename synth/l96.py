"""Lorenz-96 forecast model (input generator for the small cycling workload).

dx_i/dt = (x_{i+1} - x_{i-2}) x_{i-1} - x_i + F with cyclic indices (Sec. 6.2, Eq. l96),
integrated with classical fourth-order Runge-Kutta. Works on one state (n,) or on an
ensemble laid out (n, N) (state index major, member fastest).
"""
import numpy as np


def l96_tendency(x: np.ndarray, forcing: float = 8.0) -> np.ndarray:
    return (np.roll(x, -1, axis=0) - np.roll(x, 2, axis=0)) * np.roll(x, 1, axis=0) - x + forcing


def l96_rk4(x: np.ndarray, dt: float, steps: int, forcing: float = 8.0) -> np.ndarray:
    x = np.array(x, dtype=np.float64, copy=True)
    for _ in range(steps):
        k1 = l96_tendency(x, forcing)
        k2 = l96_tendency(x + 0.5 * dt * k1, forcing)
        k3 = l96_tendency(x + 0.5 * dt * k2, forcing)
        k4 = l96_tendency(x + dt * k3, forcing)
        x = x + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    return x
