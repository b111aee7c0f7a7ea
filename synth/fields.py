"""Initial conditions and seeded field arrays for the 2D TM Maxwell system
(fields ordered Hx, Hy, Ez, with eps = mu = 1).

Functions take caller-supplied point coordinates; they do not know about
nodes, elements or any discretisation.
"""
import numpy as np


def gaussian_pulse(x, y, x0=0.5, y0=0.5, width=0.05):
    """Ez = exp(-|x - x0|^2 / width^2), Hx = Hy = 0.  Returns (Hx, Hy, Ez)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    ez = np.exp(-((x - x0) ** 2 + (y - y0) ** 2) / width ** 2)
    return np.zeros_like(ez), np.zeros_like(ez), ez


def cavity_mode(x, y, t):
    """Exact PEC-cavity eigenmode on [-1, 1]^2 of the TM system
    mu dHx/dt = -dEz/dy, mu dHy/dt = dEz/dx, eps dEz/dt = dHy/dx - dHx/dy
    (eps = mu = 1) with Ez = 0 on the boundary:

        Ez =  sin(pi x) sin(pi y) cos(w t)
        Hx = -(pi/w) sin(pi x) cos(pi y) sin(w t)
        Hy =  (pi/w) cos(pi x) sin(pi y) sin(w t),   w = pi sqrt(2).

    Returns (Hx, Hy, Ez).
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    w = np.pi * np.sqrt(2.0)
    ez = np.sin(np.pi * x) * np.sin(np.pi * y) * np.cos(w * t)
    hx = -(np.pi / w) * np.sin(np.pi * x) * np.cos(np.pi * y) * np.sin(w * t)
    hy = (np.pi / w) * np.cos(np.pi * x) * np.sin(np.pi * y) * np.sin(w * t)
    return hx, hy, ez


def random_fields(K, Np, seed, scale=1.0):
    """Seeded U(-scale, scale) float64 values for (Hx, Hy, Ez), shape (3, K, Np)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-scale, scale, size=(3, K, Np))


def random_permittivity(K, seed, speeds=(0.5, 1.0, 2.0)):
    """Seeded piecewise-constant medium: each element's wave speed c drawn
    uniformly from `speeds`; returns eps = 1 / c^2 per element (mu = 1)."""
    rng = np.random.default_rng(seed)
    c = rng.choice(np.asarray(speeds, dtype=np.float64), size=K)
    return 1.0 / c ** 2
