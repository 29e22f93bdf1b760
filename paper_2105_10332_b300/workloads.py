"""Seeded synthetic inputs for the swept-rule solver.

This module only builds initial fields and time steps; it holds none of the
solver's arithmetic, so the CUDA path and the CPU oracle can both take their
inputs from it.  Every generator is deterministic for a given seed.

Problems (Appendix A and B of the paper; sizes as the workloads use them):
  heat_sine    -- T0 = sin(2 pi x) sin(2 pi y) on the periodic unit square (App. A)
  heat_modes   -- a sum of seeded Fourier modes (the large heat workload)
  vortex       -- isentropic vortex on [-5, 5]^2 superimposed on a uniform
                  stream (the Shu form with beta = 5, u = v = 1, rho = p = 1;
                  App. B describes the vortex and Table A1 an alternative set
                  of constants, see ``vortex_table_a1``)
  vortex_dt    -- a fixed time step from the CFL number and the initial field
"""
import math

import numpy as np

MASK64 = (1 << 64) - 1


def splitmix64(seed):
    """SplitMix64 (Steele, Lea & Flood 2014; constants as published by Vigna)."""
    x = seed & MASK64
    while True:
        x = (x + 0x9E3779B97F4A7C15) & MASK64
        z = x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        yield z ^ (z >> 31)


def uniform01(gen):
    """A double in [0, 1) from the top 53 bits of one SplitMix64 draw."""
    return (next(gen) >> 11) * (1.0 / (1 << 53))


def heat_grid(nx, ny):
    """Node coordinates x_i = i/nx, y_j = j/ny of the periodic unit square (App. A)."""
    x = np.arange(nx, dtype=np.float64) / nx
    y = np.arange(ny, dtype=np.float64) / ny
    return x, y


def heat_sine(nx, ny):
    """App. A initial field sin(2 pi x) sin(2 pi y), shape [ny, nx]."""
    x, y = heat_grid(nx, ny)
    return np.outer(np.sin(2 * math.pi * y), np.sin(2 * math.pi * x))


def heat_modes_spec(seed=20210521, nmodes=8, kmax=16):
    """Mode list [(a, kx, ky, phx, phy)]: a ~ U(-1,1), k ~ U{1..kmax}, phase ~ U(0, 2 pi)."""
    g = splitmix64(seed)
    modes = []
    for _ in range(nmodes):
        a = 2.0 * uniform01(g) - 1.0
        kx = 1 + int(uniform01(g) * kmax)
        ky = 1 + int(uniform01(g) * kmax)
        phx = 2.0 * math.pi * uniform01(g)
        phy = 2.0 * math.pi * uniform01(g)
        modes.append((a, kx, ky, phx, phy))
    return modes


def heat_modes(nx, ny, seed=20210521, nmodes=8, kmax=16):
    """Sum of seeded modes a sin(2 pi kx x + phx) sin(2 pi ky y + phy), shape [ny, nx]."""
    x, y = heat_grid(nx, ny)
    u = np.zeros((ny, nx))
    for a, kx, ky, phx, phy in heat_modes_spec(seed, nmodes, kmax):
        u += a * np.outer(np.sin(2 * math.pi * ky * y + phy), np.sin(2 * math.pi * kx * x + phx))
    return u


def heat_dt(nx, r=0.1, alpha=1.0):
    """Time step with r = alpha dt / dx^2 on the unit square (dx = 1/nx)."""
    dx = 1.0 / nx
    return r * dx * dx / alpha, dx


def vortex(nx, ny=None, beta=5.0, gamma=1.4, u_inf=1.0, v_inf=1.0, rho_inf=1.0, p_inf=1.0,
           half_width=5.0, xc=0.0, yc=0.0):
    """Isentropic vortex at cell centres of [-L, L]^2; returns (q [4, ny, nx], dx).

    Perturbations (Shu form): du = -beta/(2 pi) e^{(1-r^2)/2} (y-yc),
    dv = +beta/(2 pi) e^{(1-r^2)/2} (x-xc), dT = -(gamma-1) beta^2/(8 gamma pi^2) e^{1-r^2};
    rho = (1 + dT)^{1/(gamma-1)}, p = rho^gamma (rho_inf = p_inf = 1).
    The domain is periodic, so (xc, yc) is wrapped to the nearest image.
    """
    ny = nx if ny is None else ny
    L = half_width
    dx = 2 * L / nx
    xs = -L + (np.arange(nx) + 0.5) * dx
    ys = -L + (np.arange(ny) + 0.5) * (2 * L / ny)
    X, Y = np.meshgrid(xs, ys)
    rx = (X - xc + L) % (2 * L) - L
    ry = (Y - yc + L) % (2 * L) - L
    r2 = rx * rx + ry * ry
    f = np.exp(0.5 * (1.0 - r2))
    du = -beta / (2 * math.pi) * f * ry
    dv = beta / (2 * math.pi) * f * rx
    dT = -(gamma - 1.0) * beta * beta / (8.0 * gamma * math.pi * math.pi) * f * f
    T = (p_inf / rho_inf) + dT
    rho = rho_inf * (T / (p_inf / rho_inf)) ** (1.0 / (gamma - 1.0))
    p = rho * T
    u = u_inf + du
    v = v_inf + dv
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    q = np.stack([rho, rho * u, rho * v, E])
    return np.ascontiguousarray(q), dx


def vortex_table_a1(nx, ny=None, gamma=1.4, half_width=5.0, xc=0.0, yc=0.0):
    """Vortex with the constants of App. B, Table A1 (alpha = 45 deg, M = sqrt(2/gamma),
    beta = M 5 sqrt(2)/(4 pi) e^{1/2}, R = sigma = 1, p_inf = 1/gamma normalisation).

    Reading of the garbled App. B lines: Omega = beta e^{f}, f = -(x^2 + y^2)/(2 sigma^2 R^2),
    du = -(y/R) Omega, dv = +(x/R) Omega (the printed minus on dv would not
    give a vortex), dT = -(gamma-1)/2 Omega^2; rho = (1+dT)^{1/(gamma-1)},
    p = (1+dT)^{gamma/(gamma-1)}/gamma.
    """
    ny = nx if ny is None else ny
    L = half_width
    dx = 2 * L / nx
    xs = -L + (np.arange(nx) + 0.5) * dx
    ys = -L + (np.arange(ny) + 0.5) * (2 * L / ny)
    X, Y = np.meshgrid(xs, ys)
    X = (X - xc + L) % (2 * L) - L
    Y = (Y - yc + L) % (2 * L) - L
    M = math.sqrt(2.0 / gamma)
    beta = M * 5.0 * math.sqrt(2.0) / (4.0 * math.pi) * math.exp(0.5)
    om = beta * np.exp(-0.5 * (X * X + Y * Y))
    du = -Y * om
    dv = X * om
    dT = -0.5 * (gamma - 1.0) * om * om
    rho = (1.0 + dT) ** (1.0 / (gamma - 1.0))
    p = (1.0 + dT) ** (gamma / (gamma - 1.0)) / gamma
    a = math.radians(45.0)
    u = M * math.cos(a) + du
    v = M * math.sin(a) + dv
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return np.ascontiguousarray(np.stack([rho, rho * u, rho * v, E])), dx


def vortex_dt(q, dx, t_end, cfl=0.25, gamma=1.4):
    """Fixed step for a run to t_end: dt0 = cfl dx / max(|u|+c, |v|+c) over the
    initial cells, N = ceil(t_end / dt0), dt = t_end / N.  Returns (dt, N)."""
    rho, mx, my, E = q
    u = mx / rho
    v = my / rho
    p = (gamma - 1.0) * (E - 0.5 * rho * (u * u + v * v))
    c = np.sqrt(gamma * p / rho)
    smax = float(np.max(np.maximum(np.abs(u) + c, np.abs(v) + c)))
    dt0 = cfl * dx / smax
    N = int(math.ceil(t_end / dt0))
    return t_end / N, N


def batch_sides(count=256, lo=64, hi=2048, multiple=32, seed=20210521):
    """Square grid sides drawn log-uniform in [lo, hi] and rounded to a multiple."""
    g = splitmix64(seed ^ 0xBA7C4)
    sides = []
    for _ in range(count):
        s = math.exp(math.log(lo) + uniform01(g) * (math.log(hi) - math.log(lo)))
        s = int(round(s / multiple)) * multiple
        sides.append(min(max(s, lo), hi))
    return sides
