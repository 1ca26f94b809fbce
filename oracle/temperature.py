"""FP64 oracle of the TemperatureGrid sensor (Appendix "TemperatureGrid Sensor
Model").  Test infrastructure only: the tests, the entry point's smoke check
and the bench's CPU baseline use it; the product path never does.

One step of a grid of n_x x n_y x n_z cells with voxel size (dx, dy, dz), in
the paper's order (diffusion and internal source, contact conduction, then
radiation and convection), and the measured readout's first-order lag:

- diffusion: the grid is mirror-padded to twice its size on every axis, a
  real-input FFT taken, every mode divided by 1 + alpha dt k^2 (k the
  wavenumber vector of the padded grid, k^2 floored at eps), the inverse FFT
  taken and the result cropped back to the grid;
- source: T += dt q / (dz rho c_p), q in W/m^2 per cell;
- contact conduction: a contact on cell c with a body at T_other of
  conductivity k_b and contact area A adds dt Q / (rho c_p) with
  k_eff = 2 k k_b / (k + k_b), L = V / A, flux = k_eff (T_other - T_c) / L and
  Q = flux A / V, V the cell volume; all contacts of a step see the cell
  temperatures after the source and their changes add;
- radiation and convection on every cell on a face of the grid:
  T -= dt (eps_r sigma (T_K^4 - T_amb,K^4) + h (T - T_amb)) / (rho c_p),
  T_K = T + 273.15, taken as printed;
- lag: T_meas += dt / tau (T - T_meas) for tau > 0, else T_meas = T.

The contact area of a manifold: its points projected on their mean plane
(the plane through the centroid normal to the least-variance direction),
ordered by polar angle about the centroid, shoelace polygon area; fewer than
three points give a disk of radius delta, pi delta^2; the conduction update
floors the area at pi (d_w delta)^2.  (The paper prints the disk as "pi
delta" and the floor as "pi d_w delta", lengths where an area is meant; read
as the disk of radius delta and of radius d_w delta.)
"""
from __future__ import annotations

import numpy as np

SIGMA = 5.670e-8
KELVIN = 273.15


def diffuse(T: np.ndarray, d, alpha: float, dt: float, eps: float = 1e-12) -> np.ndarray:
    """Implicit spectral diffusion with mirror padding (Neumann walls)."""
    T = np.asarray(T, np.float64)
    n = T.shape
    Tp = np.pad(T, [(0, m) for m in n], mode="symmetric")  # T_0..T_{n-1}, T_{n-1}..T_0 on every axis
    F = np.fft.rfftn(Tp)
    kx = 2 * np.pi * np.fft.fftfreq(2 * n[0], d[0])
    ky = 2 * np.pi * np.fft.fftfreq(2 * n[1], d[1])
    kz = 2 * np.pi * np.fft.rfftfreq(2 * n[2], d[2])
    k2 = kx[:, None, None] ** 2 + ky[None, :, None] ** 2 + kz[None, None, :] ** 2
    F = F / (1.0 + alpha * dt * np.maximum(k2, eps))
    return np.fft.irfftn(F, s=Tp.shape, axes=(0, 1, 2))[: n[0], : n[1], : n[2]]


def surface_mask(n) -> np.ndarray:
    m = np.zeros(n, bool)
    m[0], m[-1], m[:, 0], m[:, -1], m[:, :, 0], m[:, :, -1] = True, True, True, True, True, True
    return m


def step(T, T_meas, d, mat: dict, dt: float, t_amb: float, source=None, contacts=(), eps: float = 1e-12):
    """One step of one grid.  mat: k, rho, cp, emissivity, h, tau.  contacts:
    iterable of (flat cell index, T_other, k_other, area).  Returns (T, T_meas)."""
    rc = mat["rho"] * mat["cp"]
    alpha = mat["k"] / rc
    T = diffuse(T, d, alpha, dt, eps)
    if source is not None:
        T = T + dt * np.asarray(source, np.float64) / (d[2] * rc)
    V = d[0] * d[1] * d[2]
    flat = T.reshape(-1)
    dT = np.zeros_like(flat)
    for c, t_o, k_o, A in contacts:
        k_eff = 2.0 * mat["k"] * k_o / (mat["k"] + k_o)
        L = V / A
        flux = k_eff * (t_o - flat[c]) / L
        Q = flux * A / V
        dT[c] += dt * Q / rc
    T = (flat + dT).reshape(T.shape)
    s = surface_mask(T.shape)
    TK, TaK = T + KELVIN, t_amb + KELVIN
    q = mat["emissivity"] * SIGMA * (TK ** 4 - TaK ** 4) + mat["h"] * (T - t_amb)
    T = np.where(s, T - dt * q / rc, T)
    T_meas = np.asarray(T_meas, np.float64)
    if mat["tau"] > 0:
        T_meas = T_meas + dt / mat["tau"] * (T - T_meas)
    else:
        T_meas = T.copy()
    return T, T_meas


def contact_area(points, depth: float, d_w: float = 1.0) -> float:
    """Contact area of one manifold, floored at pi (d_w depth)^2."""
    p = np.asarray(points, np.float64).reshape(-1, 3)
    if len(p) < 3:
        area = np.pi * depth * depth
    else:
        c = p.mean(0)
        _, _, vt = np.linalg.svd(p - c)
        u, v = vt[0], vt[1]  # the mean plane's axes (normal vt[2])
        x, y = (p - c) @ u, (p - c) @ v
        order = np.argsort(np.arctan2(y, x), kind="stable")
        x, y = x[order], y[order]
        area = 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))
    return max(area, np.pi * (d_w * depth) ** 2)
