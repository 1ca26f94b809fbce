"""Pins of the TemperatureGrid oracle (Appendix "TemperatureGrid Sensor Model")
against closed forms.

Diffusion: with mirror padding the grid's cosine modes cos(pi m (i + 1/2) / n)
are eigenfunctions of the padded FFT filter, so a single mode decays by exactly
1 / (1 + alpha dt k^2), k = pi m / (n d), and products of modes by
1 / (1 + alpha dt (k_x^2 + k_y^2 + k_z^2)); the zero mode (total heat) only by
1 / (1 + alpha dt eps).  Source, conduction, radiation/convection and the lag
are checked term by term; the contact area on planar polygons of known area.
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import temperature as TO

N = (8, 6, 10)
D = (1.0e-3, 1.5e-3, 0.8e-3)


def _mode(n, m):
    return np.cos(np.pi * m * (np.arange(n) + 0.5) / n)


@pytest.mark.parametrize("axis,m", [(0, 1), (0, 5), (1, 2), (2, 1), (2, 9)])
def test_single_cosine_mode_decays_in_closed_form(axis, m):
    shape = [1, 1, 1]
    shape[axis] = N[axis]
    T = 30.0 + 5.0 * np.broadcast_to(_mode(N[axis], m).reshape(shape), N)
    ad = 2e-7
    out = TO.diffuse(T, D, alpha=ad, dt=1.0)
    k = np.pi * m / (N[axis] * D[axis])
    expect = 30.0 / (1 + ad * 1e-12) + 5.0 * np.broadcast_to(_mode(N[axis], m).reshape(shape), N) / (1 + ad * k * k)
    assert np.allclose(out, expect, rtol=0, atol=1e-12)
    assert abs(1 / (1 + ad * k * k) - 1) > 1e-3  # the decay is visible


def test_product_mode_uses_the_sum_of_squared_wavenumbers():
    mx, mz = 3, 4
    T = np.einsum("i,j,k->ijk", _mode(N[0], mx), np.ones(N[1]), _mode(N[2], mz))
    ad = 1e-7
    out = TO.diffuse(T, D, alpha=ad, dt=1.0)
    k2 = (np.pi * mx / (N[0] * D[0])) ** 2 + (np.pi * mz / (N[2] * D[2])) ** 2
    assert np.allclose(out, T / (1 + ad * k2), rtol=0, atol=1e-13)


def test_heat_is_conserved_and_the_field_relaxes_to_its_mean():
    rng = np.random.default_rng(0)
    T = 20 + 10 * rng.random(N)
    out = TO.diffuse(T, D, alpha=1e-7, dt=5e-3)
    assert np.isclose(out.sum(), T.sum(), rtol=1e-13)
    far = TO.diffuse(T, D, alpha=1.0, dt=1e3)
    assert np.allclose(far, T.mean(), atol=1e-9)
    assert np.allclose(TO.diffuse(T, D, alpha=0.0, dt=1.0), T, atol=1e-12)


def test_zero_flux_walls_keep_mirror_symmetry():
    rng = np.random.default_rng(1)
    T = rng.random(N)
    T = T + T[::-1]  # symmetric under the x flip
    out = TO.diffuse(T, D, alpha=3e-7, dt=1.0)
    assert np.allclose(out, out[::-1], atol=1e-13)


MAT = dict(k=0.2, rho=1100.0, cp=1500.0, emissivity=0.9, h=10.0, tau=0.0)


def _interior_cell():
    return np.ravel_multi_index((3, 2, 4), N)


def test_source_adds_dt_q_over_dz_rho_cp():
    T0 = np.full(N, 22.0)
    q = np.zeros(N)
    q[3, 2, 4] = 500.0
    mat = dict(MAT, k=0.0, emissivity=0.0, h=0.0)  # no diffusion, no surface loss
    T, _ = TO.step(T0, T0, D, mat, dt=0.01, t_amb=22.0, source=q)
    expect = T0.copy()
    expect[3, 2, 4] += 0.01 * 500.0 / (D[2] * 1100 * 1500)
    assert np.allclose(T, expect, rtol=0, atol=1e-12)


def test_contact_conduction_closed_form_and_harmonic_mean():
    T0 = np.full(N, 22.0)
    c = _interior_cell()
    mat = dict(MAT, emissivity=0.0, h=0.0)
    A, kb, To, dt = 2e-6, 1.0, 45.0, 5e-3
    T, _ = TO.step(T0, T0, D, mat, dt=dt, t_amb=22.0, contacts=[(c, To, kb, A)])
    V = D[0] * D[1] * D[2]
    keff = 2 * 0.2 * kb / (0.2 + kb)
    dT = dt * (keff * (To - 22.0) * A / V * A / V) / (1100 * 1500)
    flat = T.reshape(-1)
    assert np.isclose(flat[c] - 22.0, dT, rtol=1e-12)
    assert np.allclose(np.delete(flat, c), 22.0, atol=1e-12)  # uniform start: diffusion leaves the rest
    # equal conductivities: k_eff = k; two contacts on one cell add (both see the same T_cell)
    T2, _ = TO.step(T0, T0, D, dict(mat, k=1.0), dt=dt, t_amb=22.0, contacts=[(c, To, 1.0, A), (c, To, 1.0, A)])
    d1 = dt * (1.0 * (To - 22.0) * (A / V) ** 2) / (1100 * 1500)
    assert np.isclose(T2.reshape(-1)[c] - 22.0, 2 * d1, rtol=1e-12)


def test_radiation_and_convection_act_on_face_cells_only():
    rng = np.random.default_rng(3)
    T0 = 30 + rng.random(N)
    mat = dict(MAT, k=0.0)
    dt, ta = 0.02, 22.0
    T, _ = TO.step(T0, T0, D, mat, dt=dt, t_amb=ta)
    s = TO.surface_mask(N)
    assert s.sum() == np.prod(N) - np.prod([n - 2 for n in N])
    assert np.allclose(T[~s], T0[~s], rtol=0, atol=1e-12)  # interior: only the FFT round trip
    q = 0.9 * 5.670e-8 * ((T0 + 273.15) ** 4 - (ta + 273.15) ** 4) + 10.0 * (T0 - ta)
    assert np.allclose(T[s], (T0 - dt * q / (1100 * 1500))[s], rtol=0, atol=1e-12)


def test_measured_readout_lags_with_time_constant():
    T0 = np.full(N, 22.0)
    mat = dict(MAT, k=0.0, emissivity=0.0, h=0.0, tau=0.1)
    q = np.full(N, 1e4)
    Tm = T0.copy()
    T = T0.copy()
    dt = 0.01
    for _ in range(5):
        T, Tm_new = TO.step(T, Tm, D, mat, dt=dt, t_amb=22.0, source=q)
        assert np.allclose(Tm_new, Tm + dt / 0.1 * (T - Tm), atol=1e-12)
        Tm = Tm_new
    assert np.all(Tm < T)
    T1, Tm0 = TO.step(T, Tm, D, dict(mat, tau=0.0), dt=dt, t_amb=22.0)
    assert np.array_equal(Tm0, T1)


def test_conduction_sees_the_field_after_the_source():
    T0 = np.full(N, 22.0)
    c = _interior_cell()
    q = np.zeros(N)
    q.reshape(-1)[c] = 2e3
    mat = dict(MAT, k=0.2, emissivity=0.0, h=0.0)
    dt, A = 5e-3, 2e-6
    T, _ = TO.step(T0, T0, D, dict(mat, k=1e-30), dt=dt, t_amb=22.0, source=q, contacts=[(c, 45.0, 0.2, A)])
    ts = 22.0 + dt * 2e3 / (D[2] * 1100 * 1500)
    keff = 2 * 1e-30 * 0.2 / (1e-30 + 0.2)
    V = D[0] * D[1] * D[2]
    assert np.isclose(T.reshape(-1)[c], ts + dt * keff * (45.0 - ts) * (A / V) ** 2 / (1100 * 1500), rtol=1e-12)


def test_contact_area_of_planar_polygons():
    R = Rotation.from_rotvec([0.3, 0.5, -0.2]).as_matrix()
    sq = np.array([[0, 0, 0], [2, 0, 0], [2, 1, 0], [0, 1, 0]], float)[[2, 0, 3, 1]]  # shuffled
    assert np.isclose(TO.contact_area(sq @ R.T + 5.0, depth=0.0), 2.0, rtol=1e-12)
    th = np.linspace(0, 2 * np.pi, 7)[:-1]
    hexa = np.stack([np.cos(th), np.sin(th), np.zeros(6)], 1)[[3, 1, 5, 0, 2, 4]]
    assert np.isclose(TO.contact_area(hexa @ R.T, depth=0.0), 1.5 * np.sqrt(3), rtol=1e-12)
    assert np.isclose(TO.contact_area(sq[:2], depth=1e-3), np.pi * 1e-6)  # a disk of radius delta
    assert np.isclose(TO.contact_area(sq * 1e-3, depth=1e-3, d_w=1.0), np.pi * 1e-6)  # 2e-6 floored at pi (d_w delta)^2
    assert np.isclose(TO.contact_area(sq * 1e-3, depth=1e-3, d_w=0.5), 2e-6)  # above the floor
