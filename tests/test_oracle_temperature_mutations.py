"""Mutation checks of the TemperatureGrid pins: each test plants one plausible
mistake in the oracle (on the CPU, through monkeypatching) and requires at
least one pin to fail on it."""
import numpy as np
import pytest

import test_oracle_temperature as P
from oracle import temperature as TO


def _fails(pins):
    for pin in pins:
        try:
            pin()
        except AssertionError:
            return True
    return False


def _diffuse_with(pad_mode="symmetric", k_factor=1.0):
    def diffuse(T, d, alpha, dt, eps=1e-12):
        T = np.asarray(T, np.float64)
        n = T.shape
        Tp = np.pad(T, [(0, m) for m in n], mode=pad_mode)
        if Tp.shape != tuple(2 * m for m in n):  # whole-sample reflection drops a sample: pad it back
            Tp = np.pad(Tp, [(0, 2 * m - s) for m, s in zip(n, Tp.shape)], mode="edge")
        F = np.fft.rfftn(Tp)
        kx = k_factor * 2 * np.pi * np.fft.fftfreq(2 * n[0], d[0])
        ky = k_factor * 2 * np.pi * np.fft.fftfreq(2 * n[1], d[1])
        kz = k_factor * 2 * np.pi * np.fft.rfftfreq(2 * n[2], d[2])
        k2 = kx[:, None, None] ** 2 + ky[None, :, None] ** 2 + kz[None, None, :] ** 2
        F = F / (1.0 + alpha * dt * np.maximum(k2, eps))
        return np.fft.irfftn(F, s=Tp.shape, axes=(0, 1, 2))[: n[0], : n[1], : n[2]]
    return diffuse


DIFFUSION_PINS = [lambda: P.test_single_cosine_mode_decays_in_closed_form(0, 1),
                  lambda: P.test_single_cosine_mode_decays_in_closed_form(2, 9),
                  P.test_product_mode_uses_the_sum_of_squared_wavenumbers,
                  P.test_heat_is_conserved_and_the_field_relaxes_to_its_mean,
                  P.test_zero_flux_walls_keep_mirror_symmetry]


@pytest.mark.parametrize("mutant", [dict(pad_mode="reflect"), dict(k_factor=2.0)])
def test_diffusion_mistakes_are_caught(monkeypatch, mutant):
    monkeypatch.setattr(TO, "diffuse", _diffuse_with(**mutant))
    assert _fails(DIFFUSION_PINS)


def _step_with(kelvin=TO.KELVIN, mean="harmonic", source_axis=2, lag_from_old=False):
    diffuse = _diffuse_with()

    def step(T, T_meas, d, mat, dt, t_amb, source=None, contacts=(), eps=1e-12):
        rc = mat["rho"] * mat["cp"]
        T0 = np.asarray(T, np.float64)
        T = diffuse(T0, d, mat["k"] / rc, dt, eps)
        if source is not None:
            T = T + dt * np.asarray(source, np.float64) / (d[source_axis] * rc)
        V = d[0] * d[1] * d[2]
        flat = T.reshape(-1)
        dT = np.zeros_like(flat)
        for c, t_o, k_o, A in contacts:
            k_eff = 2.0 * mat["k"] * k_o / (mat["k"] + k_o) if mean == "harmonic" else 0.5 * (mat["k"] + k_o)
            dT[c] += dt * (k_eff * (t_o - flat[c]) / (V / A)) * A / V / rc
        T = (flat + dT).reshape(T.shape)
        s = TO.surface_mask(T.shape)
        q = mat["emissivity"] * TO.SIGMA * ((T + kelvin) ** 4 - (t_amb + kelvin) ** 4) + mat["h"] * (T - t_amb)
        T = np.where(s, T - dt * q / rc, T)
        T_meas = np.asarray(T_meas, np.float64)
        src = T0 if lag_from_old else T
        T_meas = T_meas + dt / mat["tau"] * (src - T_meas) if mat["tau"] > 0 else src.copy()
        return T, T_meas
    return step


STEP_PINS = [P.test_source_adds_dt_q_over_dz_rho_cp, P.test_contact_conduction_closed_form_and_harmonic_mean,
             P.test_radiation_and_convection_act_on_face_cells_only, P.test_measured_readout_lags_with_time_constant,
             P.test_conduction_sees_the_field_after_the_source]


@pytest.mark.parametrize("mutant", [dict(kelvin=0.0), dict(mean="arithmetic"), dict(source_axis=0),
                                    dict(lag_from_old=True)])
def test_step_mistakes_are_caught(monkeypatch, mutant):
    monkeypatch.setattr(TO, "step", _step_with(**mutant))
    assert _fails(STEP_PINS)


def test_the_unmutated_copy_passes_every_pin(monkeypatch):
    monkeypatch.setattr(TO, "step", _step_with())
    monkeypatch.setattr(TO, "diffuse", _diffuse_with())
    assert not _fails(STEP_PINS + DIFFUSION_PINS)


def test_an_unsquared_area_floor_is_caught(monkeypatch):
    orig = TO.contact_area

    def area(points, depth, d_w=1.0):
        a = orig(points, depth, d_w)
        return max(a, np.pi * d_w * depth)
    monkeypatch.setattr(TO, "contact_area", area)
    assert _fails([P.test_contact_area_of_planar_polygons])
