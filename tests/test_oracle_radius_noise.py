"""Pins of the oracle's probe-radius noise (Appendix "Sensor Noise Model",
probe-level imperfections): the noisy readout sees the radius
R~ = max(0, R + eps), eps uniform on [-rho, rho] per taxel and step, while the
clean readout keeps R.  Checked against the closed forms on a flat pad over a
plane (penetration R - phi set per probe), with every other noise knob off.
"""
import numpy as np
from scipy import stats

import oracle
from paper_2606_22332_gb300 import workload as W
from _scenes import oracle_scene, pad_workload, quiet_params

K = 1e4
RHO = 3e-4


def _run(wl, steps=1, step0=0):
    sc = oracle_scene(wl)
    st = sc.new_state()
    sc.reset(st, 0)
    return [sc.step(st, wl.inputs(step0 + s)) for s in range(steps)], st


def _params(**over):
    p = quiet_params(**over)
    p["c"] = 0.0  # no damping: the force is k times the depth
    return p


def test_offsets_are_uniform_and_enter_depth_and_force():
    wl = pad_workload(1e-3, 50, 40, params=_params(rho=RHO))
    (out,), _ = _run(wl)
    base, _ = _run(pad_workload(1e-3, 50, 40, params=_params()))
    # the clean readout keeps R
    for k in ("depth_clean", "contact_clean", "ft_clean"):
        assert np.array_equal(out[k], base[0][k]), k
    eps = out["depth_noisy"] - out["depth_clean"]   # depth 1 mm > rho: R~ - phi = d + eps
    assert eps.min() >= -RHO and eps.max() <= RHO
    n = eps.size
    assert abs(eps.mean()) < 4 * RHO / np.sqrt(3 * n)
    assert abs(eps.var() / (RHO * RHO / 3) - 1) < 0.1
    assert stats.kstest(eps / RHO, "uniform", args=(-1, 2)).pvalue > 1e-3
    # the noisy force/torque chain starts from the force at the perturbed depth
    fz = out["ft_noisy"][2]
    assert np.allclose(fz, K * out["depth_noisy"], rtol=1e-12, atol=0)


def test_probes_just_clear_of_contact_touch_with_a_quarter_probability():
    # phi = R + rho / 2: clean depth 0, noisy depth max(0, eps - rho/2)
    wl = pad_workload(-RHO / 2, 60, 50, params=_params(rho=RHO))
    (out,), _ = _run(wl)
    assert np.all(out["depth_clean"] == 0.0) and np.all(out["ft_clean"] == 0.0)
    dn = out["depth_noisy"]
    touch = dn > 0
    p = touch.mean()
    assert abs(p - 0.25) < 4 * np.sqrt(0.25 * 0.75 / dn.size)
    assert dn.max() <= RHO / 2 + 1e-15


def test_noisy_contact_bit_has_its_own_schmitt_state():
    p = _params(rho=RHO)
    eta_on, eta_off = p["eta_on"], p["eta_off"]
    # probes exactly at eta_on: clean contact needs d > eta_on (off); noisy contact iff eps > 0
    wl = pad_workload(eta_on, 40, 40, params=p)
    outs, st = _run(wl, steps=2)
    y_ref = np.zeros(outs[0]["depth_noisy"].shape, dtype=np.uint8)
    for out in outs:
        assert np.all(out["contact_clean"] == 0)
        dn = out["depth_noisy"]
        y_ref = ((dn > eta_on) | (y_ref.astype(bool) & (dn > eta_off))).astype(np.uint8)
        assert np.array_equal(out["contact_noisy"], y_ref)
    assert 0.3 < y_ref.mean() < 0.8


def test_radius_clamps_at_zero():
    # R = 1e-4 < rho; probe centre on the surface (phi = 0): noisy depth = max(0, R + eps)
    R = 1e-4
    wl = pad_workload(R, 60, 50, params=_params(rho=RHO), R=R)
    (out,), _ = _run(wl)
    dn = out["depth_noisy"]
    zero = dn == 0.0
    assert abs(zero.mean() - (RHO - R) / (2 * RHO)) < 4 * np.sqrt(1 / 3 * 2 / 3 / dn.size)
    assert dn.max() <= R + RHO + 1e-15


def test_offsets_are_a_function_of_seed_taxel_and_step():
    wl = pad_workload(1e-3, 10, 10, params=_params(rho=RHO))
    (a,), _ = _run(wl)
    (b,), _ = _run(wl)
    assert np.array_equal(a["depth_noisy"], b["depth_noisy"])
    (c,), _ = _run(wl, step0=1)
    assert not np.array_equal(a["depth_noisy"], c["depth_noisy"])
