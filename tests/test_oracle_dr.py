"""Pins of the oracle's per-step domain randomisation (config 4 of the
evaluation: mu in U(0.4, 1.2), k in U(5e3, 2e4) N/m, object scale in
U(0.8, 1.2), drawn per env and step from Philox with tag DR).

The draws are pinned by their distribution (range, binary32 values,
uniformity, independence, replay) and by what they do to a step: a plate at
a known depth gives F = k_dr d, a clamped tangential force is mu_dr |F_n|,
and a scaled sphere reads the distance of a sphere of radius s_dr r.
"""
import numpy as np
from scipy import stats

import oracle
from paper_2606_22332_gb300 import workload as W
from _scenes import oracle_scene, pad_workload, quiet_params

DR = {"mu": (0.4, 1.2), "k": (5e3, 2e4), "scale": (0.8, 1.2)}


def _draws(params, n_envs, step):
    return np.array([oracle.dr_draw(params, e, step) for e in range(n_envs)])


def test_draws_are_binary32_uniform_independent_and_replayable():
    p = quiet_params(dr=DR)
    v = _draws(p, 4000, 7)
    for j, key in enumerate(("mu", "k", "scale")):
        lo, hi = DR[key]
        x = v[:, j]
        assert np.all((x >= np.float32(lo)) & (x <= np.float32(hi)))
        assert np.array_equal(x, x.astype(np.float32).astype(np.float64))
        assert stats.kstest((x - lo) / (hi - lo), "uniform").pvalue > 1e-3
    c = np.corrcoef(v.T)
    assert np.all(np.abs(c[np.triu_indices(3, 1)]) < 0.06)
    assert np.array_equal(v, _draws(p, 4000, 7))
    w = _draws(p, 4000, 8)
    assert np.mean(v == w) < 1e-3
    assert stats.pearsonr(v[:, 1], w[:, 1]).statistic ** 2 < 0.01


def test_degenerate_bounds_give_the_bound():
    p = quiet_params(dr={"mu": (0.8, 0.8), "k": (1e4, 1e4), "scale": (1.0, 1.0)})
    v = _draws(p, 50, 3)
    assert np.all(v == np.array([np.float32(0.8), 1e4, 1.0]))


def test_plate_force_uses_the_drawn_stiffness_and_friction():
    depths = np.linspace(2e-4, 2e-3, 6).reshape(2, 3)
    p = quiet_params(dr=DR)
    # a fast tangential slide keeps the Coulomb clamp active: |f_t| = mu |f_n|
    wl = pad_workload(depths, 2, 3, params=p, link_vel=(100.0, 0, 0, 0, 0, 0))
    sc = oracle_scene(wl)
    st = sc.new_state(); sc.reset(st, 0)
    for step in (0, 5, 11):
        mu, k, s = oracle.dr_draw(p, 0, step)
        out = sc.step(st, wl.inputs(step))
        d = out["depth_clean"]
        f = out["ft_clean"][:3].T
        assert np.all(d > 0)
        assert np.allclose(f[:, 2], k * d, rtol=1e-12)
        ft = np.hypot(f[:, 0], f[:, 1])
        assert np.allclose(ft, mu * np.abs(f[:, 2]), rtol=1e-12)


def test_sphere_distance_uses_the_drawn_scale():
    p = quiet_params(dr=DR)
    p["dt"] = 0.005
    wl = pad_workload(0.0, 1, 1, params=p)
    wl.objects = [W.ObjectSpec(kind="sphere", radius=0.03)]
    wl.x[:] = 0; wl.y[:] = 0; wl.z[:] = 0
    wl.link_pose[0, 0, :3] = (0.0, 0.0, 0.0315)
    wl.link_pose[0, 0, 3:] = (1, 0, 0, 0)
    sc = oracle_scene(wl)
    st = sc.new_state(); sc.reset(st, 0)
    for step in range(6):
        s = oracle.dr_draw(p, 0, step)[2]
        out = sc.step(st, wl.inputs(step))
        r = float(np.float32(0.03)) * s
        expect = float(np.float32(0.0315)) - r - float(np.float32(1e-3))
        assert np.isclose(out["dist"][0], expect, atol=1e-15)
