"""Pins of the oracle's sensor formulas and noise model against closed forms.

Plate pressed to a known depth (F = k d, tau = x cross F), no penetration
(zero force), the Coulomb-clamp branches, the damping sign, the Schmitt
trigger on a hand-worked chatter sequence, the hysteresis step response,
crosstalk on uniform fields, drift variance, dead-taxel statistics, link
sums and agg_force, fillers and object scale.
"""
import numpy as np
import pytest
from scipy import stats
from scipy.spatial.transform import Rotation

import oracle
from paper_2606_22332_gb300 import workload as W
from _scenes import oracle_scene, pad_workload, quiet_params

K = 1e4


def run(wl, steps=1, st=None, sc=None, episode=0, step0=0):
    sc = sc or oracle_scene(wl)
    if st is None:
        st = sc.new_state()
        sc.reset(st, episode)
    outs = [sc.step(st, wl.inputs(step0 + s)) for s in range(steps)]
    return sc, st, outs


# ---------------------------------------------------------------- Schmitt (Eq. 3)
def test_schmitt_chatter_sequence():
    d = [0.0, 6e-4, 4e-4, 3e-4, 1e-4, 3e-4, 6e-4, 1.9e-4, 5e-4, 5.01e-4, 2e-4]
    expect = [0, 1, 1, 1, 0, 0, 1, 0, 0, 1, 0]   # worked by hand from the rule
    y, got = 0, []
    for v in d:
        y = oracle.schmitt(y, v, 5e-4, 2e-4)
        got.append(y)
    assert got == expect


def test_schmitt_without_hysteresis_is_threshold():
    rng = np.random.default_rng(0)
    y = 0
    for v in rng.uniform(0, 1e-3, 200):
        y = oracle.schmitt(y, v, 5e-4, 5e-4)
        assert y == int(v > 5e-4)


# ---------------------------------------------------------------- force law (Eqs. 4-9 + clamp)
def test_plate_force_equals_k_depth_and_torque_is_x_cross_f():
    rng = np.random.default_rng(1)
    depths = rng.uniform(1e-5, 3e-3, (4, 6))
    wl = pad_workload(depths, 4, 6, params=quiet_params())
    _, _, (out,) = run(wl)
    d = out["depth_clean"]
    ref_d = W.f32(wl.R).astype(float) - (0.01 + wl.z.astype(float))  # R - height of the probe
    assert np.allclose(d, ref_d, atol=1e-15)
    f = out["ft_clean"][:3].T
    tau = out["ft_clean"][3:].T
    assert np.allclose(f[:, :2], 0.0, atol=1e-12)
    assert np.allclose(f[:, 2], K * d, rtol=1e-12)
    x = np.stack([wl.x, wl.y, wl.z], 1).astype(float)
    assert np.allclose(tau, np.cross(x, f), atol=1e-12)


def test_no_penetration_gives_zero():
    wl = pad_workload(-np.linspace(1e-6, 5e-3, 12).reshape(3, 4), 3, 4, params=quiet_params(),
                      link_vel=(0.1, -0.2, 0.3, 1, 2, 3), obj_vel=(0.5, 0, 0, 0, 0, 4))
    _, _, (out,) = run(wl)
    assert np.all(out["depth_clean"] == 0.0)
    assert np.all(out["ft_clean"] == 0.0)
    assert np.all(out["contact_clean"] == 0)
    assert np.all(out["dist"] > 0)


def test_force_frames_against_independent_geometry():
    """Sphere object, random link and object poses, velocities: the link-frame
    force from quantities computed here with scipy rotations."""
    rng = np.random.default_rng(2)
    p = quiet_params()
    for trial in range(20):
        r = 0.03
        RC = Rotation.random(random_state=rng.integers(1 << 30))
        RL = Rotation.random(random_state=rng.integers(1 << 30))
        pC = rng.normal(0, 0.01, 3)
        x = rng.normal(0, 0.01, 3)
        # put the probe 1.5 mm inside the sphere's surface
        u = rng.normal(size=3); u /= np.linalg.norm(u)
        q_target = pC + (r - 1.5e-3) * u
        pL = q_target - RL.apply(x)
        vL, wL, vC, wC = rng.normal(0, 0.1, 3), rng.normal(0, 1, 3), rng.normal(0, 0.1, 3), rng.normal(0, 1, 3)
        wl = pad_workload(0.0, 1, 1, params=p)
        wl.objects = [W.ObjectSpec(kind="sphere", radius=r)]
        wl.x[:] = x[0]; wl.y[:] = x[1]; wl.z[:] = x[2]
        wl.link_pose[0, 0, :3] = pL; wl.link_pose[0, 0, 3:] = np.roll(RL.as_quat(), 1)
        wl.obj_pose[0, :3] = pC; wl.obj_pose[0, 3:] = np.roll(RC.as_quat(), 1)
        wl.link_vel[0, 0] = np.r_[vL, wL]; wl.obj_vel[0] = np.r_[vC, wC]
        # the inputs are stored in float32: recompute everything from them
        xs = np.array([wl.x[0], wl.y[0], wl.z[0]], float)
        RLs = Rotation.from_quat(np.roll(wl.link_pose[0, 0, 3:].astype(float), -1))
        pLs = wl.link_pose[0, 0, :3].astype(float)
        pCs = wl.obj_pose[0, :3].astype(float)
        vL, wL = wl.link_vel[0, 0, :3].astype(float), wl.link_vel[0, 0, 3:].astype(float)
        vC, wC = wl.obj_vel[0, :3].astype(float), wl.obj_vel[0, 3:].astype(float)
        q = pLs + RLs.apply(xs)
        dist = np.linalg.norm(q - pCs)
        m = (q - pCs) / dist
        d = float(np.float32(1e-3)) - (dist - r)
        mbar = RLs.inv().apply(m)
        vrel = RLs.inv().apply((vC + np.cross(wC, q - pCs)) - (vL + np.cross(wL, q - pLs)))
        vn = vrel @ mbar * mbar
        vt = vrel - vn
        fn = K * d * mbar + p["c"] * d * vn
        ft = -p["k_t"] * vt * min(1.0, p["mu"] * np.linalg.norm(fn) / (p["k_t"] * np.linalg.norm(vt)))
        f = fn + ft
        tau = np.cross(xs, f) - p["k_omega"] * ((wC - wL) @ m) * mbar
        _, _, (out,) = run(wl)
        assert np.isclose(out["depth_clean"][0], d, rtol=1e-12, atol=1e-16)
        assert np.allclose(out["ft_clean"][:3, 0], f, rtol=1e-10, atol=1e-12)
        assert np.allclose(out["ft_clean"][3:, 0], tau, rtol=1e-10, atol=1e-12)


def test_coulomb_clamp_branches_and_damping_sign():
    p = quiet_params()
    x = np.array([0.01, 0.0, 0.02]); mbar = np.array([0.0, 0.0, 1.0])
    d = 1e-3
    vrel = np.array([0.3, -0.4, 0.0])          # purely tangential, |v_t| = 0.5
    f_free, _ = oracle.taxel_force(p, K, None, d, x, mbar, vrel, 0.0)
    assert np.allclose(f_free, [-p["k_t"] * 0.3, p["k_t"] * 0.4, K * d])
    f0, _ = oracle.taxel_force(p, K, 0.0, d, x, mbar, vrel, 0.0)
    assert np.allclose(f0, [0, 0, K * d])
    # clamp active: |f_t| = mu |f_n| = 1e-4 * 10 N = 1e-3 < k_t |v_t| = 1
    mu = 1e-4
    fc, _ = oracle.taxel_force(p, K, mu, d, x, mbar, vrel, 0.0)
    assert np.isclose(np.linalg.norm(fc[:2]), mu * K * d)
    assert np.allclose(fc[:2] / np.linalg.norm(fc[:2]), [-0.6, 0.8])
    # damping: approach (object moving along +m towards the probe) adds force
    fa, _ = oracle.taxel_force(p, K, None, d, x, mbar, [0, 0, 0.2], 0.0)
    fr, _ = oracle.taxel_force(p, K, None, d, x, mbar, [0, 0, -0.2], 0.0)
    assert np.isclose(fa[2], K * d + p["c"] * d * 0.2) and np.isclose(fr[2], K * d - p["c"] * d * 0.2)
    # alpha = 1.2: s = d^1.2
    p12 = dict(p, alpha=1.2)
    f12, _ = oracle.taxel_force(p12, 500.0, None, d, x, mbar, [0, 0, 0], 0.0)
    assert np.isclose(f12[2], 500.0 * d ** 1.2)
    # spin torque along the normal
    _, tau = oracle.taxel_force(p, K, None, d, x, mbar, [0, 0, 0], 0.7)
    assert np.allclose(tau, np.cross(x, [0, 0, K * d]) - p["k_omega"] * 0.7 * mbar)


# ---------------------------------------------------------------- hysteresis (Eqs. 29-30)
def test_hysteresis_step_response_closed_form():
    p = quiet_params()
    p["noise"]["depth"] = W.noise_group(beta=0.1, tau=0.05)
    d0 = 2e-3
    wl_on = pad_workload(d0, 1, 2, params=p)
    sc = oracle_scene(wl_on)
    st = sc.new_state(); sc.reset(st, 0)
    a = np.exp(-p["dt"] / 0.05)
    x = sc.step(st, wl_on.inputs(0))["depth_clean"][0]
    assert np.isclose(x, d0, rtol=1e-9)
    for t in range(1, 8):
        out = sc.step(st, wl_on.inputs(0))
        assert np.isclose(out["depth_noisy"][0], x + 0.1 * a ** t * x, rtol=1e-12)
    # falling step: depth drops to zero -> undershoot -0.1 (1 - a^8) x, decaying
    wl_off = pad_workload(-1e-3, 1, 2, params=p)
    sc_off = oracle_scene(wl_off)
    xi = a ** 7 * x
    for t in range(5):
        out = sc_off.step(st, wl_off.inputs(0))
        xi = a * xi + ((0.0 - x) if t == 0 else 0.0)
        assert out["depth_clean"][0] == 0.0
        assert np.isclose(out["depth_noisy"][0], 0.1 * xi, rtol=1e-12)
        assert out["depth_noisy"][0] < 0


# ---------------------------------------------------------------- crosstalk (Eq. 31)
def test_crosstalk_weights():
    w = oracle.crosstalk_weights(1.0)
    assert np.isclose(w.sum(), 1.0)
    assert np.allclose(w, w.T) and np.allclose(w, w[::-1, ::-1])
    c = 1.0 / (1 + 4 * np.exp(-0.5) + 4 * np.exp(-1.0))
    assert np.isclose(w[1, 1], c) and np.isclose(w[0, 1], c * np.exp(-0.5)) and np.isclose(w[0, 0], c * np.exp(-1.0))


@pytest.mark.parametrize("wrap", [0, 1])
def test_crosstalk_preserves_uniform_field(wrap):
    p = quiet_params(chi=0.05)
    rows, cols = 5, 7
    wl = pad_workload(1.5e-3, rows, cols, params=p, wrap=wrap)
    _, _, (out,) = run(wl)
    fz = out["ft_clean"][2].reshape(rows, cols)
    assert np.allclose(fz, fz[0, 0], rtol=1e-12)
    nz = out["ft_noisy"][2].reshape(rows, cols)
    w = oracle.crosstalk_weights(1.0)
    for r in range(rows):
        for c in range(cols):
            inside = sum(w[di + 1, dj + 1] for di in (-1, 0, 1) for dj in (-1, 0, 1)
                         if 0 <= r + di < rows and (wrap or 0 <= c + dj < cols))
            assert np.isclose(nz[r, c], fz[r, c] * (1 - 0.05 + 0.05 * inside), rtol=1e-12)
    assert np.allclose(nz[1:-1, 1:-1], fz[1:-1, 1:-1], rtol=1e-12)


def test_crosstalk_of_a_point_source():
    p = quiet_params(chi=0.05)
    depths = np.full((3, 3), -1e-3); depths[1, 1] = 2e-3
    wl = pad_workload(depths, 3, 3, params=p)
    _, _, (out,) = run(wl)
    fz = out["ft_clean"][2].reshape(3, 3)
    nz = out["ft_noisy"][2].reshape(3, 3)
    w = oracle.crosstalk_weights(1.0)
    expect = 0.05 * w * fz[1, 1]
    expect[1, 1] += 0.95 * fz[1, 1]
    assert np.allclose(nz, expect, rtol=1e-12)


# ---------------------------------------------------------------- base noise (Eq. 25)
def test_drift_variance_grows_linearly():
    p = quiet_params()
    p["noise"]["ft"] = W.noise_group(sigma_rw=1e-3)
    wl = pad_workload(-1e-3, 40, 50, params=p)     # 2000 taxels, no contact
    _, _, outs = run(wl, steps=30)
    for t in (0, 9, 29):
        z = outs[t]["ft_noisy"].reshape(-1)
        var = (t + 1) * 1e-6
        n = z.size
        lo, hi = stats.chi2.ppf([1e-4, 1 - 1e-4], n) * var / n
        assert lo < np.mean(z * z) < hi


def test_white_noise_bias_quantisation():
    p = quiet_params()
    p["noise"]["depth"] = W.noise_group(bias=1e-3, sigma_white=2e-4)
    wl = pad_workload(-1e-3, 50, 40, params=p)
    _, _, (out,) = run(wl)
    z = out["depth_noisy"] - 1e-3
    assert abs(z.mean()) < 4 * 2e-4 / np.sqrt(z.size)
    assert abs(z.std() / 2e-4 - 1) < 0.06
    p["noise"]["depth"] = W.noise_group(quant=1e-4)
    wl = pad_workload(np.linspace(1e-5, 2e-3, 20).reshape(4, 5), 4, 5, params=p)
    _, _, (out,) = run(wl)
    assert np.allclose(out["depth_noisy"], 1e-4 * np.rint(out["depth_clean"] / 1e-4), atol=1e-18)


def test_gain_scales_reading():
    p = quiet_params()
    p["noise"]["depth"] = W.noise_group(gain_lo=1.5, gain_hi=1.5)
    wl = pad_workload(1e-3, 2, 3, params=p)
    _, _, (out,) = run(wl)
    assert np.allclose(out["depth_noisy"], 1.5 * out["depth_clean"], rtol=1e-15)
    p["noise"]["depth"] = W.noise_group(gain_lo=0.85, gain_hi=1.15)
    wl = pad_workload(1e-3, 20, 30, params=p)
    _, _, (out,) = run(wl)
    g = out["depth_noisy"] / out["depth_clean"]
    assert g.min() >= 0.85 and g.max() <= 1.15 and abs(g.mean() - 1.0) < 0.01


# ---------------------------------------------------------------- dead taxels (Eq. 28)
def test_dead_rate_and_stuck_for_episode():
    p = quiet_params(p_dead=0.3)
    p["noise"]["ft"] = W.noise_group(sigma_rw=1e-3, stuck_lo=0.0, stuck_hi=0.0)
    wl = pad_workload(1e-3, 100, 100, params=p)
    sc, st, outs = run(wl, steps=3)
    dead = (st["flags"] >> 1) & 1
    n = dead.size
    assert abs(dead.mean() - 0.3) < 4 * np.sqrt(0.3 * 0.7 / n)
    for out in outs:
        assert np.all(out["depth_noisy"][dead == 1] == 0.0)
        assert np.all(out["ft_noisy"][:, dead == 1] == 0.0)
        assert np.all(out["contact_noisy"][dead == 1] == 0)
        assert np.all(out["contact_noisy"][dead == 0] == out["contact_clean"][dead == 0])
    st2 = sc.new_state(); sc.reset(st2, 1)
    dead2 = (st2["flags"] >> 1) & 1
    assert abs(dead2.mean() - 0.3) < 4 * np.sqrt(0.3 * 0.7 / n)
    assert 0 < (dead != dead2).mean()
    st3 = sc.new_state(); sc.reset(st3, 0)
    assert np.array_equal((st3["flags"] >> 1) & 1, dead)


def test_stuck_value_range():
    p = quiet_params(p_dead=1.0)
    p["noise"]["depth"] = W.noise_group(stuck_lo=0.1, stuck_hi=0.2)
    wl = pad_workload(1e-3, 30, 30, params=p)
    _, _, (out,) = run(wl)
    z = out["depth_noisy"]
    assert z.min() >= 0.1 and z.max() <= 0.2 and stats.kstest((z - 0.1) / 0.1, "uniform").pvalue > 1e-3


# ---------------------------------------------------------------- links, fillers, scale
def test_link_sums_counts_and_agg_force():
    rng = np.random.default_rng(3)
    depths = rng.uniform(-1e-3, 2e-3, (3, 4))
    wl = pad_workload(depths, 3, 4, params=quiet_params())
    _, _, (out,) = run(wl)
    rec, cnt = out["link_sums"][0], out["link_counts"][0]
    d = out["depth_clean"]
    assert np.allclose(rec[0:3], [0, 0, K * d.sum()], atol=1e-12)
    x = np.stack([wl.x, wl.y, wl.z], 1).astype(float)
    assert np.allclose(rec[3:6], np.cross(x, np.c_[0 * d, 0 * d, K * d]).sum(0), atol=1e-12)
    assert cnt[0] == int((d > 5e-4).sum()) == out["contact_clean"].sum()
    # agg_force = 1e4 * ZYX(sum d_j n_j), n_j = (0, 0, -1)
    assert np.allclose(rec[12:15], [-1e4 * d.sum(), 0, 0], atol=1e-12)


def test_fillers_return_zero():
    p = W.default_params(5)
    p["noise"]["depth"] = W.noise_group(bias=0.3, sigma_rw=0.1, beta=0.1)
    wl = pad_workload(1e-3, 2, 5, params=p)
    wl.R[[1, 4, 7]] = 0.0
    _, st, outs = run(wl, steps=3)
    for out in outs:
        for k in ("depth_clean", "depth_noisy", "dist"):
            assert np.all(out[k][[1, 4, 7]] == 0.0)
        assert np.all(out["ft_clean"][:, [1, 4, 7]] == 0.0) and np.all(out["ft_noisy"][:, [1, 4, 7]] == 0.0)
        assert np.all(out["depth_noisy"][[0, 2, 3]] != 0.0)
    assert np.all((st["flags"][[1, 4, 7]] >> 1) == 0)


def test_object_scale_matches_scaled_sphere():
    p = quiet_params()
    wl = pad_workload(0.0, 1, 1, params=p)
    rng = np.random.default_rng(4)
    for s in (0.8, 1.0, 1.2):
        wl.objects = [W.ObjectSpec(kind="sphere", radius=0.03)]
        qs = rng.normal(size=3); qs *= (0.03 * s - 5e-4) / np.linalg.norm(qs)
        wl.link_pose[0, 0, :3] = qs; wl.link_pose[0, 0, 3:] = (1, 0, 0, 0)
        wl.x[:] = 0; wl.y[:] = 0; wl.z[:] = 0
        wl.env_params = np.array([[0.8, K, s]], np.float32)
        _, _, (out,) = run(wl)
        qf = wl.link_pose[0, 0, :3].astype(float)
        r = float(np.float32(0.03)) * float(np.float32(s))
        assert np.isclose(out["dist"][0], np.linalg.norm(qf) - r - float(np.float32(1e-3)), atol=1e-15)
