"""Pins of the oracle's point-cloud ProximityTaxel (Appendix A "ProximityTaxel")
against closed forms: one flat pad taxel (normal -z) over an object at the
origin whose tracked points are placed by hand.  For a point at p inside the
sensing sphere of radius R around the taxel at q (normal a):
P = R - |p - q|, f = k rho P a + ks rho P v_t, tau = k rho P (p - q) x a,
rho = density / N, reported in the link frame.
"""
import numpy as np
from scipy.spatial.transform import Rotation

from paper_2606_22332_gb300 import workload as W
from _scenes import oracle_scene, pad_workload, quiet_params

RPC, K, KS, DENS = 0.01, 300.0, 10.0, 100.0


def _taxel(depth=0.0):
    """One taxel; its world position (the pad link at height 0.01, identity)."""
    wl = pad_workload(depth, 1, 1, params=quiet_params())
    q = np.array([wl.x[0], wl.y[0], 0.01 + wl.z[0]], np.float64)
    return wl, q


def _pc(wl, cloud, step=0, **inp):
    sc = oracle_scene(wl)
    i = dict(wl.inputs(step), **inp)
    return sc.pc_prox([np.asarray(cloud, np.float64)], i, RPC, K, KS, DENS)[:, 0]


def test_point_on_the_normal_axis():
    wl, q = _taxel()
    r = 0.004
    ft = _pc(wl, [q + r * np.array([0, 0, -1.0])])   # along a = -z
    P = RPC - r
    assert np.allclose(ft, [0, 0, -K * DENS * P, 0, 0, 0], rtol=1e-6, atol=1e-9)


def test_points_outside_the_sphere_give_zero():
    wl, q = _taxel()
    ft = _pc(wl, [q + np.array([0.0, 0.0, -0.0101]), q + np.array([0.008, 0.007, 0.0])])
    assert np.all(ft == 0.0)


def test_symmetric_ring_cancels_shear_and_torque():
    wl, q = _taxel()
    n, rr, h = 8, 0.003, 0.005
    th = 2 * np.pi * np.arange(n) / n
    ring = q + np.stack([rr * np.cos(th), rr * np.sin(th), -h * np.ones(n)], 1)
    ft = _pc(wl, ring)
    P = RPC - np.hypot(rr, h)
    rho = DENS / n
    assert np.allclose(ft[:3], [0, 0, -K * rho * n * P], rtol=1e-6, atol=1e-9)
    assert np.allclose(ft[3:], 0.0, atol=1e-9)


def test_moving_object_shear_keeps_only_the_tangential_velocity():
    wl, q = _taxel()
    r = 0.004
    v = np.array([0.2, -0.1, 0.5])   # the normal part (z) must drop out
    wl.obj_vel = np.asarray([[*v, 0, 0, 0]], np.float32)
    ft = _pc(wl, [q + r * np.array([0, 0, -1.0])])
    P = RPC - r
    vt = np.array([v[0], v[1], 0.0]).astype(np.float32).astype(np.float64)
    expect = K * DENS * P * np.array([0, 0, -1.0]) + KS * DENS * P * vt
    assert np.allclose(ft[:3], expect, rtol=1e-6, atol=1e-9)


def test_density_divides_by_the_tracked_point_count():
    wl, q = _taxel()
    near = q + 0.004 * np.array([0, 0, -1.0])
    far = q + np.array([0.0, 0.0, -0.5])
    f1 = _pc(wl, [near])
    f4 = _pc(wl, [near, far, far, far])
    assert np.allclose(f4, f1 / 4, rtol=1e-12)


def test_link_frame_output_is_invariant_under_a_rigid_rotation_of_the_scene():
    wl, q = _taxel()
    pts = q + np.array([[0.001, -0.002, -0.004], [-0.003, 0.0015, -0.006], [0.002, 0.002, -0.002]])
    ft0 = _pc(wl, pts)
    Rot = Rotation.from_rotvec([0.3, -0.5, 0.8])
    # rotate the link about the world origin: its pose and, with the object, every tracked point
    qw = Rot.as_quat()  # x, y, z, w
    lp = wl.link_pose.copy()
    lp[0, 0, :3] = Rot.apply(lp[0, 0, :3].astype(np.float64))
    lp[0, 0, 3:] = [qw[3], qw[0], qw[1], qw[2]]
    op = wl.obj_pose.copy()
    op[0, 3:] = [qw[3], qw[0], qw[1], qw[2]]           # the object (the cloud's frame) rotates too
    wl.link_pose, wl.obj_pose = lp.astype(np.float32), op.astype(np.float32)
    ft1 = _pc(wl, pts)
    assert np.allclose(ft1, ft0, rtol=1e-5, atol=1e-7 * np.abs(ft0).max())


def test_object_scale_scales_the_cloud():
    wl, q = _taxel()
    s = 1.25
    p_hat = (q + 0.004 * np.array([0, 0, -1.0])) / s   # object frame, unscaled
    inp = wl.inputs(0)
    env = np.asarray([[0.8, 1e4, s]], np.float32)
    ft = _pc(wl, [p_hat], env_params=env)
    r = np.linalg.norm(s * p_hat - q)
    assert np.allclose(ft, [0, 0, -K * DENS * (RPC - r), 0, 0, 0], rtol=1e-6, atol=1e-9)
