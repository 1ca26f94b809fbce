"""Pins of the oracle's ElastomerTaxel shear anchors (Eqs. 19-20).

Scene: one env, an identity link at height 0.01 carrying one 15 x 15 pad
(1 mm pitch) at the link origin, normal +z, tangent +x (bitangent +y), so a
point's pad coordinates are its world offset from (0, 0, 0.01).  The elastomer
is the box under the pad: 15 mm x 15 mm, `thickness` deep.  The env object
carries a hand-placed cloud and is moved by its pose.  Closed forms: a point
anchors at e = (z_t, z_b) once its elastomer SDF is below -eta_enter, lets go
above +eta_exit, and while anchored with penetration h moves marker j at
(a_j, b_j) by s_s (z - e)_tangential h exp(-lambda_s |(a_j, b_j) - z_tangential|^2).
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from paper_2606_22332_gb300 import workload as W
from _scenes import oracle_scene, pad_workload, quiet_params

SH = dict(s_s=100.0, lambda_s=2000.0, eta_enter=1e-5, eta_exit=1e-4, thickness=2e-3)
H0 = 0.01   # link height
HALF = 7.5e-3


def _setup(n_objects=1, n_max=8):
    wl = pad_workload(-1e-3, 1, 1, params=quiet_params())
    wl.objects = [W.ObjectSpec(kind="sphere", radius=0.01) for _ in range(n_objects)]
    pads = dict(pads_per_env=1, rows=15, cols=15, pitch=1e-3, pad_link=np.zeros((1, 1), np.int32),
                pad_frame=np.array([[[0, 0, 0, 0, 0, 1, 1, 0, 0]]], np.float32),
                s_d=1.0, alpha=1.2, lambda_d=1.0 / (2 * 1.5e-3 ** 2), c=1.0, eps=1e-3, radius=2)
    sc = oracle_scene(wl)
    return wl, pads, sc, sc.new_shear_state(1, n_max)


def _inp(wl, pos, oid=0, quat=(1, 0, 0, 0), link_pose=None, scale=None):
    op = np.zeros((1, 7), np.float32)
    op[0, :3] = pos
    op[0, 3:] = quat
    inp = dict(wl.inputs(0), obj_pose=op, obj_id=np.array([oid], np.int32), pose_dt=0.0)
    if link_pose is not None:
        inp["link_pose"] = link_pose
    if scale is not None:
        inp["env_params"] = np.asarray([[0.8, 1e4, scale]], np.float32)
    return inp


def _z(pos):
    """pad coordinates of a cloud point at the object origin with the object at `pos` (float32 inputs)"""
    p = np.asarray(pos, np.float32).astype(np.float64)
    return np.array([p[0], p[1], p[2] - float(np.float32(H0))])


def _marker_ab():
    r, c = np.meshgrid(np.arange(15), np.arange(15), indexing="ij")
    return ((r - 7) * 1e-3).reshape(-1), ((c - 7) * 1e-3).reshape(-1)


def _expect(z, e, h):
    a, b = _marker_ab()
    g = np.exp(-SH["lambda_s"] * ((a - z[0]) ** 2 + (b - z[1]) ** 2))
    u = np.zeros((225, 3))
    u[:, 1] = SH["s_s"] * (z[0] - e[0]) * h * g
    u[:, 2] = SH["s_s"] * (z[1] - e[1]) * h * g
    return u


def _step(sc, wl, pads, st, pos, cloud=((0, 0, 0),), **kw):
    clouds = [np.asarray(cloud, np.float64)] * len(wl.objects)
    u, na, mg = sc.shear_step(pads, clouds, SH, _inp(wl, pos, **kw), st)
    return u[0, 0], int(na[0, 0]), float(mg[0, 0])


def test_drag_of_an_anchored_point_closed_form():
    wl, pads, sc, st = _setup()
    p0 = (0.0, 0.0, H0 - 5e-4)
    u, na, _ = _step(sc, wl, pads, st, p0)
    z0 = _z(p0)
    assert na == 1 and np.all(u == 0.0)                       # anchored where it is: z - e = 0
    assert np.allclose(st["anchors"][0, 0, 0], z0[:2], rtol=0, atol=0)
    p1 = (2e-4, -1e-4, H0 - 4e-4)
    u, na, _ = _step(sc, wl, pads, st, p1)
    z1 = _z(p1)
    assert na == 1
    assert np.allclose(u, _expect(z1, z0, -z1[2]), rtol=1e-12, atol=0)
    assert np.all(u[:, 0] == 0.0)                             # the tangential projection leaves no normal part


def test_enter_and_exit_hysteresis_keeps_shear_history():
    wl, pads, sc, st = _setup()
    # shallower than eta_enter: in contact, but no anchor and no shear
    u, na, _ = _step(sc, wl, pads, st, (0.0, 0.0, H0 - 5e-6))
    assert na == 0 and np.all(u == 0.0)
    # pressed in: anchors at (0, 0)
    u, na, _ = _step(sc, wl, pads, st, (0.0, 0.0, H0 - 5e-4))
    assert na == 1 and np.all(u == 0.0)
    e = _z((0.0, 0.0, H0 - 5e-4))[:2]
    # lifted 50 um above the surface (below eta_exit): the anchor stays, h = 0 so no shear
    u, na, _ = _step(sc, wl, pads, st, (0.0, 0.0, H0 + 5e-5))
    assert na == 1 and np.all(u == 0.0)
    # pressed again 1 mm away: sheared against the old anchor
    p = (1e-3, 0.0, H0 - 3e-4)
    u, na, _ = _step(sc, wl, pads, st, p)
    z = _z(p)
    assert na == 1 and np.allclose(u, _expect(z, e, -z[2]), rtol=1e-12, atol=0)
    # lifted above eta_exit: released
    u, na, _ = _step(sc, wl, pads, st, (1e-3, 0.0, H0 + 2e-4))
    assert na == 0 and np.all(np.isnan(st["anchors"][0, 0, 0]))
    # pressed again: a fresh anchor where it is, no shear
    u, na, _ = _step(sc, wl, pads, st, p)
    assert na == 1 and np.all(u == 0.0)
    assert np.allclose(st["anchors"][0, 0, 0], z[:2], rtol=0, atol=0)


def test_elastomer_is_the_box_under_the_pad():
    wl, pads, sc, st = _setup()
    # beside the footprint, below the surface plane: outside the elastomer
    u, na, _ = _step(sc, wl, pads, st, (HALF + 1e-3, 0.0, H0 - 5e-4))
    assert na == 0 and np.all(u == 0.0)
    # below the elastomer's bottom face (thickness 2 mm): outside too
    u, na, _ = _step(sc, wl, pads, st, (0.0, 0.0, H0 - 3e-3))
    assert na == 0 and np.all(u == 0.0)
    # 30 um inside a side face, 0.5 mm deep: the side face is the nearest, h = 30 um
    p0 = (HALF - 3e-5, 0.0, H0 - 5e-4)
    _step(sc, wl, pads, st, p0)
    p1 = (HALF - 3e-5, 2e-4, H0 - 5e-4)
    u, na, _ = _step(sc, wl, pads, st, p1)
    z0, z1 = _z(p0), _z(p1)
    h = HALF - z1[0]
    assert na == 1 and abs(h - 3e-5) < 1e-9
    assert np.allclose(u, _expect(z1, z0, h), rtol=1e-12, atol=0)


def test_points_superpose():
    wl, pads, sc, st = _setup()
    c2 = ((0, 0, 0), (3e-3, -2e-3, 1e-4))
    p0, p1 = (0.0, 0.0, H0 - 5e-4), (-4e-4, 3e-4, H0 - 3e-4)
    _step(sc, wl, pads, st, p0, cloud=c2)
    u2, na2, _ = _step(sc, wl, pads, st, p1, cloud=c2)
    parts = []
    for c in c2:
        _, _, scc, s1 = _setup()
        _step(scc, wl, pads, s1, p0, cloud=(c,))
        parts.append(_step(scc, wl, pads, s1, p1, cloud=(c,)))
    assert na2 == parts[0][1] + parts[1][1] == 2
    assert np.allclose(u2, parts[0][0] + parts[1][0], rtol=1e-12, atol=1e-300)
    assert np.abs(parts[1][0]).max() > 0


def test_output_is_invariant_under_a_rigid_motion_of_the_scene():
    wl, pads, sc, st = _setup()
    cloud = ((0, 0, 0), (1e-3, 2e-3, 2e-4), (-2e-3, 1e-3, 1e-4))
    seq = [(0.0, 0.0, H0 - 5e-4), (3e-4, -2e-4, H0 - 4e-4)]
    ref = [_step(sc, wl, pads, st, p, cloud=cloud) for p in seq]
    Rot = Rotation.from_rotvec([0.4, -0.7, 0.2])
    qw = Rot.as_quat()
    quat = (qw[3], qw[0], qw[1], qw[2])
    lp = wl.link_pose.copy()
    lp[0, 0, :3] = Rot.apply([0.0, 0.0, H0])
    lp[0, 0, 3:] = quat
    _, _, sc2, st2 = _setup()
    for p, (u0, na0, _) in zip(seq, ref):
        u, na, _ = _step(sc2, wl, pads, st2, Rot.apply(np.asarray(p, np.float64)), cloud=cloud, quat=quat,
                         link_pose=lp.astype(np.float32))
        assert na == na0
        assert np.allclose(u, u0, rtol=2e-4, atol=1e-5 * np.abs(u0).max())
    assert np.abs(ref[1][0]).max() > 0


def test_a_new_object_clears_the_anchors():
    wl, pads, sc, st = _setup(n_objects=2)
    _step(sc, wl, pads, st, (0.0, 0.0, H0 - 5e-4), oid=0)
    u, na, _ = _step(sc, wl, pads, st, (5e-4, 0.0, H0 - 5e-4), oid=1)
    assert na == 1 and np.all(u == 0.0) and st["anchor_obj"][0, 0] == 1
    u, na, _ = _step(sc, wl, pads, st, (5e-4, 0.0, H0 - 5e-4), oid=0)
    assert np.all(u == 0.0) and st["anchor_obj"][0, 0] == 0


def test_object_scale_scales_the_cloud():
    wl, pads, sc, st = _setup()
    s = 2.0
    cloud = ((1e-3, 0, 0),)
    _step(sc, wl, pads, st, (0.0, 0.0, H0 - 5e-4), cloud=cloud, scale=s)
    p1 = (0.0, 3e-4, H0 - 5e-4)
    u, na, _ = _step(sc, wl, pads, st, p1, cloud=cloud, scale=s)
    off = [s * float(np.float32(1e-3)), 0, 0]   # the cloud is read as float32
    z0 = _z((0.0, 0.0, H0 - 5e-4)) + off
    z1 = _z(p1) + off
    assert na == 1 and np.allclose(u, _expect(z1, z0, -z1[2]), rtol=1e-12, atol=0)


@pytest.mark.parametrize("depth", [9e-6, 1.1e-5])
def test_enter_threshold_is_strict(depth):
    wl, pads, sc, st = _setup()
    _, na, mg = _step(sc, wl, pads, st, (0.0, 0.0, H0 - depth))
    assert na == (1 if depth > SH["eta_enter"] else 0)
    assert mg > 0
