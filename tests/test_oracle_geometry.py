"""Pins of the oracle's geometry: poses, analytic SDFs, exact mesh distance,
winding number, the sampled-grid query and the grid bake.

Each check compares against something other than the oracle's own formula:
scipy's rotation routines, closed forms worked by hand, brute-force
sampling, an independent analytic SDF, or scipy's grid interpolator.
"""
import numpy as np
import pytest
from scipy.interpolate import RegularGridInterpolator
from scipy.spatial.transform import Rotation

import oracle
from paper_2606_22332_gb300 import workload as W


# ---------------------------------------------------------------- poses
def test_quat_to_mat_matches_scipy():
    rng = np.random.default_rng(1)
    for _ in range(50):
        q = rng.normal(size=4)
        R = oracle.quat_to_mat(q)
        ref = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()  # scipy is scalar-last
        assert np.allclose(R, ref, atol=1e-14)


def test_quat_to_mat_known_rotation():
    c = np.cos(np.pi / 4)
    R = oracle.quat_to_mat([c, 0, 0, c])  # +90 deg about z
    assert np.allclose(R @ [1, 0, 0], [0, 1, 0], atol=1e-15)
    assert np.allclose(R @ [0, 1, 0], [-1, 0, 0], atol=1e-15)


def test_advance_pose_matches_scipy():
    rng = np.random.default_rng(2)
    for _ in range(30):
        p0, v, w = rng.normal(size=3), rng.normal(size=3), rng.normal(size=3)
        q0 = rng.normal(size=4)
        tau = rng.uniform(0, 2)
        p, R = oracle.advance_pose(p0, q0, v, w, tau)
        R0 = Rotation.from_quat([q0[1], q0[2], q0[3], q0[0]])
        ref = (Rotation.from_rotvec(w * tau) * R0).as_matrix()
        assert np.allclose(R, ref, atol=1e-13)
        assert np.allclose(p, p0 + v * tau, atol=1e-15)
    p, R = oracle.advance_pose([1, 2, 3], [1, 0, 0, 0], [0, 0, 0], [0, 0, 0], 5.0)
    assert np.array_equal(R, np.eye(3))


# ---------------------------------------------------------------- analytic SDFs
def test_sphere_sdf_closed_form():
    s = oracle.Obj.sphere(0.03)
    phi, g = s.sdf([[0.05, 0, 0], [0, 0.01, 0], [0.02, 0.02, 0.01]])
    assert np.allclose(phi, [0.02, -0.02, 0.03 - 0.03], atol=1e-16)
    assert np.allclose(g[0], [1, 0, 0]) and np.allclose(g[1], [0, 1, 0])
    assert np.allclose(g[2], np.array([2, 2, 1]) / 3)


def test_box_sdf_hand_values():
    b = oracle.Obj.box([1.0, 2.0, 3.0])
    pts = [[0, 0, 0], [0.5, 0, 0], [0, -1.5, 0], [2, 3, 4], [2, 3, 0], [-2, 0, 0], [0, 0, -3.25]]
    phi, g = b.sdf(pts)
    assert np.allclose(phi, [-1, -0.5, -0.5, np.sqrt(3), np.sqrt(2), 1, 0.25])
    assert np.allclose(g[0], [1, 0, 0]) or np.allclose(g[0], [-1, 0, 0])
    assert np.allclose(g[2], [0, -1, 0])
    assert np.allclose(g[3], np.ones(3) / np.sqrt(3))
    assert np.allclose(g[4], [1 / np.sqrt(2), 1 / np.sqrt(2), 0])
    assert np.allclose(g[5], [-1, 0, 0])
    assert np.allclose(g[6], [0, 0, -1])


def test_plane_sdf():
    phi, g = oracle.Obj.plane().sdf([[3, 4, 0.2], [0, 0, -0.1]])
    assert np.allclose(phi, [0.2, -0.1]) and np.allclose(g, [[0, 0, 1], [0, 0, 1]])


# ---------------------------------------------------------------- triangles
A, B, C = np.array([0.0, 0, 0]), np.array([1.0, 0, 0]), np.array([0.0, 1, 0])


@pytest.mark.parametrize("p,cp,region", [
    ([0.2, 0.2, 0.5], [0.2, 0.2, 0.0], 0),      # above the face
    ([-1, -1, 0.3], [0, 0, 0], 1),              # vertex a
    ([2, -0.5, 0], [1, 0, 0], 2),               # vertex b
    ([-0.2, 3, 1], [0, 1, 0], 3),               # vertex c
    ([0.5, -2, 0], [0.5, 0, 0], 4),             # edge ab
    ([-2, 0.4, -1], [0, 0.4, 0], 5),            # edge ac
    ([1, 1, 0], [0.5, 0.5, 0], 6),              # edge bc
])
def test_closest_point_regions_by_hand(p, cp, region):
    d, got, reg = oracle.closest_point_triangle(p, A, B, C)
    assert reg == region
    assert np.allclose(got, cp, atol=1e-15)
    assert np.isclose(d, np.linalg.norm(np.asarray(p) - cp))


def test_closest_point_brute_force():
    rng = np.random.default_rng(3)
    n = 400
    uu, vv = np.meshgrid(np.linspace(0, 1, n + 1), np.linspace(0, 1, n + 1))
    keep = uu + vv <= 1
    bary = np.stack([uu[keep], vv[keep]], 1)
    for _ in range(25):
        a, b, c = rng.normal(size=(3, 3))
        pts = a + bary[:, :1] * (b - a) + bary[:, 1:] * (c - a)
        p = rng.normal(size=3) * 2
        d, cp, _ = oracle.closest_point_triangle(p, a, b, c)
        brute = np.linalg.norm(pts - p, axis=1).min()
        h = max(np.linalg.norm(b - a), np.linalg.norm(c - a)) / n
        assert d <= brute + 1e-12
        assert brute - d <= 2 * h


# ---------------------------------------------------------------- meshes
def cube_mesh(h):
    V = np.array([[x, y, z] for x in (-h, h) for y in (-h, h) for z in (-h, h)])
    from scipy.spatial import ConvexHull
    F = ConvexHull(V).simplices
    F = W.orient_outward(V, F)
    return W.f32(V), F.astype(np.int32)


def icosphere(level):
    t = (1 + 5 ** 0.5) / 2
    V = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0], [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], float)
    from scipy.spatial import ConvexHull
    F = W.orient_outward(V, ConvexHull(V).simplices)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    for _ in range(level):
        V, F = W.subdivide(V, F)
        V /= np.linalg.norm(V, axis=1, keepdims=True)
    return V, F


def test_winding_number_closed_meshes():
    V, F = cube_mesh(1.0)
    assert np.isclose(oracle.winding_number(V, F, [0.1, 0.2, -0.3]), 1.0, atol=1e-12)
    assert np.isclose(oracle.winding_number(V, F, [3, 0, 0]), 0.0, atol=1e-12)
    assert np.isclose(oracle.winding_number(V, F[:, [0, 2, 1]], [0.1, 0.2, -0.3]), -1.0, atol=1e-12)
    Vt = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], np.float32)
    Ft = W.orient_outward(Vt.astype(float), np.array([[0, 1, 2], [0, 1, 3], [0, 2, 3], [1, 2, 3]])).astype(np.int32)
    assert np.isclose(oracle.winding_number(Vt, Ft, [0.1, 0.1, 0.1]), 1.0, atol=1e-12)
    assert np.isclose(oracle.winding_number(Vt, Ft, [0.5, 0.5, 0.5]), 0.0, atol=1e-12)


def test_mesh_sdf_equals_box_sdf_on_cube():
    V, F = cube_mesh(0.02)
    h = float(np.float32(0.02))  # the mesh stores float32 vertices
    mesh, box = oracle.Obj.mesh(V, F), oracle.Obj.box([h, h, h])
    rng = np.random.default_rng(4)
    q = rng.uniform(-0.04, 0.04, (2000, 3))
    pm, gm = mesh.sdf(q)
    pb, gb = box.sdf(q)
    assert np.allclose(pm, pb, atol=1e-15)
    # gradients agree wherever the nearest feature is unique (off the medial set)
    a = np.sort(np.abs(np.abs(q) - h), axis=1)
    ok = (pb > 1e-4) | ((pb < 0) & (a[:, 1] - a[:, 0] > 1e-4))
    assert np.allclose(gm[ok], gb[ok], atol=1e-9)


def test_mesh_sdf_converges_to_sphere():
    errs = []
    rng = np.random.default_rng(5)
    q = rng.normal(size=(300, 3)); q *= (rng.uniform(0.3, 1.7, (300, 1)) / np.linalg.norm(q, axis=1, keepdims=True))
    sph = oracle.Obj.sphere(1.0)
    ps, _ = sph.sdf(q)
    for lvl in (2, 3, 4):
        V, F = icosphere(lvl)
        pm, _ = oracle.Obj.mesh(V.astype(np.float32), F.astype(np.int32)).sdf(q)
        errs.append(np.abs(pm - ps).max())
    # chordal error of a subdivided icosphere shrinks ~4x per level (O(h^2))
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0
    assert errs[2] < 2e-3


def test_mesh_sdf_inside_convex_hull_is_plane_distance():
    rng = np.random.default_rng(6)
    V, F = W.hull_mesh(rng, 64, 0.04)
    Vd = V.astype(np.float64)
    n = np.cross(Vd[F[:, 1]] - Vd[F[:, 0]], Vd[F[:, 2]] - Vd[F[:, 0]])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    off = np.einsum("ij,ij->i", n, Vd[F[:, 0]])
    q = rng.normal(0, 0.004, (500, 3))
    plane = (q @ n.T - off)          # signed plane distances, negative inside
    inside = (plane < 0).all(axis=1)
    assert inside.sum() > 100
    pm, _ = oracle.Obj.mesh(V, F).sdf(q[inside])
    assert np.allclose(pm, plane[inside].max(axis=1), atol=1e-12)


# ---------------------------------------------------------------- grids
def _grid(values, lo, hi, fp16=False):
    return oracle.Obj.grid(values, lo, hi, fp16=fp16)


def test_grid_exact_at_nodes_and_matches_scipy():
    rng = np.random.default_rng(7)
    nx, ny, nz = 7, 5, 6
    vals = rng.normal(size=(nz, ny, nx)).astype(np.float32)
    lo, hi = np.array([-1.0, -2.0, 0.5]), np.array([2.0, 1.0, 3.0])
    g = _grid(vals, lo, hi)
    xs = [np.linspace(lo[a], hi[a], n) for a, n in zip(range(3), (nx, ny, nz))]
    nodes = np.stack(np.meshgrid(*xs, indexing="ij"), -1).reshape(-1, 3)
    phi, _ = g.sdf(nodes)
    ref = vals.transpose(2, 1, 0).reshape(-1).astype(np.float64)
    assert np.allclose(phi, ref, atol=1e-14)
    interp = RegularGridInterpolator(xs, vals.transpose(2, 1, 0).astype(np.float64))
    q = rng.uniform(lo, hi, (1000, 3))
    phi, _ = g.sdf(q)
    assert np.allclose(phi, interp(q), atol=1e-13)


def test_grid_reproduces_linear_field_and_gradient():
    n = 9
    lo, hi = np.array([-0.02, -0.03, -0.01]), np.array([0.03, 0.02, 0.04])
    a, b = np.array([0.3, -0.5, 0.8]), 0.004
    xs = [np.linspace(lo[i], hi[i], n) for i in range(3)]
    X, Y, Z = np.meshgrid(*xs, indexing="ij")
    vals = (a[0] * X + a[1] * Y + a[2] * Z + b).transpose(2, 1, 0)
    g = _grid(vals.astype(np.float32), lo, hi)
    rng = np.random.default_rng(8)
    q = rng.uniform(lo, hi, (500, 3))
    phi, grad = g.sdf(q)
    # the stored float32 values are the field rounded; compare to the rounding size
    assert np.allclose(phi, q @ a + b, atol=1e-8)
    assert np.allclose(grad, a / np.linalg.norm(a), atol=1e-5)


def test_grid_outside_box_adds_distance():
    vals = np.zeros((4, 4, 4), np.float32)
    g = _grid(vals, [0, 0, 0], [1, 1, 1])
    phi, _ = g.sdf([[2.0, 0.5, 0.5], [-1, -1, 0.5], [0.5, 0.5, 0.5]])
    assert np.allclose(phi, [1.0, np.sqrt(2), 0.0])


def test_grid_fp16_values_widened_exactly():
    rng = np.random.default_rng(9)
    v = rng.normal(0, 0.01, (3, 3, 3)).astype(np.float16)
    g = _grid(v.view(np.uint16), [0, 0, 0], [1, 1, 1], fp16=True)
    nodes = np.array([[i / 2, j / 2, k / 2] for k in range(3) for j in range(3) for i in range(3)])
    phi, _ = g.sdf(nodes)
    assert np.array_equal(phi, v.reshape(-1).astype(np.float64))


def test_bake_cube_matches_box_sdf():
    V, F = cube_mesh(0.02)
    dims = np.array([11, 9, 10])
    lo, hi = np.array([-0.03, -0.03, -0.03]), np.array([0.03, 0.03, 0.03])
    grid = oracle.bake_grid(V, F, dims, lo, hi)
    xs = [lo[i] + np.arange(dims[i]) * ((hi[i] - lo[i]) / (dims[i] - 1)) for i in range(3)]
    nodes = np.stack(np.meshgrid(*xs, indexing="ij"), -1).reshape(-1, 3)
    h = float(np.float32(0.02))
    pb, _ = oracle.Obj.box([h, h, h]).sdf(nodes)
    ref = pb.reshape(dims[0], dims[1], dims[2]).transpose(2, 1, 0).astype(np.float32)
    assert np.array_equal(grid, ref)
    g16 = oracle.bake_grid(V, F, dims, lo, hi, fp16=True)
    assert np.array_equal(g16, pb.reshape(dims[0], dims[1], dims[2]).transpose(2, 1, 0).astype(np.float16).view(np.uint16))
