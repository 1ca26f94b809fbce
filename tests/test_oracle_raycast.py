"""Pins of the oracle's raycast depth backend ("Two contact-depth backends"):
per triangle a sphere-triangle closest-point test (R - dist) and a ray test
along the sensing direction (R - t); the deepest wins, with the face normal
of its triangle.  Closed forms on a plate and a cube (face, edge and vertex
regions), the property that the ray test is never deeper than the
closest-point test (the hit lies on the triangle), bounds on a tessellated
sphere and scale covariance.
"""
import numpy as np
import pytest

import oracle

PLATE_V = np.array([[-1, -1, 0], [1, -1, 0], [1, 1, 0], [-1, 1, 0]], np.float32)
PLATE_F = np.array([[0, 1, 2], [0, 2, 3]], np.int32)  # counter-clockwise seen from +z

CUBE_V = np.array([[x, y, z] for x in (-1, 1) for y in (-1, 1) for z in (-1, 1)], np.float32)


def _cube_faces():
    # outward-wound triangles of the cube [-1, 1]^3 (vertex index = 4 (x>0) + 2 (y>0) + (z>0))
    quads = [(0, 1, 3, 2), (4, 6, 7, 5), (0, 4, 5, 1), (2, 3, 7, 6), (0, 2, 6, 4), (1, 5, 7, 3)]
    F = []
    for a, b, c, d in quads:
        F += [(a, b, c), (a, c, d)]
    F = np.array(F, np.int32)
    # orient every triangle outward
    for i, (a, b, c) in enumerate(F):
        n = np.cross(CUBE_V[b] - CUBE_V[a], CUBE_V[c] - CUBE_V[a])
        if np.dot(n, CUBE_V[[a, b, c]].mean(0)) < 0:
            F[i] = (a, c, b)
    return F


CUBE_F = _cube_faces()


def test_probe_above_a_plate():
    R, h = 3e-3, 1e-3
    d, n, f, ray = oracle.raycast_depth(PLATE_V, PLATE_F, 1.0, [[0.2, -0.3, h]], [[0, 0, -1]], R)
    assert np.isclose(d[0], R - h, rtol=1e-12) and np.isclose(ray[0], R - h, rtol=1e-12)
    assert np.allclose(n[0], [0, 0, 1]) and f[0] in (0, 1)


def test_out_of_reach_reads_zero():
    d, n, f, ray = oracle.raycast_depth(PLATE_V, PLATE_F, 1.0, [[0.0, 0.0, 2e-3]], [[0, 0, -1]], 1e-3)
    assert d[0] == 0.0 and f[0] == -1 and np.all(n[0] == 0)
    assert np.isclose(ray[0], 1e-3 - 2e-3)  # the ray hits 2 mm away: no penetration
    d, _, f, ray = oracle.raycast_depth(PLATE_V, PLATE_F, 1.0, [[0.0, 0.0, 2e-3]], [[0, 0, 1]], 1e-3)
    assert d[0] == 0.0 and f[0] == -1 and ray[0] == -np.inf  # pointing away: no hit at all


def test_slanted_ray_is_shallower_than_the_closest_point():
    R, h, th = 3e-3, 1e-3, 0.5
    u = [np.sin(th), 0.0, -np.cos(th)]
    d, _, _, ray = oracle.raycast_depth(PLATE_V, PLATE_F, 1.0, [[0.0, 0.0, h]], [u], R)
    assert np.isclose(ray[0], R - h / np.cos(th), rtol=1e-12)
    assert np.isclose(d[0], R - h, rtol=1e-12)


@pytest.mark.parametrize("off,normals", [((0.4e-3, 0.7e-3, 0.0), ((1, 0, 0), (0, 1, 0))),
                                         ((0.4e-3, 0.7e-3, 0.5e-3), ((1, 0, 0), (0, 1, 0), (0, 0, 1)))])
def test_cube_edge_and_vertex_distance(off, normals):
    R = 2e-3
    q = np.array([1 + off[0], 1 + off[1], (1 + off[2]) if off[2] else 0.0])
    d, n, _, _ = oracle.raycast_depth(CUBE_V, CUBE_F, 1.0, [q], [[-1, 0, 0]], R)
    assert np.isclose(d[0], R - np.linalg.norm(off), rtol=1e-9)
    assert any(np.allclose(n[0], m) for m in normals)  # a face adjacent to the nearest edge or vertex


def _icosphere(r, levels):
    t = (1 + 5 ** 0.5) / 2
    V = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    F = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2),
         (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11),
         (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    V = [np.array(v, float) / np.linalg.norm(v) for v in V]
    for _ in range(levels):
        mid = {}

        def m(a, b):
            k = (min(a, b), max(a, b))
            if k not in mid:
                p = V[a] + V[b]
                V.append(p / np.linalg.norm(p))
                mid[k] = len(V) - 1
            return mid[k]

        F = [f for a, b, c in F for f in ((a, m(a, b), m(c, a)), (b, m(b, c), m(a, b)), (c, m(c, a), m(b, c)),
                                           (m(a, b), m(b, c), m(c, a)))]
    return (np.array(V) * r).astype(np.float32), np.array(F, np.int32)


def test_tessellated_sphere_bounds_and_the_ray_never_wins():
    r = 0.02
    V, F = _icosphere(r, 2)
    tri = V[F].astype(np.float64)
    r_in = min(abs(np.dot(np.cross(b - a, c - a) / np.linalg.norm(np.cross(b - a, c - a)), a)) for a, b, c in tri)
    rng = np.random.default_rng(0)
    dirs = rng.standard_normal((60, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    rho = r + rng.uniform(-2e-3, 2e-3, 60)
    q = dirs * rho[:, None]
    u = -dirs + 0.3 * rng.standard_normal((60, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    R = 3e-3
    d, n, f, ray = oracle.raycast_depth(V, F, 1.0, q, u, R)
    outside = rho > r
    # outside the sphere the nearest surface point is between the inscribed and circumscribed spheres
    assert np.all(d[outside] <= R - (rho[outside] - r) + 1e-12)
    assert np.all(d[outside] >= np.maximum(R - (rho[outside] - r_in), 0) - 1e-12)
    assert np.all(ray <= d + 1e-15)  # the ray test never beats the closest-point test
    hit = d > 0
    assert np.all(np.einsum("ij,ij->i", n[hit], dirs[hit]) > 0.9)  # outward face normals


def test_scale_covariance():
    V, F = _icosphere(0.01, 1)
    q = np.array([[0.0105, 0.001, -0.002]])
    d1, n1, f1, _ = oracle.raycast_depth(V, F, 1.0, q, [[-1, 0, 0]], 2e-3)
    s = 1.7
    d2, n2, f2, _ = oracle.raycast_depth(V, F, s, q * s, [[-1, 0, 0]], 2e-3 * s)
    assert np.isclose(d2[0], s * d1[0], rtol=1e-9) and f1[0] == f2[0] and np.allclose(n1, n2)
