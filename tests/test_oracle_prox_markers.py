"""Pins of the oracle's proximity rays and elastomer markers.

Proximity: the first root along a ray against closed forms (sphere, plane,
box, a cube mesh), a sampled linear field (trilinear reproduces it), and
brute-force sampling of a sampled sphere grid; the ray fan; the 8-ray
reading of a probe facing a plane in closed form.  Markers: the peak
normalisations g_bar and rho_bar, a single penetrating source in closed form
(Gaussian and inverse-distance limits), a uniform depth field (interior
tangential cancellation, normal sum of the kernel), and no contact.
"""
import numpy as np
import pytest

import oracle
from paper_2606_22332_gb300 import workload as W
from _scenes import oracle_scene, pad_workload, quiet_params
from test_oracle_geometry import cube_mesh

RANGE = 0.05


# ---------------------------------------------------------------- first roots
def test_sphere_root_closed_form():
    s = oracle.Obj.sphere(0.03)
    for b in (0.0, 0.01, 0.02, 0.029):
        t, g = oracle.ray_first_root(s, [0.05, b, 0.0], [-1.0, 0.0, 0.0], RANGE)
        assert np.isclose(t, 0.05 - np.sqrt(0.03 ** 2 - b ** 2), atol=1e-15)
    t, g = oracle.ray_first_root(s, [0.06, 0.031, 0.0], [-1.0, 0.0, 0.0], RANGE)
    assert np.isnan(t) and not g
    t, g = oracle.ray_first_root(s, [0.04, 0.03 + 5e-6, 0.0], [-1.0, 0.0, 0.0], RANGE)
    assert np.isnan(t) and g                                # near miss flagged
    t, g = oracle.ray_first_root(s, [0.04, 0.03 - 1e-7, 0.0], [-1.0, 0.0, 0.0], RANGE)
    assert not np.isnan(t) and g                            # shallow crossing flagged
    t, _ = oracle.ray_first_root(s, [0.01, 0.0, 0.0], [1.0, 0.0, 0.0], RANGE)
    assert t == 0.0                                          # origin inside
    t, _ = oracle.ray_first_root(s, [0.09, 0.0, 0.0], [-1.0, 0.0, 0.0], RANGE)
    assert np.isnan(t)                                       # beyond the range


def test_scaled_sphere_root():
    s = oracle.Obj.sphere(0.03)
    for sc in (0.8, 1.2):
        q = np.array([0.07, 0.0, 0.0])
        # object frame: q / s, direction d / s; the root in world units
        t, _ = oracle.ray_first_root(s, q / sc, np.array([-1.0, 0, 0]) / sc, RANGE, scale=sc)
        assert np.isclose(t, 0.07 - 0.03 * sc, atol=1e-15)


def test_plane_and_box_roots():
    p = oracle.Obj.plane()
    th = 0.3
    t, _ = oracle.ray_first_root(p, [0, 0, 0.01], [0, np.sin(th), -np.cos(th)], RANGE)
    assert np.isclose(t, 0.01 / np.cos(th), atol=1e-16)
    b = oracle.Obj.box([0.02, 0.03, 0.04])
    t, _ = oracle.ray_first_root(b, [0.06, 0.01, 0.0], [-1, 0, 0], RANGE)
    assert np.isclose(t, 0.04)
    d = np.array([-1.0, -1.0, 0.0]) / np.sqrt(2)
    t, _ = oracle.ray_first_root(b, [0.05, 0.06, 0.0], d, RANGE)
    assert np.isclose(t, 0.03 * np.sqrt(2))   # enters through the y face at y = 0.03 (x = 0.02)


def test_mesh_root_equals_box_root():
    V, F = cube_mesh(0.02)
    h = float(np.float32(0.02))
    m, b = oracle.Obj.mesh(V, F), oracle.Obj.box([h, h, h])
    rng = np.random.default_rng(1)
    for _ in range(40):
        q = rng.uniform(-0.05, 0.05, 3)
        q[np.argmax(np.abs(q))] = np.sign(q[np.argmax(np.abs(q))]) * 0.05
        d = -q / np.linalg.norm(q) + rng.normal(0, 0.2, 3)
        d /= np.linalg.norm(d)
        tm, _ = oracle.ray_first_root(m, q, d, RANGE)
        tb, _ = oracle.ray_first_root(b, q, d, RANGE)
        assert (np.isnan(tm) and np.isnan(tb)) or np.isclose(tm, tb, atol=1e-14)


def _grid_of(fn, lo, hi, n):
    xs = [np.linspace(lo[i], hi[i], n) for i in range(3)]
    X, Y, Z = np.meshgrid(*xs, indexing="ij")
    vals = fn(X, Y, Z).transpose(2, 1, 0).astype(np.float32)
    return oracle.Obj.grid(vals, lo, hi), vals


def test_grid_root_of_linear_field():
    lo, hi = np.array([-0.04, -0.04, -0.04]), np.array([0.04, 0.04, 0.04])
    nrm = np.array([0.3, -0.4, 0.866])
    nrm /= np.linalg.norm(nrm)
    g, _ = _grid_of(lambda x, y, z: x * nrm[0] + y * nrm[1] + z * nrm[2] - 0.005, lo, hi, 17)
    rng = np.random.default_rng(2)
    for _ in range(30):
        q = rng.uniform(-0.03, 0.03, 3)
        q += nrm * (0.02 - q @ nrm)          # start 15 mm above the plane
        d = -nrm + rng.normal(0, 0.3, 3)
        d /= np.linalg.norm(d)
        t, _ = oracle.ray_first_root(g, q, d, 0.2)
        t_exact = (q @ nrm - 0.005) / -(d @ nrm)
        assert np.isclose(t, t_exact, atol=2e-8)   # float32 node values


def test_grid_root_matches_brute_force_sampling():
    lo, hi = np.array([-0.04, -0.04, -0.04]), np.array([0.04, 0.04, 0.04])
    g, _ = _grid_of(lambda x, y, z: np.sqrt(x * x + y * y + z * z) - 0.025, lo, hi, 33)
    rng = np.random.default_rng(3)
    ts = np.linspace(0, RANGE, 200001)
    for _ in range(25):
        u = rng.normal(size=3); u /= np.linalg.norm(u)
        q = u * 0.035
        d = -u + rng.normal(0, 0.4, 3); d /= np.linalg.norm(d)
        t, graze = oracle.ray_first_root(g, q, d, RANGE)
        phi, _ = g.sdf(q[None, :] + ts[:, None] * d[None, :])
        neg = np.flatnonzero(phi <= 0)
        if len(neg) == 0:
            assert np.isnan(t)
        else:
            assert not np.isnan(t) and abs(t - ts[neg[0]]) <= ts[1] + 1e-12


def test_ray_fan():
    n = np.array([0.6, 0.8, 0.0])
    dirs = oracle.prox_ray_dirs(n, 8, np.radians(30))
    assert np.allclose(np.linalg.norm(dirs, axis=1), 1.0)
    assert np.allclose(dirs[0], n)
    assert np.allclose(dirs[1:] @ n, np.cos(np.radians(30)))
    c = dirs[1:] - np.outer(dirs[1:] @ n, n)
    c /= np.linalg.norm(c, axis=1, keepdims=True)
    ang = np.arccos(np.clip(np.sum(c * np.roll(c, -1, axis=0), axis=1), -1, 1))
    assert np.allclose(ang, 2 * np.pi / 7)


def test_reading_of_a_probe_facing_a_plane():
    p = quiet_params(prox_rays=8)
    for H in (2e-3, 0.01, 0.03):
        wl = pad_workload(-(H - 1e-3), 2, 2, params=p)   # probe centres at height H above the plane
        sc = oracle_scene(wl)
        st = sc.new_state(); sc.reset(st, 0)
        out = sc.step(st, wl.inputs(0))
        c = np.cos(np.radians(30))
        hits = [(1 - H / RANGE)] + [(1 - H / c / RANGE) if H / c <= RANGE else 0.0] * 7
        assert np.allclose(out["prox_clean"], np.mean(hits), atol=1e-13)
        assert np.allclose(out["prox_noisy"], out["prox_clean"])


def test_proximity_hysteresis_step_response():
    p = quiet_params(prox_rays=8)
    p["noise"]["prox"] = W.noise_group(beta=0.1, tau=0.05)
    wl = pad_workload(-4e-3, 1, 1, params=p)
    sc = oracle_scene(wl)
    st = sc.new_state(); sc.reset(st, 0)
    a = np.exp(-p["dt"] / 0.05)
    x = sc.step(st, wl.inputs(0))["prox_clean"][0]
    for t in range(1, 5):
        out = sc.step(st, wl.inputs(0))
        assert np.isclose(out["prox_noisy"][0], x + 0.1 * a ** t * x, rtol=1e-12)


# ---------------------------------------------------------------- markers
LAM = 1.0 / (2 * 1.5e-3 ** 2)


def test_peak_normalisations():
    r = np.linspace(0, 0.01, 2_000_001)
    g = np.exp(-LAM * r * r)
    assert np.isclose((r * g).max(), np.exp(-0.5) / np.sqrt(2 * LAM), rtol=1e-9)
    eps = 1e-3
    assert np.isclose((r / (r * r + eps * eps)).max(), 1 / (2 * eps), rtol=1e-9)
    assert oracle.marker_kernel_g(LAM, 0.0) == 1.0
    assert np.isclose(oracle.marker_kernel_g(LAM, 1e-6), np.exp(-LAM * 1e-6))


def _pad_scene(obj, zw, rows=15, cols=15, pitch=1e-3, c=1.0, alpha=1.2):
    """One env, one identity link at height 0.01, one pad facing -z at world height zw."""
    wl = pad_workload(-1e-3, 1, 1, params=quiet_params())
    wl.objects = [obj]
    pads = dict(pads_per_env=1, rows=rows, cols=cols, pitch=pitch, pad_link=np.zeros((1, 1), np.int32),
                pad_frame=np.array([[[0, 0, zw - 0.01, 0, 0, -1, 1, 0, 0]]], np.float32),
                s_d=1.0, alpha=alpha, lambda_d=LAM, c=c, eps=pitch, radius=2)
    return wl, pads


@pytest.mark.parametrize("c", [1.0, 0.0, 0.4])
def test_single_source_closed_form(c):
    r_s, delta = 2e-3, 1e-4
    wl, pads = _pad_scene(W.ObjectSpec(kind="sphere", radius=r_s), r_s - delta, c=c)
    sc = oracle_scene(wl)
    u, h = sc.markers(pads, wl.inputs(0))
    u, h = u[0, 0].reshape(15, 15, 3), h[0, 0].reshape(15, 15)
    hc = h[7, 7]  # the centre marker alone penetrates, by delta (float32 inputs)
    assert abs(hc - delta) < 1e-8 and (h > 0).sum() == 1
    gbar = np.exp(-0.5) / np.sqrt(2 * LAM)
    rbar = 1 / (2 * 1e-3)
    for a in range(15):
        for b in range(15):
            da, db = a - 7, b - 7
            if max(abs(da), abs(db)) > 2:
                assert np.allclose(u[a, b], 0.0)
                continue
            # tangential offset r = x_j - x_i in pad axes (tu = +x, tv = n x tu = -y)
            rt = np.array([da * 1e-3, db * 1e-3])
            r2 = rt @ rt
            g = np.exp(-LAM * r2)
            w = hc * (c * g / gbar + (1 - c) * (1 / (r2 + 1e-6)) / rbar)
            assert np.isclose(u[a, b, 0], hc ** 1.2 * g, rtol=1e-9, atol=1e-18)
            assert np.allclose(u[a, b, 1:], rt * w, rtol=1e-9, atol=1e-18)


def test_uniform_depth_field():
    zw = -3e-4  # the whole pad 0.3 mm into the half-space z <= 0
    wl, pads = _pad_scene(W.ObjectSpec(kind="plane"), zw)
    sc = oracle_scene(wl)
    u, h = sc.markers(pads, wl.inputs(0))
    u, h = u[0, 0].reshape(15, 15, 3), h[0, 0].reshape(15, 15)
    hz = -(float(np.float32(zw - 0.01)) + 0.01)
    assert np.allclose(h, hz, atol=1e-15)
    k = sum(np.exp(-LAM * ((i * 1e-3) ** 2 + (j * 1e-3) ** 2)) for i in range(-2, 3) for j in range(-2, 3))
    inner = u[2:-2, 2:-2]
    assert np.allclose(inner[..., 1:], 0.0, atol=1e-15)
    assert np.allclose(inner[..., 0], hz ** 1.2 * k, rtol=1e-12)
    assert np.abs(u[0, 7, 1:]).max() > 1e-6   # edge markers are pulled tangentially


def test_no_contact_no_displacement():
    wl, pads = _pad_scene(W.ObjectSpec(kind="plane"), 2e-3)
    u, h = oracle_scene(wl).markers(pads, wl.inputs(0))
    assert np.all(h == 0) and np.all(u == 0)


def test_a_ray_that_skims_the_surface_is_grazing():
    """A ray that enters a sphere but leaves it again before it is 20 um deep
    is flagged like a near miss; one whose chord goes deeper is not.  The
    sphere is small (r = 1 mm) so that both rays cross at slopes above the
    shallow-angle limit (0.05), and only the depth decides."""
    r = 1e-3
    sph = oracle.Obj.sphere(r)
    for depth, want in ((10e-6, True), (50e-6, False)):
        b = r - depth                                  # distance of the ray from the centre
        q0 = np.array([-5e-3, b, 0.0])
        t, grazing = oracle.ray_first_root(sph, q0, np.array([1.0, 0.0, 0.0]), 0.05)
        assert np.isclose(t, 5e-3 - np.sqrt(r * r - b * b))
        slope = np.sqrt(1.0 - (b / r) ** 2)
        assert slope > 0.05
        assert grazing == want
