"""Seeded synthetic workloads for the tactile contact query.

This module creates INPUT DATA only: capsule links carrying taxel lattices,
procedural objects (spheres, convex hulls, superquadrics), poses and
velocities, and the parameter sets.  It contains no step of the sensing
method (no depth, force or noise arithmetic, no SDF grid or mesh query);
the links are placed with a coarse surface estimate of its own
(nearest face planes, see _PlacementSurface), which neither side reads.
Both the CUDA path and the CPU oracle consume what it returns.

The paper's own workloads (robot hands, task objects, a 10-cube scene) are
not available, so these seeded procedural stand-ins follow the sizes the
paper quotes (tens to thousands of taxels per hand, >16k environments).

Geometry conventions: SI units, quaternions (w, x, y, z).  A link is a
capsule centred at its frame origin with its axis along link +z; its taxels
sit on the cylinder as a rows x cols lattice (rows along the axis, cols around
the circumference, row-major), which is the regular lattice the spatial
crosstalk uses.  Taxel radius R = 1 mm; R = 0 marks an inactive filler.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

DT = 1.0 / 200.0          # simulation step (200 Hz)
TAXEL_RADIUS = 1e-3       # probe radius of an active taxel
PAD_ARC = np.pi / 3       # lattice arc of the batched configs: a 60-degree pad strip facing the object


def f32(x):
    """Round to the nearest float32 (the precision both sides read)."""
    return np.asarray(x, dtype=np.float32)


# ---------------------------------------------------------------------------
# parameters
# ---------------------------------------------------------------------------
def noise_group(**kw):
    g = dict(gain_lo=1.0, gain_hi=1.0, beta=0.0, tau=0.05, bias=0.0, sigma_white=0.0,
             sigma_rw=0.0, quant=0.0, stuck_lo=0.0, stuck_hi=0.0)
    g.update(kw)
    return g


def default_params(seed: int) -> dict:
    """Contact and noise parameters of the synthetic workloads: k = 1e4 N/m,
    damping 5, mu = 0.8, dead rate 2 %, drift 1e-3 per step on force/torque,
    hysteresis 0.1 (tau 0.05 s), 3x3 crosstalk 0.05."""
    return dict(
        k=1e4, c=5.0, alpha=1.0, k_t=2.0, k_omega=2.0, mu=0.8,
        eta_on=5e-4, eta_off=2e-4, dt=DT, seed=int(seed), p_dead=0.02,
        chi=0.05, xt_sigma=1.0,
        prox_rays=0, prox_range=0.05, prox_cone=float(np.radians(30.0)),
        noise=dict(
            depth=noise_group(beta=0.1, tau=0.05),
            ft=noise_group(beta=0.1, tau=0.05, sigma_rw=1e-3),
            prox=noise_group(beta=0.1, tau=0.05),
        ),
    )


# ---------------------------------------------------------------------------
# rotations (random orientation generation only)
# ---------------------------------------------------------------------------
def random_rotation(rng) -> np.ndarray:
    """Haar-uniform rotation matrix from the QR factorisation of a Gaussian matrix."""
    A = rng.standard_normal((3, 3))
    Q, Rr = np.linalg.qr(A)
    Q = Q * np.sign(np.diag(Rr))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    return Q


def mat_to_quat(M: np.ndarray) -> np.ndarray:
    """Unit quaternion (w, x, y, z) of a rotation matrix (Shepperd's branch choice)."""
    t = np.trace(M)
    if t > 0:
        s = np.sqrt(t + 1.0) * 2
        q = [0.25 * s, (M[2, 1] - M[1, 2]) / s, (M[0, 2] - M[2, 0]) / s, (M[1, 0] - M[0, 1]) / s]
    elif M[0, 0] > M[1, 1] and M[0, 0] > M[2, 2]:
        s = np.sqrt(1.0 + M[0, 0] - M[1, 1] - M[2, 2]) * 2
        q = [(M[2, 1] - M[1, 2]) / s, 0.25 * s, (M[0, 1] + M[1, 0]) / s, (M[0, 2] + M[2, 0]) / s]
    elif M[1, 1] > M[2, 2]:
        s = np.sqrt(1.0 + M[1, 1] - M[0, 0] - M[2, 2]) * 2
        q = [(M[0, 2] - M[2, 0]) / s, (M[0, 1] + M[1, 0]) / s, 0.25 * s, (M[1, 2] + M[2, 1]) / s]
    else:
        s = np.sqrt(1.0 + M[2, 2] - M[0, 0] - M[1, 1]) * 2
        q = [(M[1, 0] - M[0, 1]) / s, (M[0, 2] + M[2, 0]) / s, (M[1, 2] + M[2, 1]) / s, 0.25 * s]
    q = np.asarray(q)
    return q / np.linalg.norm(q)


def unit(v):
    return v / np.linalg.norm(v)


# ---------------------------------------------------------------------------
# procedural meshes
# ---------------------------------------------------------------------------
def orient_outward(verts: np.ndarray, faces: np.ndarray) -> np.ndarray:
    """Flip every face whose winding disagrees with a positive enclosed volume
    (for convex hull faces: whose normal points towards the interior point)."""
    c = verts.mean(axis=0)
    a, b, cc = verts[faces[:, 0]], verts[faces[:, 1]], verts[faces[:, 2]]
    n = np.cross(b - a, cc - a)
    flip = np.einsum("ij,ij->i", n, a - c) < 0
    faces = faces.copy()
    faces[flip] = faces[flip][:, [0, 2, 1]]
    return faces


def subdivide(verts: np.ndarray, faces: np.ndarray):
    """Planar 1->4 midpoint subdivision (leaves the surface unchanged)."""
    verts = [tuple(v) for v in verts]
    index = {}

    def mid(i, j):
        key = (min(i, j), max(i, j))
        if key not in index:
            index[key] = len(verts)
            verts.append(tuple((np.asarray(verts[i]) + np.asarray(verts[j])) / 2.0))
        return index[key]

    out = []
    for a, b, c in faces:
        ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
        out += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)]
    return np.asarray(verts), np.asarray(out, dtype=np.int64)


def hull_mesh(rng, n_points: int, extent: float = 0.04, min_faces: int = 0):
    """Convex hull of Gaussian points, scaled to `extent` along its longest
    axis, centred on its vertex mean, subdivided until it has >= min_faces."""
    from scipy.spatial import ConvexHull

    P = rng.standard_normal((n_points, 3))
    hull = ConvexHull(P)
    used = np.unique(hull.simplices)
    remap = -np.ones(n_points, np.int64)
    remap[used] = np.arange(len(used))
    V = P[used]
    F = remap[hull.simplices]
    V = V - V.mean(axis=0)
    V = V * (extent / (V.max(axis=0) - V.min(axis=0)).max())
    F = orient_outward(V, F)
    while len(F) < min_faces:
        V, F = subdivide(V, F)
    return f32(V), F.astype(np.int32)


def superquadric_mesh(rng, eps1: float, eps2: float, axes, n_eta: int, n_omega: int = 64):
    """UV tessellation of a superellipsoid with exponents eps1 (latitude) and
    eps2 (longitude) and semi-axes `axes`; 2 n_omega (n_eta - 1) faces."""
    def spow(w, e):
        return np.sign(w) * np.abs(w) ** e

    a1, a2, a3 = axes
    verts = [(0.0, 0.0, -a3)]
    for i in range(1, n_eta):
        eta = -np.pi / 2 + i * np.pi / n_eta
        for j in range(n_omega):
            om = -np.pi + 2 * np.pi * j / n_omega
            ce, se = spow(np.cos(eta), eps1), spow(np.sin(eta), eps1)
            verts.append((a1 * ce * spow(np.cos(om), eps2), a2 * ce * spow(np.sin(om), eps2), a3 * se))
    verts.append((0.0, 0.0, a3))
    V = np.asarray(verts)
    north = len(V) - 1

    def vid(i, j):  # ring i in 1..n_eta-1
        return 1 + (i - 1) * n_omega + (j % n_omega)

    F = []
    for j in range(n_omega):
        F.append((0, vid(1, j + 1), vid(1, j)))
    for i in range(1, n_eta - 1):
        for j in range(n_omega):
            F.append((vid(i, j), vid(i, j + 1), vid(i + 1, j + 1)))
            F.append((vid(i, j), vid(i + 1, j + 1), vid(i + 1, j)))
    for j in range(n_omega):
        F.append((north, vid(n_eta - 1, j), vid(n_eta - 1, j + 1)))
    F = np.asarray(F, dtype=np.int64)
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    vol = np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0
    if vol < 0:
        F = F[:, [0, 2, 1]]
    return f32(V), F.astype(np.int32)


# ---------------------------------------------------------------------------
# objects
# ---------------------------------------------------------------------------
@dataclass
class ObjectSpec:
    kind: str                     # 'sphere' | 'box' | 'plane' | 'mesh' | 'grid' | 'neural'
    radius: float = 0.0
    half: tuple = (0.0, 0.0, 0.0)
    verts: np.ndarray | None = None
    faces: np.ndarray | None = None
    dims: tuple | None = None     # grid nodes per axis (x, y, z)
    lo: np.ndarray | None = None  # float32 box corners
    hi: np.ndarray | None = None
    fp16: bool = False
    values: np.ndarray | None = None  # [z][y][x] float32 or binary16 bits (uint16), set by a bake
    name: str = ""
    # learned SDF ('neural'; the grid fields above hold its fallback grid, verts/faces the exact mesh)
    net: object = None                # a trained network handle, or None to build one from the arrays below
    nsdf_lo: np.ndarray | None = None
    nsdf_hi: np.ndarray | None = None
    nsdf_table: np.ndarray | None = None    # uint16 [16][65536][2] binary16 bits
    nsdf_weights: np.ndarray | None = None  # uint16 [6208] bfloat16 bits: W1 [64][32], W2 [64][64], W3 [64]
    nsdf_err_mm: float = -1.0
    # tracked surface points (object frame, [n][3]) for the point-cloud ProximityTaxel
    cloud: np.ndarray | None = None


def bf16_bits(x) -> np.ndarray:
    """float32 values rounded to the nearest bfloat16 (ties to even), as uint16 bits."""
    b = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    return ((b + 0x7FFF + ((b >> 16) & 1)) >> 16).astype(np.uint16)


def random_nsdf_params(rng, table_scale: float = 1.0, out_scale: float = 20.0):
    """Seeded learned-SDF parameters for parity tests: table entries uniform in
    +-table_scale (binary16), weights uniform in +-sqrt(6 / (fan_in + fan_out))
    (bfloat16; W3 scaled by out_scale so outputs span millimetres)."""
    table = rng.uniform(-table_scale, table_scale, (16, 65536, 2)).astype(np.float16).view(np.uint16)
    w1 = rng.uniform(-1, 1, (64, 32)) * np.sqrt(6 / 96)
    w2 = rng.uniform(-1, 1, (64, 64)) * np.sqrt(6 / 128)
    w3 = rng.uniform(-1, 1, 64) * np.sqrt(6 / 65) * out_scale
    weights = bf16_bits(np.concatenate([w1.reshape(-1), w2.reshape(-1), w3]))
    return table, weights


def surface_samples(rng, verts: np.ndarray, faces: np.ndarray, n: int):
    """n points uniform over the mesh surface (area-weighted) and their face normals."""
    V = verts.astype(np.float64)
    a, b, c = V[faces[:, 0]], V[faces[:, 1]], V[faces[:, 2]]
    cr = np.cross(b - a, c - a)
    area = 0.5 * np.linalg.norm(cr, axis=1)
    f = rng.choice(len(faces), n, p=area / area.sum())
    r1, r2 = np.sqrt(rng.uniform(size=n)), rng.uniform(size=n)
    p = (1 - r1)[:, None] * a[f] + (r1 * (1 - r2))[:, None] * b[f] + (r1 * r2)[:, None] * c[f]
    nrm = cr[f] / np.linalg.norm(cr[f], axis=1, keepdims=True)
    return p, nrm


def object_cloud(rng, o: "ObjectSpec", n: int):
    """n tracked surface points of an object (float32 [n][3], object frame;
    Appendix A "ProximityTaxel" samples tracked links into a surface point
    cloud at reset): area-weighted on a mesh, uniform on a sphere or a box;
    None for a plane (unbounded)."""
    if o.verts is not None and o.faces is not None:
        return surface_samples(rng, o.verts, o.faces, n)[0].astype(np.float32)
    if o.kind == "sphere":
        v = rng.standard_normal((n, 3))
        return (o.radius * v / np.linalg.norm(v, axis=1, keepdims=True)).astype(np.float32)
    if o.kind == "box":
        h = np.asarray(o.half, np.float64)
        areas = np.array([h[1] * h[2], h[0] * h[2], h[0] * h[1]] * 2)
        f = rng.choice(6, n, p=areas / areas.sum())
        p = rng.uniform(-1, 1, (n, 3)) * h
        ax = f % 3
        p[np.arange(n), ax] = np.where(f < 3, 1.0, -1.0) * h[ax]
        return p.astype(np.float32)
    return None


def add_clouds(wl: "Workload", n: int = 5000, seed: int = 20260099) -> "Workload":
    """Give every object of the workload n tracked surface points."""
    rng = np.random.default_rng(seed)
    for o in wl.objects:
        o.cloud = object_cloud(rng, o, n)
    return wl


def sdf_sample_points(rng, verts: np.ndarray, faces: np.ndarray, lo, hi, n: int, band: float = 5e-3) -> np.ndarray:
    """Learned-SDF training / probe points (float32 [n][3], object frame): half
    within `band` of the surface (a surface point moved along its normal by
    U(-band, band)), half uniform in the box [lo, hi]."""
    n_near = n // 2
    p, nrm = surface_samples(rng, verts, faces, n_near)
    near = p + nrm * rng.uniform(-band, band, (n_near, 1))
    lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
    near = np.clip(near, lo, hi)
    uni = lo + (hi - lo) * rng.uniform(size=(n - n_near, 3))
    pts = np.concatenate([near, uni])
    return f32(pts[rng.permutation(n)])


def grid_box(verts: np.ndarray):
    """Per-axis box = bounding-box centre +- 0.6 x extent (a 1.2x padded box)."""
    lo, hi = verts.min(axis=0).astype(np.float64), verts.max(axis=0).astype(np.float64)
    c, ext = (lo + hi) / 2, hi - lo
    return f32(c - 0.6 * ext), f32(c + 0.6 * ext)


def make_grid_object(verts, faces, n: int, fp16: bool, name="") -> ObjectSpec:
    lo, hi = grid_box(verts)
    return ObjectSpec(kind="grid", verts=verts, faces=faces, dims=(n, n, n), lo=lo, hi=hi, fp16=fp16, name=name)


def support(obj: ObjectSpec, R: np.ndarray, u: np.ndarray) -> float:
    """Extent of the object along world direction u (the support function),
    used only to place links near the surface."""
    if obj.kind == "sphere":
        return float(obj.radius)
    if obj.kind == "box":
        return float(np.abs(R.T @ u) @ np.asarray(obj.half))
    return float((obj.verts.astype(np.float64) @ (R.T @ u)).max())


# ---------------------------------------------------------------------------
# scenes
# ---------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    n_envs: int
    max_links: int
    taxel_offsets: np.ndarray       # int64 [E+1]
    taxel_gid0: np.ndarray          # int64 [E] global id of each env's first taxel
    env_gid: np.ndarray             # int32 [E]
    link_rows: np.ndarray           # int32 [E*L]
    link_cols: np.ndarray           # int32 [E*L]
    link_wrap: np.ndarray           # uint8 [E*L]
    x: np.ndarray; y: np.ndarray; z: np.ndarray      # float32 [T]
    nx: np.ndarray; ny: np.ndarray; nz: np.ndarray   # float32 [T]
    R: np.ndarray                   # float32 [T]
    objects: list
    obj_id: np.ndarray              # int32 [E]
    link_pose: np.ndarray           # float32 [E, L, 7]
    link_vel: np.ndarray            # float32 [E, L, 6]
    obj_pose: np.ndarray            # float32 [E, 7]
    obj_vel: np.ndarray             # float32 [E, 6]
    params: dict
    steps: int = 1
    env_params: np.ndarray | None = None
    pads: dict | None = None          # elastomer marker pads (see add_pads)
    meta: dict = field(default_factory=dict)

    @property
    def n_taxels(self) -> int:
        return int(self.taxel_offsets[-1])

    @property
    def n_active(self) -> int:
        return int((self.R > 0).sum())

    def geom(self) -> dict:
        return {k: getattr(self, k) for k in ("taxel_offsets", "taxel_gid0", "env_gid", "link_rows", "link_cols",
                                              "link_wrap", "x", "y", "z", "nx", "ny", "nz", "R")}

    def inputs(self, step: int) -> dict:
        """Per-step inputs: time-0 poses advanced by step * dt, RNG step counter."""
        return dict(link_pose=self.link_pose, link_vel=self.link_vel, obj_pose=self.obj_pose,
                    obj_vel=self.obj_vel, obj_id=self.obj_id, env_params=self.env_params,
                    pose_dt=float(step) * self.params["dt"], step=int(step))

    def subset(self, envs) -> "Workload":
        """The same envs as a smaller scene that keeps global taxel and env ids."""
        envs = np.asarray(envs, dtype=np.int64)
        L = self.max_links
        off = self.taxel_offsets
        counts = off[envs + 1] - off[envs]
        new_off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
        idx = np.concatenate([np.arange(off[e], off[e + 1]) for e in envs]) if len(envs) else np.zeros(0, np.int64)
        lidx = (envs[:, None] * L + np.arange(L)[None, :]).reshape(-1)
        sub = Workload(
            name=self.name + "[subset]", n_envs=len(envs), max_links=L, taxel_offsets=new_off,
            taxel_gid0=self.taxel_gid0[envs].copy(), env_gid=self.env_gid[envs].copy(),
            link_rows=self.link_rows[lidx].copy(), link_cols=self.link_cols[lidx].copy(),
            link_wrap=self.link_wrap[lidx].copy(),
            x=self.x[idx], y=self.y[idx], z=self.z[idx], nx=self.nx[idx], ny=self.ny[idx], nz=self.nz[idx],
            R=self.R[idx], objects=self.objects, obj_id=self.obj_id[envs].copy(),
            link_pose=self.link_pose[envs].copy(), link_vel=self.link_vel[envs].copy(),
            obj_pose=self.obj_pose[envs].copy(), obj_vel=self.obj_vel[envs].copy(), params=self.params,
            steps=self.steps, env_params=None if self.env_params is None else self.env_params[envs].copy(),
            meta=dict(self.meta),
        )
        if self.pads is not None:
            sub.pads = dict(self.pads, pad_link=self.pads["pad_link"][envs].copy(),
                            pad_frame=self.pads["pad_frame"][envs].copy())
        return sub


def capsule_lattice(rows: int, cols: int, radius: float, length: float, n_active: int, arc: float = 2 * np.pi):
    """Taxels on the cylinder of a capsule (axis link +z), rows along the
    axis and cols around an arc centred on link +x (the full circumference
    when arc = 2 pi); the slots past n_active are R = 0 fillers."""
    r = np.arange(rows)[:, None] * np.ones((1, cols))
    c = np.ones((rows, 1)) * np.arange(cols)[None, :]
    if arc >= 2 * np.pi:
        th = 2 * np.pi * c / cols
    else:
        th = -arc / 2 + arc * (c + 0.5) / cols
    zz = -length / 2 + (r + 0.5) * length / rows
    x = radius * np.cos(th); y = radius * np.sin(th)
    nx = np.cos(th); ny = np.sin(th); nz = np.zeros_like(th)
    Rr = np.full(rows * cols, TAXEL_RADIUS)
    Rr[n_active:] = 0.0
    return [a.reshape(-1) for a in (x, y, zz, nx, ny, nz)] + [Rr]


def random_rotations(rng, n: int) -> np.ndarray:
    """n Haar-uniform rotation matrices (batched QR of Gaussian matrices)."""
    A = rng.standard_normal((n, 3, 3))
    Q, Rr = np.linalg.qr(A)
    Q = Q * np.sign(np.diagonal(Rr, axis1=1, axis2=2))[:, None, :]
    neg = np.linalg.det(Q) < 0
    Q[neg, :, 0] = -Q[neg, :, 0]
    return Q


def mats_to_quats(M: np.ndarray) -> np.ndarray:
    """Batched mat_to_quat."""
    out = np.empty(M.shape[:-2] + (4,))
    flat = M.reshape(-1, 3, 3)
    o = out.reshape(-1, 4)
    t = np.trace(flat, axis1=1, axis2=2)
    c0 = t > 0
    c1 = ~c0 & (flat[:, 0, 0] > flat[:, 1, 1]) & (flat[:, 0, 0] > flat[:, 2, 2])
    c2 = ~c0 & ~c1 & (flat[:, 1, 1] > flat[:, 2, 2])
    c3 = ~c0 & ~c1 & ~c2
    m = flat
    with np.errstate(invalid="ignore", divide="ignore"):
        s = np.sqrt(np.maximum(t + 1.0, 0)) * 2
        q0 = np.stack([0.25 * s, (m[:, 2, 1] - m[:, 1, 2]) / s, (m[:, 0, 2] - m[:, 2, 0]) / s, (m[:, 1, 0] - m[:, 0, 1]) / s], 1)
        s = np.sqrt(np.maximum(1.0 + m[:, 0, 0] - m[:, 1, 1] - m[:, 2, 2], 0)) * 2
        q1 = np.stack([(m[:, 2, 1] - m[:, 1, 2]) / s, 0.25 * s, (m[:, 0, 1] + m[:, 1, 0]) / s, (m[:, 0, 2] + m[:, 2, 0]) / s], 1)
        s = np.sqrt(np.maximum(1.0 + m[:, 1, 1] - m[:, 0, 0] - m[:, 2, 2], 0)) * 2
        q2 = np.stack([(m[:, 0, 2] - m[:, 2, 0]) / s, (m[:, 0, 1] + m[:, 1, 0]) / s, 0.25 * s, (m[:, 1, 2] + m[:, 2, 1]) / s], 1)
        s = np.sqrt(np.maximum(1.0 + m[:, 2, 2] - m[:, 0, 0] - m[:, 1, 1], 0)) * 2
        q3 = np.stack([(m[:, 1, 0] - m[:, 0, 1]) / s, (m[:, 0, 2] + m[:, 2, 0]) / s, (m[:, 1, 2] + m[:, 2, 1]) / s, 0.25 * s], 1)
    o[c0], o[c1], o[c2], o[c3] = q0[c0], q1[c1], q2[c2], q3[c3]
    o /= np.linalg.norm(o, axis=1, keepdims=True)
    return out


def _unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


class _PlacementSurface:
    """Approximate signed distance of an object's surface, used only to place
    links so that a chosen share of taxels penetrates (input construction,
    not the sensing method): closed forms for the analytic kinds, and for
    meshes (convex hulls and superquadrics with exponents <= 2, both convex)
    the largest signed distance to the planes of the 16 faces whose centroids
    are nearest.  Inside a convex polytope, and outside it over a face, the
    largest plane distance over all faces is the exact signed distance; the
    16 nearest faces reproduce it to ~1e-5 mm within 3 mm of the workloads'
    surfaces.  Returns (phi, unit normal of the deciding plane)."""

    def __init__(self, obj):
        self.obj = obj
        self.tree = None
        if obj.verts is not None and obj.faces is not None and obj.kind not in ("sphere", "box", "plane"):
            from scipy.spatial import cKDTree

            V = obj.verts.astype(np.float64)
            F = np.asarray(obj.faces, np.int64)
            cen = V[F].mean(axis=1)
            nrm = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
            nrm /= np.maximum(np.linalg.norm(nrm, axis=1, keepdims=True), 1e-300)
            self.nrm, self.off = nrm, np.einsum("ij,ij->i", nrm, cen)
            self.k = min(8, len(F))
            self.tree = cKDTree(cen)

    def __call__(self, q):
        o = self.obj
        if len(q) == 0:
            return np.zeros(0), np.zeros((0, 3))
        if o.kind == "sphere":
            r = np.linalg.norm(q, axis=1)
            return r - float(o.radius), q / np.maximum(r, 1e-300)[:, None]
        if o.kind == "plane":
            return q[:, 2].copy(), np.tile([0.0, 0.0, 1.0], (len(q), 1))
        if o.kind == "box":
            d = np.abs(q) - np.asarray(o.half, np.float64)
            out = np.maximum(d, 0.0)
            on = np.linalg.norm(out, axis=1)
            ax = np.argmax(d, axis=1)
            n_in = np.zeros_like(q)
            n_in[np.arange(len(q)), ax] = np.sign(q[np.arange(len(q)), ax])
            n_out = np.sign(q) * out / np.maximum(on, 1e-300)[:, None]
            inside = on == 0.0
            return np.where(inside, d.max(axis=1), on), np.where(inside[:, None], n_in, n_out)
        _, idx = self.tree.query(q, k=self.k, workers=-1)
        idx = idx.reshape(len(q), -1)
        phi = np.empty(len(q))
        face = np.empty(len(q), np.int64)

        def chunk(a):  # numpy releases the GIL inside these array operations
            sl = slice(a, min(a + (1 << 16), len(q)))
            i, x = idx[sl], q[sl]
            nn = self.nrm[i]
            d = nn[..., 0] * x[:, 0:1] + nn[..., 1] * x[:, 1:2] + nn[..., 2] * x[:, 2:3] - self.off[i]
            b = d.argmax(axis=1)
            r = np.arange(len(b))
            phi[sl], face[sl] = d[r, b], i[r, b]

        from concurrent.futures import ThreadPoolExecutor

        with ThreadPoolExecutor(8) as ex:
            list(ex.map(chunk, range(0, len(q), 1 << 16)))
        return phi, self.nrm[face]


def _assemble(name, rng, objects, env_obj, env_lattices, params, steps, pen_share=(0.1, 0.3), max_press=2e-3,
              max_links=None, arc=2 * np.pi):
    """Place every env's links around its object and build the arrays.

    env_lattices[e] is a list of (rows, cols, n_active) per link.  Each link is
    a capsule (radius 8-12 mm, cylinder 20-45 mm) whose lattice arc faces the
    object along a random direction u, its axis perpendicular to u.  Every env
    draws a target share f ~ U(pen_share) of its active taxels that penetrate
    (probe sphere reaching into the object) at the time-0 poses, and all its
    links are pressed from touching the object's support plane towards the
    object by one depth delta_e, solved per env so that the share is met:
    per taxel the press depth at which it starts to penetrate is linearised
    from the placement surface (its distance over the slope n . u), delta_e is
    set between the k-th and (k+1)-th smallest of them (k = round(f n)), and
    the envs whose share, re-evaluated at delta_e, misses the target by more
    than 1 % get up to three more such corrections from there.  The realised
    shares and depths are kept in meta["placement"].  Vectorised over envs
    and links."""
    E = len(env_lattices)
    L = max_links or max(len(lat) for lat in env_lattices)
    rows = np.zeros((E, L), np.int32); cols = np.zeros((E, L), np.int32); nact = np.zeros((E, L), np.int64)
    uniform = all(lat == env_lattices[0] for lat in env_lattices[1:]) if E > 1 else True
    if uniform and env_lattices[0]:
        lat = np.asarray(env_lattices[0], np.int64)
        rows[:, :len(lat)], cols[:, :len(lat)], nact[:, :len(lat)] = lat[:, 0], lat[:, 1], lat[:, 2]
    else:
        for e, lat in enumerate(env_lattices):
            for l, (r, c, na) in enumerate(lat):
                rows[e, l], cols[e, l], nact[e, l] = r, c, na
    env_obj = np.asarray(env_obj, np.int64)
    # object poses
    RC = random_rotations(rng, E)
    pC = rng.normal(0.0, 0.005, (E, 3))
    obj_pose = np.zeros((E, 7), np.float32)
    obj_pose[:, :3] = pC
    obj_pose[:, 3:] = mats_to_quats(RC)
    obj_vel = np.concatenate([rng.normal(0.0, 0.1, (E, 3)), rng.normal(0.0, 1.0, (E, 3))], 1).astype(np.float32)
    # links
    f_target = rng.uniform(*pen_share, E)
    rc = rng.uniform(8e-3, 12e-3, (E, L))
    ln = rng.uniform(20e-3, 45e-3, (E, L))
    u = _unit(rng.standard_normal((E, L, 3)))
    d_obj = np.einsum("eji,elj->eli", RC, u)          # directions in each object's frame
    h = np.einsum("ei,eli->el", pC, u)
    for k, obj in enumerate(objects):
        sel = env_obj == k
        if not sel.any():
            continue
        dk = d_obj[sel]
        if obj.kind == "sphere":
            h[sel] += float(obj.radius)
        elif obj.kind == "box":
            h[sel] += np.abs(dk) @ np.asarray(obj.half, np.float64)
        elif obj.kind == "plane":
            h[sel] += 0.0
        else:
            Vd = obj.verts.astype(np.float64)
            h[sel] += (dk.reshape(-1, 3) @ Vd.T).max(axis=1).reshape(dk.shape[:2])
    axis = _unit(np.cross(u, rng.standard_normal((E, L, 3))))
    e1 = -u                                            # lattice column 0 faces the object
    e2 = np.cross(axis, e1)
    RL = np.stack([e1, e2, axis], axis=-1)
    link_vel = np.concatenate([rng.normal(0.0, 0.1, (E, L, 3)), rng.normal(0.0, 1.0, (E, L, 3))], -1).astype(np.float32)
    absent = rows * cols == 0
    # taxels of every link lattice, in CSR order
    n_link = (rows.astype(np.int64) * cols).reshape(-1)
    starts = np.concatenate([[0], np.cumsum(n_link)])
    T = int(starts[-1])
    link_of = np.repeat(np.arange(E * L), n_link)
    j = np.arange(T) - starts[link_of]
    cl = cols.reshape(-1)[link_of].astype(np.int64)
    rl = rows.reshape(-1)[link_of].astype(np.int64)
    rr, cc = j // cl, j % cl
    if arc >= 2 * np.pi:
        th = 2 * np.pi * cc / cl
    else:
        th = -arc / 2 + arc * (cc + 0.5) / cl
    radius = rc.reshape(-1)[link_of]
    length = ln.reshape(-1)[link_of]
    x = radius * np.cos(th); y = radius * np.sin(th)
    z = -length / 2 + (rr + 0.5) * length / rl
    Rt = np.where(j < nact.reshape(-1)[link_of], TAXEL_RADIUS, 0.0)
    off = np.concatenate([[0], np.cumsum(n_link.reshape(E, L).sum(1))]).astype(np.int64)

    # ---- press depth per env (time-0 poses, float32 inputs as both sides read them)
    env_of = link_of // L
    touch = (h + rc)[..., None] * u                    # link centres touching the support plane
    # a taxel can penetrate at press delta only if it reaches the support plane:
    # radius (1 - cos th) - R < delta; farther ones never do for delta <= max_press
    cand = np.flatnonzero((Rt > 0) & (radius * (1.0 - np.cos(th)) - Rt < max_press))
    ce, cl_ = env_of[cand], link_of[cand]
    xl = np.stack([x[cand], y[cand], z[cand]], 1)
    xw = np.einsum("nij,nj->ni", RL.reshape(E * L, 3, 3)[cl_], xl) + touch.reshape(E * L, 3)[cl_]
    q0 = np.einsum("nji,nj->ni", RC[ce], xw - pC[ce])    # object frame, touching (press 0)
    del xw, xl
    dirs = d_obj.reshape(E * L, 3)[cl_]                  # a press delta moves a taxel by -delta dirs
    surfaces = [_PlacementSurface(o) for o in objects]
    oid_c = env_obj[ce]

    def phi_at(delta_env, which):
        """placement-surface phi and normal of candidates `which` with env presses delta_env"""
        i = which
        q = q0[i] - delta_env[ce[i], None] * dirs[i]
        phi = np.empty(len(i)); nrm = np.empty((len(i), 3))
        for k, srf in enumerate(surfaces):
            s = np.flatnonzero(oid_c[i] == k)
            if len(s):
                phi[s], nrm[s] = srf(q[s])
        return phi, nrm

    n_act = np.bincount(env_of[Rt > 0], minlength=E).astype(np.int64)
    k_target = np.rint(f_target * n_act).astype(np.int64)
    n_cand = np.bincount(ce, minlength=E)
    cstart = np.concatenate([[0], np.cumsum(n_cand)])
    width = int(n_cand.max()) if E else 0

    def solve(thr, base):
        """per env: the press between the k-th and (k+1)-th smallest threshold"""
        M = np.full((E, max(width, 1) + 1), np.inf)
        M[ce, np.arange(len(ce)) - cstart[ce]] = thr
        M.sort(axis=1)
        k = np.minimum(k_target, width)
        lo = np.where(k > 0, M[np.arange(E), np.maximum(k - 1, 0)], -np.inf)
        hi = M[np.arange(E), k]
        d = np.where(np.isfinite(lo) & np.isfinite(hi), 0.5 * (lo + hi),
                     np.where(np.isfinite(lo), lo + 1e-5, np.where(np.isfinite(hi), hi - 1e-5, base)))
        return np.clip(d, 0.0, max_press)

    delta = np.zeros(E)
    phi, nrm = phi_at(delta, np.arange(len(cand)))
    slope = np.maximum(np.einsum("ij,ij->i", nrm, dirs), 0.05)
    thr = (phi - Rt[cand]) / slope                     # press at which each candidate starts to penetrate
    delta = solve(thr, delta)
    # taxels whose linearised threshold lies within 0.5 mm of their env's
    # press are re-evaluated at it (every env first, then the envs still off
    # target); the rest keep the linear model's verdict
    redo = np.ones(E, bool)
    for _ in range(4):
        near = np.flatnonzero(redo[ce] & (np.abs(thr - delta[ce]) < 5e-4))
        phi_n, nrm_n = phi_at(delta, near)
        slope[near] = np.maximum(np.einsum("ij,ij->i", nrm_n, dirs[near]), 0.05)
        thr[near] = delta[ce[near]] + (phi_n - Rt[cand][near]) / slope[near]
        pen = thr < delta[ce]
        got = np.bincount(ce, weights=pen.astype(np.float64), minlength=E)
        off_target = (np.abs(got - k_target) > 0.01 * np.maximum(n_act, 1)) & (delta < max_press)
        if not off_target.any():
            break
        delta = np.where(off_target, solve(thr, delta), delta)
        redo = off_target
    pen = thr < delta[ce]
    got = np.bincount(ce, weights=pen.astype(np.float64), minlength=E)
    depth_c = np.maximum(delta[ce] - thr, 0.0) * slope  # R - phi of the penetrating candidates
    share = got / np.maximum(n_act, 1)
    centre = touch - delta[:, None, None] * u
    link_pose = np.zeros((E, L, 7), np.float32)
    link_pose[..., 3] = 1.0
    link_pose[..., :3] = centre
    link_pose[..., 3:] = mats_to_quats(RL)
    link_pose[absent] = (0, 0, 0, 1, 0, 0, 0)
    link_vel[absent] = 0
    wrap = np.full(E * L, 1 if arc >= 2 * np.pi else 0, np.uint8)
    wrap[absent.reshape(-1)] = 0
    pd = depth_c[depth_c > 0]
    meta = {"placement": {
        "target_share": [float(pen_share[0]), float(pen_share[1])],
        "share_mean": float(share.mean()) if E else 0.0,
        "share_p5_p50_p95": [float(v) for v in np.percentile(share, [5, 50, 95])] if E else [],
        "envs_within_2pct": float(np.mean(np.abs(share - f_target) <= 0.02)) if E else 1.0,
        "press_mm_p5_p50_p95": [float(v) * 1e3 for v in np.percentile(delta, [5, 50, 95])] if E else [],
        "depth_mm_p50_p90_max": ([float(v) * 1e3 for v in np.percentile(pd, [50, 90])] + [float(pd.max()) * 1e3])
        if len(pd) else [],
        "estimate": "nearest-face-plane distance of the exact meshes at the time-0 poses"},
        "placement_env": {"target": f_target, "share": share, "press": delta}}
    return Workload(
        name=name, n_envs=E, max_links=L, taxel_offsets=off, taxel_gid0=off[:-1].copy(),
        env_gid=np.arange(E, dtype=np.int32), link_rows=rows.reshape(-1), link_cols=cols.reshape(-1), link_wrap=wrap,
        x=f32(x), y=f32(y), z=f32(z), nx=f32(np.cos(th)), ny=f32(np.sin(th)), nz=f32(np.zeros(T)), R=f32(Rt),
        objects=objects, obj_id=env_obj.astype(np.int32), link_pose=link_pose, link_vel=link_vel,
        obj_pose=obj_pose, obj_vel=obj_vel, params=params, steps=steps, meta=meta,
    )


def add_pads(wl: Workload, pads_per_env: int = 5, rows: int = 16, cols: int = 16, pitch: float = 1e-3,
             sigma: float = 1.5e-3) -> Workload:
    """Planar 16 x 16 marker pads (1 mm pitch) on the first `pads_per_env`
    links of every env (the fingertips), each tangent to its capsule on the
    side facing the object: origin (r, 0, 0), normal +x, tangent +z (the
    capsule radius r is read back from the link's taxel positions).
    Dilation: s_d = 1, alpha = 1.2, c = 1, lambda_d = 1 / (2 sigma^2),
    eps = pitch, 5 x 5 neighbourhood."""
    E, L = wl.n_envs, wl.max_links
    frame = np.zeros((E, pads_per_env, 9), np.float32)
    link = np.zeros((E, pads_per_env), np.int32)
    rows_ = wl.link_rows.reshape(E, L); cols_ = wl.link_cols.reshape(E, L)
    starts = wl.taxel_offsets[:-1, None] + np.concatenate(
        [np.zeros((E, 1), np.int64), np.cumsum((rows_ * cols_).astype(np.int64), 1)[:, :-1]], 1)
    for p in range(pads_per_env):
        link[:, p] = p
        t0 = starts[:, p]
        r = np.sqrt(wl.x[t0].astype(np.float64) ** 2 + wl.y[t0].astype(np.float64) ** 2)
        frame[:, p, 0] = r
        frame[:, p, 3] = 1.0
        frame[:, p, 8] = 1.0
    wl.pads = dict(pads_per_env=pads_per_env, rows=rows, cols=cols, pitch=pitch, pad_link=link, pad_frame=frame,
                   s_d=1.0, alpha=1.2, lambda_d=1.0 / (2 * sigma * sigma), c=1.0, eps=pitch, radius=2)
    return wl


def config0(seed: int = 20260001, n_envs: int = 64, n_meshes: int = 8) -> Workload:
    """Plain method: 16 capsule links with 200 taxels; per env a sphere
    (r = 30 mm, analytic) or a ~2,000-face mesh (hull of 64 Gaussian points,
    40 mm extent, subdivided twice); one step."""
    rng = np.random.default_rng(seed)
    objects = [ObjectSpec(kind="sphere", radius=float(f32(0.03)), name="sphere30")]
    for i in range(n_meshes):
        V, F = hull_mesh(rng, 64, 0.04, min_faces=1500)
        objects.append(ObjectSpec(kind="mesh", verts=V, faces=F, name=f"hull{i}"))
    env_obj = [0 if rng.uniform() < 0.5 else 1 + int(rng.integers(n_meshes)) for _ in range(n_envs)]
    lat = [(3, 4, 12)] * 12 + [(2, 7, 14)] * 4
    lattices = []
    for _ in range(n_envs):
        order = rng.permutation(16)
        lattices.append([lat[i] for i in order])
    return _assemble("config0", rng, objects, env_obj, lattices, default_params(seed), steps=1)


def config1_objects(rng, n_objects: int = 8, n_grid: int = 64, fp16: bool = False, faces=(3000, 6000)):
    """Half superquadrics (exponents U(0.3, 2)), half convex hulls of 64-256
    points, each with a grid spec over its 1.2x padded bounding box."""
    objs = []
    for i in range(n_objects):
        if i % 2 == 0:
            e1, e2 = rng.uniform(0.3, 2.0, 2)
            axes = rng.uniform(0.012, 0.020, 3)
            target = rng.integers(faces[0], faces[1] + 1)
            n_eta = max(3, int(round(target / 128.0)) + 1)
            V, F = superquadric_mesh(rng, e1, e2, axes, n_eta=n_eta, n_omega=64)
            name = f"superquadric{i}"
        else:
            V, F = hull_mesh(rng, int(rng.integers(64, 257)), 0.04, min_faces=faces[0])
            name = f"hull{i}"
        objs.append(make_grid_object(V, F, n_grid, fp16, name=name))
    return objs


def config1(seed: int = 20260002, n_envs: int = 4096, n_links: int = 20, rows: int = 5, cols: int = 10,
            n_objects: int = 8, n_grid: int = 64, steps: int = 100) -> Workload:
    """Batched grid path: n_envs x 20 links x 50 taxels (5 x 10), 8 objects
    as 64^3 FP32 grids, 100 steps of constant-velocity motion."""
    rng = np.random.default_rng(seed)
    objects = config1_objects(rng, n_objects, n_grid, fp16=False)
    env_obj = rng.integers(0, n_objects, n_envs)
    lattices = [[(rows, cols, rows * cols)] * n_links for _ in range(n_envs)]
    return _assemble("config1", rng, objects, env_obj, lattices, default_params(seed), steps=steps,
                     arc=PAD_ARC)


def uneven_lattices(rng, n_envs, taxels=(200, 1000), links=(10, 20), cols=10):
    """T_e ~ U{taxels}, L_e ~ U{links}; each link's share as a lattice of
    `cols` columns whose last row is padded with R = 0 fillers."""
    out = []
    for _ in range(n_envs):
        T = int(rng.integers(taxels[0], taxels[1] + 1))
        L = int(rng.integers(links[0], links[1] + 1))
        base, rem = divmod(T, L)
        lat = []
        for l in range(L):
            n = base + (1 if l < rem else 0)
            c = min(cols, n)
            r = -(-n // c)
            lat.append((r, c, n))
        out.append(lat)
    return out


def metric_run(seed: int = 20260003, n_envs: int = 20480, n_objects: int = 64, n_grid: int = 96,
               steps: int = 200, faces=(3000, 6000)) -> Workload:
    """Headline workload: n_envs x 20 links x 50 taxels (1,000 per env),
    64 objects as 96^3 FP16 grids, full noise model."""
    rng = np.random.default_rng(seed)
    objects = config1_objects(rng, n_objects, n_grid, fp16=True, faces=faces)
    env_obj = rng.integers(0, n_objects, n_envs)
    lattices = [[(5, 10, 50)] * 20 for _ in range(n_envs)]
    return _assemble("metric_run", rng, objects, env_obj, lattices, default_params(seed), steps=steps,
                     arc=PAD_ARC)


def config2(seed: int = 20260003, n_envs: int = 20480, n_objects: int = 64, n_grid: int = 96,
            steps: int = 200, faces=(3000, 6000)) -> Workload:
    """Full sensor set at scale: uneven T_e ~ U{200..1000}, L_e ~ U{10..20},
    64 objects as 96^3 FP16 grids."""
    rng = np.random.default_rng(seed)
    objects = config1_objects(rng, n_objects, n_grid, fp16=True, faces=faces)
    env_obj = rng.integers(0, n_objects, n_envs)
    lattices = uneven_lattices(rng, n_envs)
    params = default_params(seed)
    params["prox_rays"] = 8
    wl = _assemble("config2", rng, objects, env_obj, lattices, params, steps=steps, max_links=20,
                   arc=PAD_ARC)
    return add_pads(wl)


CONFIG4_DR = {"mu": (0.4, 1.2), "k": (5e3, 2e4), "scale": (0.8, 1.2)}


def config4(seed: int = 20260005, n_envs: int = 20480, n_objects: int = 256, n_grid: int = 96,
            steps: int = 500, faces=(3000, 6000)) -> Workload:
    """Mixed workload with learned parts: uneven T_e ~ U{200..1000} over
    L_e ~ U{10..20} links, 256 objects (96^3 FP16 grid specs; the caller
    trains a network per object), per-step domain randomisation of mu, k and
    the object scale (CONFIG4_DR)."""
    rng = np.random.default_rng(seed)
    objects = config1_objects(rng, n_objects, n_grid, fp16=True, faces=faces)
    env_obj = rng.integers(0, n_objects, n_envs)
    lattices = uneven_lattices(rng, n_envs)
    params = default_params(seed)
    params["dr"] = dict(CONFIG4_DR)
    return _assemble("config4", rng, objects, env_obj, lattices, params, steps=steps, max_links=20, arc=PAD_ARC)


# ---------------------------------------------------------------- TemperatureGrid
TEMP_SILICONE = (0.2, 1100.0, 1500.0, 0.9, 10.0, 0.05, 22.0)   # k, rho, c_p, emissivity, h, tau, base (C)
TEMP_ALUMINIUM = (200.0, 2700.0, 900.0, 0.1, 10.0, 0.0, 22.0)


def temperature_grids(seed: int = 20260011, n_envs: int = 20480, links_per_env: int = 5, dims=(8, 8, 16),
                      extent=(0.02, 0.02, 0.04), metal_share: float = 0.0) -> dict:
    """TemperatureGrid sensors, one per fingertip link (n_envs x links_per_env
    grids of dims cells over a link box of `extent` m, the paper's voxel size
    extent / dims).  Materials: a silicone-like skin (k 0.2 W/m/K, rho 1100,
    c_p 1500, emissivity 0.9, h 10, tau 50 ms), each value scaled by
    U(0.8, 1.2) per grid; a `metal_share` of the grids are aluminium-like
    (k 200, no lag).  Start at the base temperature 22 C."""
    rng = np.random.default_rng(seed)
    G = n_envs * links_per_env
    voxel = np.tile(np.asarray(extent, np.float32) / np.asarray(dims, np.float32), (G, 1))
    mat = np.tile(np.asarray(TEMP_SILICONE, np.float32), (G, 1))
    mat[:, :5] *= rng.uniform(0.8, 1.2, (G, 5)).astype(np.float32)
    mat[:, 3] = np.minimum(mat[:, 3], 1.0)  # emissivity <= 1
    metal = rng.random(G) < metal_share
    mat[metal] = np.asarray(TEMP_ALUMINIUM, np.float32)
    return dict(G=G, dims=tuple(dims), voxel=voxel, material=mat)


def temperature_contacts(rng, G: int, dims, share: float = 0.2, max_per_grid: int = 4, hot_share: float = 0.125,
                         t_hot: float = 45.0, t_amb: float = 22.0) -> dict:
    """Per-step contacts of the fingertip grids with the bin's balls: a `share`
    of the grids touch a ball on 1..max_per_grid cells of one face (the
    voxels under the contact patch), the ball hot (45 C) with probability
    `hot_share`, else at ambient; ball conductivity U(0.2, 2) W/m/K; patch
    areas U(2, 20) mm^2 (the contact manifold's shoelace area).  CSR over grids."""
    nx, ny, nz = dims
    touch = rng.random(G) < share
    counts = np.where(touch, rng.integers(1, max_per_grid + 1, G), 0)
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    C = int(off[-1])
    g_of = np.repeat(np.arange(G), counts)
    face = rng.integers(0, 6, G)[g_of]
    i = rng.integers(0, nx, C); j = rng.integers(0, ny, C); k = rng.integers(0, nz, C)
    i = np.where(face == 0, 0, np.where(face == 1, nx - 1, i))
    j = np.where(face == 2, 0, np.where(face == 3, ny - 1, j))
    k = np.where(face == 4, 0, np.where(face == 5, nz - 1, k))
    hot = (rng.random(G) < hot_share)[g_of]
    return dict(offsets=off, cell=((i * ny + j) * nz + k).astype(np.int32),
                temp=np.where(hot, t_hot, t_amb + rng.uniform(-0.5, 0.5, C)).astype(np.float32),
                k=rng.uniform(0.2, 2.0, C).astype(np.float32), area=rng.uniform(2e-6, 2e-5, C).astype(np.float32))
