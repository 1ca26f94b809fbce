"""Small hand-built scenes and conversions shared by the tests."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2606_22332_gb300 import workload as W


def oracle_nsdf(lo, hi, table, weights):
    """The oracle's copy of learned-SDF parameters (weights split W1 | W2 | W3)."""
    w = np.asarray(weights, np.uint16).reshape(-1)
    return oracle.Nsdf(lo, hi, table, w[:2048].reshape(64, 32), w[2048:6144].reshape(64, 64), w[6144:])


def neural_in_use(o, params):
    """The upload rule: the network answers when 0 <= err * s_max <= nsdf_max_err_mm."""
    smax = params["dr"]["scale"][1] if params.get("dr") else 1.0
    return 0 <= o.nsdf_err_mm and o.nsdf_err_mm * smax <= params.get("nsdf_max_err_mm", 0.2)


def oracle_objects(objects, params=None):
    out = []
    for o in objects:
        if o.kind == "sphere":
            out.append(oracle.Obj.sphere(o.radius))
        elif o.kind == "box":
            out.append(oracle.Obj.box(o.half))
        elif o.kind == "plane":
            out.append(oracle.Obj.plane())
        elif o.kind == "mesh":
            out.append(oracle.Obj.mesh(o.verts, o.faces))
        elif o.kind == "grid" or (o.kind == "neural" and not neural_in_use(o, params or {})):
            assert o.values is not None, "grid object has no baked values"
            out.append(oracle.Obj.grid(o.values, o.lo, o.hi, fp16=o.fp16))
        elif o.kind == "neural":
            assert o.nsdf_table is not None, "the oracle needs the network's parameters"
            net = oracle_nsdf(o.nsdf_lo, o.nsdf_hi, o.nsdf_table, o.nsdf_weights)
            out.append(oracle.Obj.neural(net, o.values, o.lo, o.hi, fp16=o.fp16))
        else:
            raise ValueError(o.kind)
    return out


def oracle_scene(wl: W.Workload):
    return oracle.OracleScene(wl.geom(), oracle_objects(wl.objects, wl.params), wl.params)


def neural_switch_band(wl, used, band=1e-6):
    """Taxels of the envs whose object answers through its network that lie
    within `band` of the switch between network and fallback grid (the grid's
    s phi = R + 1 mm, reading R30): the GPU decides that switch on its FP32
    grid distance, the oracle on its FP64 one, so there either field may
    answer.  A grid-only oracle scene (each such object replaced by its
    fallback grid) gives the grid's distance at every taxel; its state is
    not used.  Returns a function of the step's inputs."""
    objs = []
    for k, o in enumerate(wl.objects):
        if o.kind == "neural":
            o = W.ObjectSpec(kind="grid", dims=o.dims, lo=o.lo, hi=o.hi, fp16=o.fp16, values=o.values)
        objs.append(o)
    sub = W.Workload(**{f: getattr(wl, f) for f in wl.__dataclass_fields__})
    sub.objects = objs
    grid_scene = oracle_scene(sub)
    st = grid_scene.new_state()
    grid_scene.reset(st, 0)
    in_net = np.repeat(np.isin(wl.obj_id, list(used)), np.diff(wl.taxel_offsets)) & (wl.R > 0)

    def at(inputs):
        out = grid_scene.step(st, inputs)
        return in_net & (np.abs(out["dist"] - 1e-3) < band)

    return at


def pad_workload(depths, rows, cols, params=None, wrap=0, pitch=1e-3, obj=None,
                 link_vel=(0, 0, 0, 0, 0, 0), obj_vel=(0, 0, 0, 0, 0, 0), R=1e-3, link_quat=(1, 0, 0, 0)):
    """One env, one flat pad link over the half-space z <= 0.

    The pad is a rows x cols lattice in the link's z = 0 plane with pitch
    `pitch`, probe normals -z (facing the plane).  The link origin sits at
    height h above the plane, so a probe at link position x is at world
    height h + x_z; `depths` (rows x cols, or a scalar) sets each probe's
    link-frame z so that its penetration R - phi equals the given depth.
    """
    depths = np.broadcast_to(np.asarray(depths, dtype=np.float64), (rows, cols))
    h = 0.01
    rr, cc = np.meshgrid(np.arange(rows), np.arange(cols), indexing="ij")
    x = (cc - (cols - 1) / 2.0) * pitch
    y = (rr - (rows - 1) / 2.0) * pitch
    z = -(h - (R - depths))          # world height of the probe = R - depth
    T = rows * cols
    params = params or W.default_params(1234)
    objs = [obj or W.ObjectSpec(kind="plane")]
    lp = np.zeros((1, 1, 7), np.float32); lp[0, 0, 2] = h; lp[0, 0, 3:] = link_quat
    lv = np.asarray(link_vel, np.float32).reshape(1, 1, 6)
    op = np.zeros((1, 7), np.float32); op[0, 3] = 1.0
    ov = np.asarray(obj_vel, np.float32).reshape(1, 6)
    f = lambda a: W.f32(np.asarray(a).reshape(-1))
    return W.Workload(
        name="pad", n_envs=1, max_links=1, taxel_offsets=np.array([0, T], np.int64),
        taxel_gid0=np.array([0], np.int64), env_gid=np.array([0], np.int32),
        link_rows=np.array([rows], np.int32), link_cols=np.array([cols], np.int32),
        link_wrap=np.array([wrap], np.uint8),
        x=f(x), y=f(y), z=f(z), nx=f(np.zeros(T)), ny=f(np.zeros(T)), nz=f(-np.ones(T)),
        R=f(np.full(T, R)), objects=objs, obj_id=np.array([0], np.int32),
        link_pose=lp, link_vel=lv, obj_pose=op, obj_vel=ov, params=params, steps=1,
    )


def quiet_params(seed=1234, **over):
    """Default parameters with every noise knob off."""
    p = W.default_params(seed)
    p["p_dead"] = 0.0
    p["chi"] = 0.0
    for g in ("depth", "ft", "prox"):
        p["noise"][g] = W.noise_group()
    p.update(over)
    return p


def bake_objects_oracle(objects, dims=None):
    """Fill every grid object's values with the oracle's exact-mesh bake
    (optionally at other dims); returns the list of objects."""
    out = []
    for o in objects:
        if o.kind == "grid":
            d = tuple(dims) if dims is not None else tuple(o.dims)
            vals = oracle.bake_grid(o.verts, o.faces, d, o.lo.astype(np.float64), o.hi.astype(np.float64), fp16=o.fp16)
            o = W.ObjectSpec(kind="grid", verts=o.verts, faces=o.faces, dims=d, lo=o.lo, hi=o.hi, fp16=o.fp16,
                             values=vals, name=o.name)
        out.append(o)
    return out


def low_poly_grid_objects(rng, n_objects, n_grid, fp16, points=(12, 40)):
    """Grid objects over low-face-count hulls (fast to bake exactly at full
    grid resolution), for full-size runs the oracle can check."""
    objs = []
    for i in range(n_objects):
        V, F = W.hull_mesh(rng, int(rng.integers(*points)), 0.04)
        objs.append(W.make_grid_object(V, F, n_grid, fp16, name=f"lowpoly{i}"))
    return bake_objects_oracle(objs)
