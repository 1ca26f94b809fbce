"""FP64 CPU oracle for the Tactile Genesis contact query and noise model.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference legs of ``bench.py`` may import this package.  It
shares no code with the CUDA path and takes no input from it.

The arithmetic lives in ``tg_oracle.c`` (plain C, double precision, one
function per passage of the paper); this module only compiles it and
marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tg_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "tg_oracle_nsdf.c")]
_LIB_PATH = os.path.join(_HERE, "_tg_oracle.so")
_lib = None
_lock = threading.Lock()

OR_SPHERE, OR_BOX, OR_PLANE, OR_MESH, OR_GRID, OR_NEURAL = 0, 1, 2, 3, 4, 5
NSDF_LEVELS, NSDF_FEATURES, NSDF_TABLE, NSDF_HIDDEN = 16, 2, 1 << 16, 64
NSDF_IN = NSDF_LEVELS * NSDF_FEATURES
NCH = 8
RING_CH = 8   # read-delay ring channels: depth, force/torque (6), noisy contact bit
LINK_REC = 18


def build(force: bool = False) -> str:
    """Compile the oracle's C sources into _tg_oracle.so (OpenMP when the compiler has it)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
        [os.path.getmtime(f) for f in _SRCS] + [os.path.getmtime(os.path.join(_HERE, "tg_oracle.h"))]
    ):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC"] + _SRCS + ["-o", _LIB_PATH + ".tmp"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:] + ["-lm"], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-lm"], check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


class ORObject(C.Structure):
    _fields_ = [
        ("kind", C.c_int32), ("radius", C.c_double), ("half", C.c_double * 3),
        ("n_verts", C.c_int32), ("n_faces", C.c_int32),
        ("verts", C.c_void_p), ("faces", C.c_void_p),
        ("dims", C.c_int32 * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
        ("fp16", C.c_int32), ("values", C.c_void_p), ("nsdf", C.c_void_p),
    ]


class ORNsdf(C.Structure):
    _fields_ = [("lo", C.c_double * 3), ("hi", C.c_double * 3), ("table", C.c_void_p), ("w1", C.c_void_p),
                ("w2", C.c_void_p), ("w3", C.c_void_p)]


class ORNoiseGroup(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "gain_lo", "gain_hi", "beta", "tau", "bias", "sigma_white", "sigma_rw", "quant", "stuck_lo", "stuck_hi")]


class ORParams(C.Structure):
    _fields_ = [
        ("k", C.c_double), ("c", C.c_double), ("alpha", C.c_double), ("k_t", C.c_double),
        ("k_omega", C.c_double), ("mu", C.c_double), ("eta_on", C.c_double), ("eta_off", C.c_double),
        ("dt", C.c_double), ("seed", C.c_uint64), ("p_dead", C.c_double),
        ("depth", ORNoiseGroup), ("ft", ORNoiseGroup), ("prox", ORNoiseGroup),
        ("chi", C.c_double), ("xt_sigma", C.c_double),
        ("prox_rays", C.c_int32), ("prox_range", C.c_double), ("prox_cone", C.c_double),
        ("dr_on", C.c_int32), ("dr_mu", C.c_double * 2), ("dr_k", C.c_double * 2), ("dr_scale", C.c_double * 2),
        ("rho", C.c_double), ("delay", C.c_int32), ("jitter", C.c_int32), ("depth_backend", C.c_int32),
    ]


class ORPads(C.Structure):
    _fields_ = [("pads_per_env", C.c_int32), ("rows", C.c_int32), ("cols", C.c_int32), ("pitch", C.c_double),
                ("pad_link", C.c_void_p), ("pad_frame", C.c_void_p),
                ("s_d", C.c_double), ("alpha", C.c_double), ("lambda_d", C.c_double), ("c", C.c_double),
                ("eps", C.c_double), ("radius", C.c_int32)]


class ORPcProx(C.Structure):
    _fields_ = [("cloud", C.c_void_p), ("cloud_off", C.c_void_p), ("radius", C.c_double), ("k", C.c_double),
                ("ks", C.c_double), ("density", C.c_double)]


class ORShear(C.Structure):
    _fields_ = [("cloud", C.c_void_p), ("cloud_off", C.c_void_p), ("s_s", C.c_double), ("lambda_s", C.c_double),
                ("eta_enter", C.c_double), ("eta_exit", C.c_double), ("thickness", C.c_double),
                ("n_max", C.c_int64)]


class ORScene(C.Structure):
    _fields_ = [
        ("n_envs", C.c_int32), ("max_links", C.c_int32),
        ("taxel_offsets", C.c_void_p), ("taxel_gid0", C.c_void_p), ("env_gid", C.c_void_p),
        ("link_rows", C.c_void_p), ("link_cols", C.c_void_p), ("link_wrap", C.c_void_p),
        ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p),
        ("nx", C.c_void_p), ("ny", C.c_void_p), ("nz", C.c_void_p), ("R", C.c_void_p),
        ("objects", C.c_void_p), ("n_objects", C.c_int32), ("params", ORParams),
    ]


class ORInputs(C.Structure):
    _fields_ = [
        ("link_pose", C.c_void_p), ("link_vel", C.c_void_p), ("obj_pose", C.c_void_p),
        ("obj_vel", C.c_void_p), ("obj_id", C.c_void_p), ("env_params", C.c_void_p),
        ("pose_dt", C.c_double), ("step", C.c_uint32),
    ]


class ORState(C.Structure):
    _fields_ = [("flags", C.c_void_p), ("hyst_prev", C.c_void_p), ("hyst_xi", C.c_void_p),
                ("drift", C.c_void_p), ("episode", C.c_void_p), ("ring", C.c_void_p)]


class OROutputs(C.Structure):
    _fields_ = [("contact_clean", C.c_void_p), ("contact_noisy", C.c_void_p),
                ("prox_clean", C.c_void_p), ("prox_noisy", C.c_void_p), ("prox_grazing", C.c_void_p),
                ("depth_clean", C.c_void_p), ("depth_noisy", C.c_void_p), ("dist", C.c_void_p),
                ("ft_clean", C.c_void_p), ("ft_noisy", C.c_void_p),
                ("link_sums", C.c_void_p), ("link_counts", C.c_void_p), ("depth_tie", C.c_void_p)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            L.or_philox4x32_10.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
            L.or_uniform.argtypes = [C.c_uint32]; L.or_uniform.restype = C.c_double
            L.or_box_muller.argtypes = [C.c_uint32, C.c_uint32, dp, dp]
            L.or_double_to_half.argtypes = [C.c_double]; L.or_double_to_half.restype = C.c_uint16
            L.or_half_to_double.argtypes = [C.c_uint16]; L.or_half_to_double.restype = C.c_double
            L.or_quat_to_mat.argtypes = [C.c_void_p, C.c_void_p]
            L.or_advance_pose.argtypes = [C.c_void_p] * 4 + [C.c_double, C.c_void_p, C.c_void_p]
            L.or_closest_point_triangle.argtypes = [C.c_void_p] * 5 + [C.POINTER(C.c_int)]
            L.or_closest_point_triangle.restype = C.c_double
            L.or_winding_number.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]
            L.or_winding_number.restype = C.c_double
            L.or_sdf_object_batch.argtypes = [C.POINTER(ORObject), C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
            L.or_schmitt.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double]; L.or_schmitt.restype = C.c_int
            L.or_taxel_force.argtypes = [C.POINTER(ORParams), C.c_double, C.c_double, C.c_double,
                                         C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p]
            L.or_crosstalk_weights.argtypes = [C.c_double, C.c_void_p]
            L.or_bake_grid.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_int32, C.c_void_p, C.c_int32]
            L.or_reset.argtypes = [C.POINTER(ORScene), C.c_void_p, C.c_uint32, C.POINTER(ORState)]
            L.or_step.argtypes = [C.POINTER(ORScene), C.POINTER(ORInputs), C.POINTER(ORState),
                                  C.POINTER(OROutputs), C.c_int32]
            L.or_step.restype = C.c_int
            L.or_ray_first_root.argtypes = [C.POINTER(ORObject), C.c_double, C.c_void_p, C.c_void_p, C.c_double,
                                            C.POINTER(C.c_int)]
            L.or_ray_first_root.restype = C.c_double
            L.or_prox_ray_dirs.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_void_p]
            L.or_bf16_to_double.argtypes = [C.c_uint16]; L.or_bf16_to_double.restype = C.c_double
            L.or_double_to_bf16.argtypes = [C.c_double]; L.or_double_to_bf16.restype = C.c_uint16
            L.or_nsdf_resolution.argtypes = [C.c_int32]; L.or_nsdf_resolution.restype = C.c_int32
            L.or_nsdf_index.argtypes = [C.c_int32, C.c_int64, C.c_int64, C.c_int64]
            L.or_nsdf_index.restype = C.c_uint32
            L.or_nsdf_eval_batch.argtypes = [C.POINTER(ORNsdf), C.c_int64, C.c_void_p, C.c_int32, C.c_void_p,
                                             C.c_void_p]
            L.or_nsdf_normal_batch.argtypes = [C.POINTER(ORNsdf), C.c_int64, C.c_void_p, C.c_int32, C.c_void_p]
            L.or_nsdf_flip_bound_batch.argtypes = [C.POINTER(ORNsdf), C.c_int64, C.c_void_p, C.c_void_p]
            L.or_nsdf_loss_grad.argtypes = [C.POINTER(ORNsdf), C.c_int64, C.c_void_p, C.c_void_p, C.c_int32,
                                            C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            L.or_nsdf_loss_grad.restype = C.c_double
            L.or_adam_step.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                       C.c_double, C.c_double, C.c_double, C.c_int32]
            L.or_dr_draw.argtypes = [C.POINTER(ORParams), C.c_uint32, C.c_uint32, C.c_void_p]
            L.or_read_delay.argtypes = [C.POINTER(ORParams), C.c_uint32, C.c_uint32]
            L.or_read_delay.restype = C.c_int32
            L.or_marker_kernel_g.argtypes = [C.c_double, C.c_double]
            L.or_marker_kernel_g.restype = C.c_double
            L.or_markers.argtypes = [C.POINTER(ORScene), C.POINTER(ORPads), C.POINTER(ORInputs), C.c_void_p,
                                     C.c_void_p, C.c_int32]
            L.or_pc_prox.argtypes = [C.POINTER(ORScene), C.POINTER(ORPcProx), C.POINTER(ORInputs), C.c_void_p,
                                     C.c_int32]
            L.or_shear_step.argtypes = [C.POINTER(ORScene), C.POINTER(ORPads), C.POINTER(ORShear),
                                        C.POINTER(ORInputs), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.c_int32]
            L.or_raycast_depth.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_double, C.c_void_p, C.c_void_p,
                                           C.c_double, C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_double)]
            L.or_raycast_depth.restype = C.c_double
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data if a is not None else None


# --------------------------------------------------------------------------
# primitives
# --------------------------------------------------------------------------
def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(_p(c), _p(k), _p(o))
    return o


def uniform(x):
    return lib().or_uniform(int(x))


def box_muller(x0, x1):
    z0, z1 = C.c_double(), C.c_double()
    lib().or_box_muller(int(x0), int(x1), C.byref(z0), C.byref(z1))
    return z0.value, z1.value


def double_to_half(x):
    return lib().or_double_to_half(float(x))


def half_to_double(h):
    return lib().or_half_to_double(int(h))


def quat_to_mat(q):
    q = np.ascontiguousarray(q, np.float64)
    R = np.zeros(9)
    lib().or_quat_to_mat(_p(q), _p(R))
    return R.reshape(3, 3)


def advance_pose(p0, q0, v, w, tau):
    a = [np.ascontiguousarray(t, np.float64) for t in (p0, q0, v, w)]
    p = np.zeros(3); R = np.zeros(9)
    lib().or_advance_pose(*[_p(t) for t in a], float(tau), _p(p), _p(R))
    return p, R.reshape(3, 3)


def closest_point_triangle(p, a, b, c):
    arr = [np.ascontiguousarray(t, np.float64) for t in (p, a, b, c)]
    cp = np.zeros(3)
    reg = C.c_int()
    d = lib().or_closest_point_triangle(*[_p(t) for t in arr], _p(cp), C.byref(reg))
    return d, cp, reg.value


def winding_number(verts, faces, p):
    V = np.ascontiguousarray(verts, np.float32); F = np.ascontiguousarray(faces, np.int32)
    p = np.ascontiguousarray(p, np.float64)
    return lib().or_winding_number(_p(V), _p(F), len(F), _p(p))


class Obj:
    """An oracle object; keeps the arrays its ctypes struct points at alive."""

    def __init__(self, kind, radius=0.0, half=(0, 0, 0), verts=None, faces=None,
                 dims=(0, 0, 0), lo=(0, 0, 0), hi=(0, 0, 0), values=None, fp16=False):
        self.keep = []
        s = ORObject()
        s.kind = kind
        s.radius = float(radius)
        s.half[:] = [float(h) for h in half]
        if verts is not None:
            V = np.ascontiguousarray(verts, np.float32); F = np.ascontiguousarray(faces, np.int32)
            self.keep += [V, F]
            s.n_verts, s.n_faces = len(V), len(F)
            s.verts, s.faces = _p(V), _p(F)
        if values is not None:
            vals = np.ascontiguousarray(values, np.uint16 if fp16 else np.float32)
            self.keep.append(vals)
            s.values = _p(vals)
            s.fp16 = 1 if fp16 else 0
        s.dims[:] = [int(d) for d in dims]
        s.lo[:] = [float(v) for v in lo]
        s.hi[:] = [float(v) for v in hi]
        self.s = s

    @staticmethod
    def sphere(r):
        return Obj(OR_SPHERE, radius=r)

    @staticmethod
    def box(half):
        return Obj(OR_BOX, half=half)

    @staticmethod
    def plane():
        return Obj(OR_PLANE)

    @staticmethod
    def mesh(verts, faces):
        return Obj(OR_MESH, verts=verts, faces=faces)

    @staticmethod
    def grid(values, lo, hi, fp16=False):
        values = np.asarray(values)
        nz, ny, nx = values.shape
        return Obj(OR_GRID, dims=(nx, ny, nz), lo=lo, hi=hi, values=values, fp16=fp16)

    @staticmethod
    def neural(net: "Nsdf", grid_values=None, grid_lo=None, grid_hi=None, fp16=True):
        """A learned-SDF object; the optional grid is its fallback (proximity rays march it)."""
        if grid_values is not None:
            grid_values = np.asarray(grid_values)
            nz, ny, nx = grid_values.shape
            o = Obj(OR_NEURAL, dims=(nx, ny, nz), lo=grid_lo, hi=grid_hi, values=grid_values, fp16=fp16)
        else:
            o = Obj(OR_NEURAL)
        o.keep.append(net)
        o.s.nsdf = C.cast(C.pointer(net.s), C.c_void_p).value
        return o

    def sdf(self, q):
        q = np.ascontiguousarray(np.atleast_2d(q), np.float64)
        n = len(q)
        phi = np.zeros(n); g = np.zeros((n, 3))
        lib().or_sdf_object_batch(C.byref(self.s), _p(q), n, _p(phi), _p(g))
        return phi, g


class Nsdf:
    """Learned SDF parameters for the oracle: box lo/hi (m), table [16][2^16][2]
    binary16 bits, w1 [64][32], w2 [64][64], w3 [64] bfloat16 bits."""

    def __init__(self, lo, hi, table, w1, w2, w3):
        self.table = np.ascontiguousarray(table, np.uint16).reshape(NSDF_LEVELS, NSDF_TABLE, NSDF_FEATURES)
        self.w1 = np.ascontiguousarray(w1, np.uint16).reshape(NSDF_HIDDEN, NSDF_IN)
        self.w2 = np.ascontiguousarray(w2, np.uint16).reshape(NSDF_HIDDEN, NSDF_HIDDEN)
        self.w3 = np.ascontiguousarray(w3, np.uint16).reshape(NSDF_HIDDEN)
        s = ORNsdf()
        s.lo[:] = [float(v) for v in lo]
        s.hi[:] = [float(v) for v in hi]
        s.table, s.w1, s.w2, s.w3 = _p(self.table), _p(self.w1), _p(self.w2), _p(self.w3)
        self.s = s

    def eval(self, q, round=True, grad=False):
        """phi (m) and, with grad, the raw gradient d phi / d q (not normalised)."""
        q = np.ascontiguousarray(np.atleast_2d(q), np.float64)
        n = len(q)
        phi = np.zeros(n)
        g = np.zeros((n, 3)) if grad else None
        lib().or_nsdf_eval_batch(C.byref(self.s), n, _p(q), 1 if round else 0, _p(phi), _p(g) if grad else None)
        return (phi, g) if grad else phi

    def normal(self, q, round=True):
        """Contact-normal gradient (tetrahedral central difference, h = 0.25 mm), not normalised."""
        q = np.ascontiguousarray(np.atleast_2d(q), np.float64)
        g = np.zeros((len(q), 3))
        lib().or_nsdf_normal_batch(C.byref(self.s), len(q), _p(q), 1 if round else 0, _p(g))
        return g

    def flip_bound(self, q):
        """Per point, the largest output change (mm) one bfloat16 rounding flip can cause."""
        q = np.ascontiguousarray(np.atleast_2d(q), np.float64)
        out = np.zeros(len(q))
        lib().or_nsdf_flip_bound_batch(C.byref(self.s), len(q), _p(q), _p(out))
        return out

    def loss_grad(self, pts, labels_mm, round=True):
        """(loss, g_w1, g_w2, g_w3, g_table) of the mean L1 loss, FP64."""
        pts = np.ascontiguousarray(pts, np.float64)
        y = np.ascontiguousarray(labels_mm, np.float64)
        g1 = np.zeros((NSDF_HIDDEN, NSDF_IN)); g2 = np.zeros((NSDF_HIDDEN, NSDF_HIDDEN)); g3 = np.zeros(NSDF_HIDDEN)
        gt = np.zeros((NSDF_LEVELS, NSDF_TABLE, NSDF_FEATURES))
        loss = lib().or_nsdf_loss_grad(C.byref(self.s), len(pts), _p(pts), _p(y), 1 if round else 0,
                                       _p(g1), _p(g2), _p(g3), _p(gt))
        return loss, g1, g2, g3, gt


def bf16_to_double(b):
    return lib().or_bf16_to_double(int(b))


def double_to_bf16(x):
    return int(lib().or_double_to_bf16(float(x)))


def nsdf_resolution(level):
    return int(lib().or_nsdf_resolution(int(level)))


def nsdf_index(level, i, j, k):
    return int(lib().or_nsdf_index(int(level), int(i), int(j), int(k)))


def adam_step(theta, m, v, g, lr, beta1, beta2, eps, t):
    """In place on float64 arrays."""
    for a in (theta, m, v, g):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().or_adam_step(theta.size, _p(theta), _p(m), _p(v), _p(g), float(lr), float(beta1), float(beta2),
                       float(eps), int(t))


def ray_first_root(obj: "Obj", q0, d, tmax, scale=1.0):
    """(t or nan, grazing) of the first root of the object's SDF along q0 + t d."""
    q0 = np.ascontiguousarray(q0, np.float64); d = np.ascontiguousarray(d, np.float64)
    g = C.c_int(0)
    t = lib().or_ray_first_root(C.byref(obj.s), float(scale), _p(q0), _p(d), float(tmax), C.byref(g))
    return t, bool(g.value)


def prox_ray_dirs(n, n_rays, cone):
    n = np.ascontiguousarray(n, np.float64)
    out = np.zeros((n_rays, 3))
    lib().or_prox_ray_dirs(_p(n), int(n_rays), float(cone), _p(out))
    return out


def marker_kernel_g(lambda_d, r2):
    return lib().or_marker_kernel_g(float(lambda_d), float(r2))


def dr_draw(params: dict, env_gid: int, step: int):
    """(mu, k, scale) drawn for one env and step by per-step domain randomisation."""
    P = make_params(params)
    out = np.zeros(3, np.float64)
    lib().or_dr_draw(C.byref(P), C.c_uint32(env_gid), C.c_uint32(step), _p(out))
    return out


def read_delay(params: dict, env_gid: int, step: int) -> int:
    """The read delay (steps) of one env at one step: delay + jitter draw."""
    return int(lib().or_read_delay(C.byref(make_params(params)), C.c_uint32(env_gid), C.c_uint32(step)))


def schmitt(prev, d, eta_on, eta_off):
    return lib().or_schmitt(int(prev), float(d), float(eta_on), float(eta_off))


def crosstalk_weights(sigma):
    w = np.zeros(9)
    lib().or_crosstalk_weights(float(sigma), _p(w))
    return w.reshape(3, 3)


def bake_grid(verts, faces, dims, lo, hi, fp16=False, threads=0):
    """Exact mesh SDF at the grid nodes, rounded to float32 or binary16 bits; [z][y][x]."""
    V = np.ascontiguousarray(verts, np.float32); F = np.ascontiguousarray(faces, np.int32)
    d = np.ascontiguousarray(dims, np.int32)
    lo = np.ascontiguousarray(lo, np.float64); hi = np.ascontiguousarray(hi, np.float64)
    out = np.zeros((d[2], d[1], d[0]), np.uint16 if fp16 else np.float32)
    lib().or_bake_grid(_p(V), _p(F), len(F), _p(d), _p(lo), _p(hi), 1 if fp16 else 0, _p(out), int(threads))
    return out


# --------------------------------------------------------------------------
# parameters
# --------------------------------------------------------------------------
_GROUP_KEYS = ("gain_lo", "gain_hi", "beta", "tau", "bias", "sigma_white", "sigma_rw", "quant", "stuck_lo", "stuck_hi")


def make_params(p: dict) -> ORParams:
    """Fill the C parameter struct from the plain dict used by the workloads."""
    P = ORParams()
    for k in ("k", "c", "alpha", "k_t", "k_omega", "eta_on", "eta_off", "dt", "p_dead", "chi", "xt_sigma"):
        setattr(P, k, float(p[k]))
    P.mu = -1.0 if p["mu"] is None or np.isinf(p["mu"]) else float(p["mu"])
    P.seed = int(p["seed"])
    P.prox_rays = int(p.get("prox_rays", 0))
    P.prox_range = float(p.get("prox_range", 0.05))
    P.prox_cone = float(p.get("prox_cone", np.radians(30.0)))
    P.rho = float(p.get("rho", 0.0))
    P.delay = int(p.get("read_delay", 0))
    P.jitter = int(p.get("read_jitter", 0))
    P.depth_backend = {"sdf": 0, "raycast": 1}[p.get("depth_backend", "sdf")]
    dr = p.get("dr")
    P.dr_on = 1 if dr else 0
    if dr:
        for k in ("mu", "k", "scale"):
            getattr(P, "dr_" + k)[0] = float(dr[k][0])
            getattr(P, "dr_" + k)[1] = float(dr[k][1])
    for gname in ("depth", "ft", "prox"):
        g = getattr(P, gname)
        for k in _GROUP_KEYS:
            setattr(g, k, float(p["noise"][gname][k]))
    return P


def taxel_force(params: dict, k, mu, d, x, mbar, vrel, dw_dot_m):
    P = make_params(params)
    arr = [np.ascontiguousarray(t, np.float64) for t in (x, mbar, vrel)]
    f = np.zeros(3); tau = np.zeros(3)
    mu_c = -1.0 if mu is None or np.isinf(mu) else float(mu)
    lib().or_taxel_force(C.byref(P), float(k), mu_c, float(d), *[_p(t) for t in arr], float(dw_dot_m), _p(f), _p(tau))
    return f, tau


# --------------------------------------------------------------------------
# whole-scene oracle
# --------------------------------------------------------------------------
class OracleScene:
    """A (sub)scene in oracle form.

    ``geom`` is a dict with the workload's static arrays (taxel_offsets,
    taxel_gid0, env_gid, link_rows, link_cols, link_wrap, x..R) and ``objects``
    a list of :class:`Obj`.
    """

    def __init__(self, geom: dict, objects: list, params: dict):
        self.keep = {}
        g = {}
        for k, dt in (("taxel_offsets", np.int64), ("taxel_gid0", np.int64), ("env_gid", np.int32),
                      ("link_rows", np.int32), ("link_cols", np.int32), ("link_wrap", np.uint8),
                      ("x", np.float32), ("y", np.float32), ("z", np.float32),
                      ("nx", np.float32), ("ny", np.float32), ("nz", np.float32), ("R", np.float32)):
            g[k] = np.ascontiguousarray(geom[k], dt)
        self.keep.update(g)
        self.n_envs = len(g["taxel_offsets"]) - 1
        self.max_links = len(g["link_rows"]) // self.n_envs
        self.T = int(g["taxel_offsets"][-1])
        self.objects = objects
        arr = (ORObject * len(objects))(*[o.s for o in objects])
        self.keep["objarr"] = arr
        S = ORScene()
        S.n_envs, S.max_links = self.n_envs, self.max_links
        for k in g:
            setattr(S, k, _p(g[k]))
        S.objects = C.cast(arr, C.c_void_p)
        S.n_objects = len(objects)
        S.params = make_params(params)
        self.S = S
        self.params = params

    def new_state(self):
        T, E = self.T, self.n_envs
        K = int(self.params.get("read_delay", 0)) + int(self.params.get("read_jitter", 0)) + 1
        return {
            "flags": np.zeros(T, np.uint8),
            "hyst_prev": np.zeros((NCH, T)), "hyst_xi": np.zeros((NCH, T)), "drift": np.zeros((NCH, T)),
            "episode": np.zeros(E, np.uint32),
            "ring": np.zeros((K, RING_CH, T)) if K > 1 else None,
        }

    def _state(self, st):
        s = ORState()
        for k in ("flags", "hyst_prev", "hyst_xi", "drift", "episode"):
            setattr(s, k, _p(st[k]))
        s.ring = _p(st.get("ring"))
        return s

    def reset(self, st, episode, env_mask=None):
        m = None if env_mask is None else np.ascontiguousarray(env_mask, np.uint8)
        s = self._state(st)
        lib().or_reset(C.byref(self.S), _p(m), int(episode), C.byref(s))

    def step(self, st, inputs: dict, threads: int = 0):
        T, E, L = self.T, self.n_envs, self.max_links
        keep = {}
        I = ORInputs()
        for k, dt in (("link_pose", np.float32), ("link_vel", np.float32), ("obj_pose", np.float32),
                      ("obj_vel", np.float32), ("obj_id", np.int32)):
            keep[k] = np.ascontiguousarray(inputs[k], dt)
            setattr(I, k, _p(keep[k]))
        if inputs.get("env_params") is not None:
            keep["env_params"] = np.ascontiguousarray(inputs["env_params"], np.float32)
            I.env_params = _p(keep["env_params"])
        I.pose_dt = float(inputs.get("pose_dt", 0.0))
        I.step = int(inputs.get("step", 0))
        out = {
            "contact_clean": np.zeros(T, np.uint8), "contact_noisy": np.zeros(T, np.uint8),
            "prox_clean": np.zeros(T), "prox_noisy": np.zeros(T), "prox_grazing": np.zeros(T, np.uint8),
            "depth_clean": np.zeros(T), "depth_noisy": np.zeros(T), "dist": np.zeros(T),
            "ft_clean": np.zeros((6, T)), "ft_noisy": np.zeros((6, T)),
            "link_sums": np.zeros((E * L, LINK_REC)), "link_counts": np.zeros((E * L, 2), np.int32),
            "depth_tie": np.zeros(T, np.uint8),
        }
        O = OROutputs()
        for k in out:
            setattr(O, k, _p(out[k]))
        s = self._state(st)
        lib().or_step(C.byref(self.S), C.byref(I), C.byref(s), C.byref(O), int(threads))
        return out

    @staticmethod
    def _pads(pads: dict, keep: dict) -> ORPads:
        keep["link"] = np.ascontiguousarray(pads["pad_link"], np.int32)
        keep["frame"] = np.ascontiguousarray(pads["pad_frame"], np.float32)
        Pd = ORPads()
        Pd.pads_per_env, Pd.rows, Pd.cols = int(pads["pads_per_env"]), int(pads["rows"]), int(pads["cols"])
        Pd.pitch = float(pads["pitch"])
        Pd.pad_link, Pd.pad_frame = _p(keep["link"]), _p(keep["frame"])
        for k in ("s_d", "alpha", "lambda_d", "c", "eps"):
            setattr(Pd, k, float(pads[k]))
        Pd.radius = int(pads["radius"])
        return Pd

    @staticmethod
    def _pose_inputs(inputs: dict, keep: dict) -> ORInputs:
        I = ORInputs()
        for k, dt in (("link_pose", np.float32), ("link_vel", np.float32), ("obj_pose", np.float32),
                      ("obj_vel", np.float32), ("obj_id", np.int32)):
            keep[k] = np.ascontiguousarray(inputs[k], dt)
            setattr(I, k, _p(keep[k]))
        if inputs.get("env_params") is not None:
            keep["env_params"] = np.ascontiguousarray(inputs["env_params"], np.float32)
            I.env_params = _p(keep["env_params"])
        I.pose_dt = float(inputs.get("pose_dt", 0.0))
        I.step = int(inputs.get("step", 0))
        return I

    def new_shear_state(self, pads_per_env: int, n_max: int) -> dict:
        """Shear-anchor state with no anchors: anchors [E][P][n_max][2] (NaN = none), anchor_obj [E][P]."""
        E = self.n_envs
        return {"anchors": np.full((E, pads_per_env, n_max, 2), np.nan),
                "anchor_obj": np.full((E, pads_per_env), -1, np.int32)}

    def shear_step(self, pads: dict, clouds, shear: dict, inputs: dict, state: dict, threads: int = 0,
                   drag: bool = False):
        """One step of the ElastomerTaxel shear anchors (Eqs. 19-20): updates
        `state` in place and returns (u [E][P][rows*cols][3] the shear part of
        the marker displacements, n_anchored [E][P], margin [E][P], and, with
        drag=True, also drag [E][P] (see or_shear_step)).  clouds[o]:
        object o's tracked points ([n_o][3], object frame); shear: s_s,
        lambda_s, eta_enter, eta_exit, thickness."""
        E = self.n_envs
        keep = {"cloud": np.ascontiguousarray(np.concatenate([np.asarray(c, np.float32).reshape(-1, 3)
                                                              for c in clouds]), np.float32),
                "off": np.ascontiguousarray(np.concatenate([[0], np.cumsum([len(c) for c in clouds])]), np.int64)}
        Pd = self._pads(pads, keep)
        an, ao = state["anchors"], state["anchor_obj"]
        assert an.dtype == np.float64 and an.flags.c_contiguous and ao.dtype == np.int32 and ao.flags.c_contiguous
        assert an.shape == (E, Pd.pads_per_env, an.shape[2], 2) and an.shape[2] >= max(len(c) for c in clouds)
        Sh = ORShear()
        Sh.cloud, Sh.cloud_off = _p(keep["cloud"]), _p(keep["off"])
        for k in ("s_s", "lambda_s", "eta_enter", "eta_exit", "thickness"):
            setattr(Sh, k, float(shear[k]))
        Sh.n_max = an.shape[2]
        I = self._pose_inputs(inputs, keep)
        M = Pd.rows * Pd.cols
        u = np.zeros((E, Pd.pads_per_env, M, 3))
        na = np.zeros((E, Pd.pads_per_env), np.int32)
        mg = np.zeros((E, Pd.pads_per_env))
        dg = np.zeros((E, Pd.pads_per_env))
        lib().or_shear_step(C.byref(self.S), C.byref(Pd), C.byref(Sh), C.byref(I), _p(an), _p(ao), _p(u), _p(na),
                            _p(mg), _p(dg), int(threads))
        return (u, na, mg, dg) if drag else (u, na, mg)

    def markers(self, pads: dict, inputs: dict, threads: int = 0):
        """Marker displacements u [E][P][rows*cols][3] (pad frame: normal, tangent, bitangent)
        and marker depths h [E][P][rows*cols].  pads: pads_per_env, rows, cols, pitch, pad_link
        [E][P], pad_frame [E][P][9], s_d, alpha, lambda_d, c, eps, radius."""
        E = self.n_envs
        keep = {}
        Pd = self._pads(pads, keep)
        I = ORInputs()
        for k, dt in (("link_pose", np.float32), ("link_vel", np.float32), ("obj_pose", np.float32),
                      ("obj_vel", np.float32), ("obj_id", np.int32)):
            keep[k] = np.ascontiguousarray(inputs[k], dt)
            setattr(I, k, _p(keep[k]))
        if inputs.get("env_params") is not None:
            keep["env_params"] = np.ascontiguousarray(inputs["env_params"], np.float32)
            I.env_params = _p(keep["env_params"])
        I.pose_dt = float(inputs.get("pose_dt", 0.0))
        I.step = int(inputs.get("step", 0))
        M = Pd.rows * Pd.cols
        u = np.zeros((E, Pd.pads_per_env, M, 3))
        h = np.zeros((E, Pd.pads_per_env, M))
        lib().or_markers(C.byref(self.S), C.byref(Pd), C.byref(I), _p(u), _p(h), int(threads))
        return u, h

    def pc_prox(self, clouds, inputs: dict, radius: float, k: float, ks: float, density: float, threads: int = 0):
        """Point-cloud ProximityTaxel: link-frame force/torque [6][T] of every taxel
        from each object's tracked points clouds[o] ([n_o][3], object frame)."""
        keep = {"cloud": np.ascontiguousarray(np.concatenate([np.asarray(c, np.float32).reshape(-1, 3)
                                                              for c in clouds]), np.float32),
                "off": np.ascontiguousarray(np.concatenate([[0], np.cumsum([len(c) for c in clouds])]), np.int64)}
        Pc = ORPcProx()
        Pc.cloud, Pc.cloud_off = _p(keep["cloud"]), _p(keep["off"])
        Pc.radius, Pc.k, Pc.ks, Pc.density = float(radius), float(k), float(ks), float(density)
        I = ORInputs()
        for kk, dt in (("link_pose", np.float32), ("link_vel", np.float32), ("obj_pose", np.float32),
                       ("obj_vel", np.float32), ("obj_id", np.int32)):
            keep[kk] = np.ascontiguousarray(inputs[kk], dt)
            setattr(I, kk, _p(keep[kk]))
        if inputs.get("env_params") is not None:
            keep["env_params"] = np.ascontiguousarray(inputs["env_params"], np.float32)
            I.env_params = _p(keep["env_params"])
        I.pose_dt = float(inputs.get("pose_dt", 0.0))
        I.step = int(inputs.get("step", 0))
        T = self.T
        ft = np.zeros((6, T))
        lib().or_pc_prox(C.byref(self.S), C.byref(Pc), C.byref(I), _p(ft), int(threads))
        return ft


def raycast_depth(verts, faces, scale: float, q, u, R):
    """Raycast depth backend at probes q [n][3] (mesh frame) with sensing
    directions u [n][3] and radii R [n]: (depth [n], normal [n][3], face [n],
    ray_pen [n]) -- see or_raycast_depth."""
    V = np.ascontiguousarray(verts, np.float32)
    F = np.ascontiguousarray(faces, np.int32)
    q = np.ascontiguousarray(q, np.float64).reshape(-1, 3)
    u = np.ascontiguousarray(u, np.float64).reshape(-1, 3)
    R = np.broadcast_to(np.asarray(R, np.float64), (len(q),))
    n = len(q)
    depth, normal = np.zeros(n), np.zeros((n, 3))
    face, ray = np.zeros(n, np.int32), np.zeros(n)
    L = lib()
    for i in range(n):
        nn = np.zeros(3)
        f, rp = C.c_int32(), C.c_double()
        depth[i] = L.or_raycast_depth(_p(V), _p(F), len(F), float(scale), _p(np.ascontiguousarray(q[i])),
                                      _p(np.ascontiguousarray(u[i])), float(R[i]), _p(nn), C.byref(f), C.byref(rp))
        normal[i], face[i], ray[i] = nn, f.value, rp.value
    return depth, normal, face, ray
