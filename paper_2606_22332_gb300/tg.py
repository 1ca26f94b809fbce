"""Thin Python binding of the C-ABI in include/tg.h (argument marshalling only).

Every step of the sensor pipeline runs in libtg.so's CUDA kernels; this
module builds the C structs, passes raw pointers (numpy arrays for host
memory, torch tensors for device memory) and the current torch stream, and
turns status codes into exceptions.  There is no fallback: if libtg.so is
missing the import of this module fails.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "csrc", "libtg.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
        "(the CUDA library is the only compute path)")

_lib = C.CDLL(LIB_PATH)

# status codes, object kinds, channels, sensors (include/tg.h)
TG_OK = 0
STATUS = {0: "TG_OK", 1: "TG_ERR_INVALID_ARG", 2: "TG_ERR_OOM", 3: "TG_ERR_CUDA", 4: "TG_ERR_STATE",
          5: "TG_ERR_TIMEOUT", 6: "TG_ERR_NUMERIC", 7: "TG_ERR_UNSUPPORTED"}
TG_OBJ_SPHERE, TG_OBJ_BOX, TG_OBJ_PLANE, TG_OBJ_MESH, TG_OBJ_GRID, TG_OBJ_NEURAL = 0, 1, 2, 3, 4, 5
NSDF_TABLE_ENTRIES, NSDF_WEIGHTS = 16 * 65536, 6208
(CH_CONTACT, CH_DEPTH, CH_DIST, CH_FORCE_TORQUE, CH_LINK_WRENCH, CH_LINK_COUNT, CH_STATE_FLAGS, CH_PROX, CH_MARKER,
 CH_PC_FT, CH_SHEAR_ANCHORS) = range(11)
TG_SENSOR_DIST, TG_SENSOR_PROX, TG_SENSOR_MARKERS, TG_SENSOR_PCPROX = 0x1, 0x2, 0x4, 0x8
LINK_REC = 18


class TGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class NoiseGroup(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "gain_lo", "gain_hi", "beta", "tau", "bias", "sigma_white", "sigma_rw", "quant", "stuck_lo", "stuck_hi")]


class Params(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("k", "c", "alpha", "k_t", "k_omega", "mu", "eta_on", "eta_off", "dt",
                                          "p_dead", "chi", "xt_sigma")] + [
        ("seed", C.c_uint64), ("depth", NoiseGroup), ("ft", NoiseGroup), ("prox", NoiseGroup),
        ("prox_rays", C.c_int32), ("prox_range", C.c_double), ("prox_cone", C.c_double),
        ("dr_on", C.c_int32), ("dr_mu", C.c_double * 2), ("dr_k", C.c_double * 2), ("dr_scale", C.c_double * 2),
        ("nsdf_max_err_mm", C.c_double), ("probe_radius_noise", C.c_double),
        ("pc_radius", C.c_double), ("pc_k", C.c_double), ("pc_ks", C.c_double), ("pc_density", C.c_double),
        ("read_delay", C.c_int32), ("read_jitter", C.c_int32), ("depth_backend", C.c_int32)]


class PadDesc(C.Structure):
    _fields_ = [("pads_per_env", C.c_int32), ("rows", C.c_int32), ("cols", C.c_int32), ("pitch", C.c_double),
                ("pad_link", C.c_void_p), ("pad_frame", C.c_void_p),
                ("s_d", C.c_double), ("alpha", C.c_double), ("lambda_d", C.c_double), ("c", C.c_double),
                ("eps", C.c_double), ("radius", C.c_int32), ("shear_points", C.c_int32),
                ("s_s", C.c_double), ("lambda_s", C.c_double), ("eta_enter", C.c_double), ("eta_exit", C.c_double),
                ("thickness", C.c_double)]


class SceneDesc(C.Structure):
    _fields_ = [("n_envs", C.c_int32), ("max_links", C.c_int32), ("taxel_offsets", C.c_void_p),
                ("link_rows", C.c_void_p), ("link_cols", C.c_void_p), ("link_wrap", C.c_void_p),
                ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p),
                ("nx", C.c_void_p), ("ny", C.c_void_p), ("nz", C.c_void_p), ("R", C.c_void_p),
                ("params", Params), ("sensors", C.c_uint32), ("taxel_gid0", C.c_int64), ("env_gid0", C.c_int32),
                ("pads", PadDesc)]


class ObjectDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("radius", C.c_float), ("half", C.c_float * 3),
                ("n_verts", C.c_int32), ("n_faces", C.c_int32), ("verts", C.c_void_p), ("faces", C.c_void_p),
                ("dims", C.c_int32 * 3), ("lo", C.c_float * 3), ("hi", C.c_float * 3),
                ("fp16", C.c_int32), ("values", C.c_void_p), ("nsdf", C.c_void_p), ("nsdf_err_mm", C.c_double),
                ("cloud", C.c_void_p), ("n_cloud", C.c_int64)]


class TempDesc(C.Structure):
    _fields_ = [("n_grids", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("voxel", C.c_void_p), ("material", C.c_void_p), ("k2_floor", C.c_double)]


class TempInputs(C.Structure):
    _fields_ = [("dt", C.c_double), ("t_amb", C.c_double), ("source", C.c_void_p), ("n_contacts", C.c_int32),
                ("contact_offsets", C.c_void_p), ("contact_cell", C.c_void_p), ("contact_temp", C.c_void_p),
                ("contact_k", C.c_void_p), ("contact_area", C.c_void_p)]


class StepInputs(C.Structure):
    _fields_ = [("link_pose", C.c_void_p), ("link_vel", C.c_void_p), ("obj_pose", C.c_void_p),
                ("obj_vel", C.c_void_p), ("obj_id", C.c_void_p), ("env_params", C.c_void_p),
                ("pose_dt", C.c_double), ("step", C.c_uint32)]


class TuneCandidate(C.Structure):
    _fields_ = [("schedule", C.c_int32), ("sorted", C.c_int32), ("ms_per_step", C.c_double),
                ("kernel", C.c_int32), ("threads", C.c_int32)]


class TuneReport(C.Structure):
    _fields_ = [("n", C.c_int32), ("chosen", C.c_int32), ("sensor_chosen", C.c_int32 * 3),
                ("cand", TuneCandidate * 32)]


# step-kernel schedules (tg_schedule), by name
SCHEDULES = ("grid", "persistent", "pipe1024", "pipe768", "pipe512", "grid384", "persistent384")
# sensor kernels with a tuned launch shape (tg_sensor_kernel), by name
SENSOR_KERNELS = ("prox", "pc_prox", "markers")
SENSOR_THREADS = (128, 256, 512)


_vp, _i32, _sz = C.c_void_p, C.c_int32, C.c_size_t
_lib.tg_create_scene.argtypes = [C.POINTER(SceneDesc), C.POINTER(_vp)]
_lib.tg_destroy_scene.argtypes = [_vp]
_lib.tg_destroy_scene.restype = None
_lib.tg_max_link_taxels.restype = C.c_int32
_lib.tg_upload_objects.argtypes = [_vp, C.POINTER(ObjectDesc), _i32]
_lib.tg_reset_envs.argtypes = [_vp, _vp, C.c_uint32, _vp]
_lib.tg_step_sensors.argtypes = [_vp, C.POINTER(StepInputs), _vp]
_lib.tg_read_taxels.argtypes = [_vp, _i32, _i32, _vp, _sz, _vp]
_lib.tg_channel_bytes.argtypes = [_vp, _i32]
_lib.tg_channel_bytes.restype = _sz
_lib.tg_get_buffer.argtypes = [_vp, _i32, _i32, C.POINTER(_vp), C.POINTER(_sz)]
_lib.tg_sync.argtypes = [_vp, _vp]
_lib.tg_last_error.argtypes = [_vp]
_lib.tg_last_error.restype = C.c_char_p
_lib.tg_save_state.argtypes = [_vp, _vp, C.POINTER(_sz)]
_lib.tg_load_state.argtypes = [_vp, _vp, _sz]
_lib.tg_profile_enable.argtypes = [_vp, _i32]
_lib.tg_profile_read.argtypes = [_vp, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int64)]
_lib.tg_bake_grid.argtypes = [_vp, _i32, _vp, _i32, _vp, _vp, _vp, _i32, _vp, _vp]
_lib.tg_mesh_sdf.argtypes = [_vp, _i32, _vp, _i32, _vp, C.c_int64, _vp, _vp, _vp]
_lib.tg_mesh_sdf_noalloc.argtypes = [_vp, _i32, _vp, _i32, _vp, C.c_int64, _vp, _vp, _vp]
_lib.tg_graph_capture.argtypes = [_vp, C.POINTER(StepInputs), C.c_double, _vp]
_lib.tg_graph_launch.argtypes = [_vp, _i32, _vp]
_lib.tg_graph_seek.argtypes = [_vp, C.c_uint32, C.c_double, C.c_double, _vp]
_lib.tg_graph_release.argtypes = [_vp]
_lib.tg_set_schedule.argtypes = [_vp, _i32, _i32]
_lib.tg_get_schedule.argtypes = [_vp, C.POINTER(_i32), C.POINTER(_i32)]
_lib.tg_set_sensor_threads.argtypes = [_vp, _i32, _i32]
_lib.tg_get_sensor_threads.argtypes = [_vp, _i32, C.POINTER(_i32)]
_lib.tg_autotune.argtypes = [_vp, C.POINTER(StepInputs), _i32, C.POINTER(TuneReport), _vp]
_lib.tg_object_info.argtypes = [_vp, _i32, C.POINTER(_i32), C.POINTER(C.c_double)]
_lib.tg_nsdf_create.argtypes = [_vp, _vp, C.c_uint64, C.POINTER(_vp)]
_lib.tg_nsdf_destroy.argtypes = [_vp]
_lib.tg_nsdf_destroy.restype = None
_lib.tg_nsdf_set_params.argtypes = [_vp, _vp, _vp]
_lib.tg_nsdf_get_params.argtypes = [_vp, _vp, _vp]
_lib.tg_nsdf_eval.argtypes = [_vp, _vp, C.c_int64, _vp, _vp, _vp]
_lib.tg_nsdf_loss_grad.argtypes = [_vp, _vp, _vp, C.c_int64, C.POINTER(C.c_double), _vp, _vp, _vp]
_lib.tg_nsdf_train.argtypes = [_vp, _vp, _vp, C.c_int64, _i32, _i32, C.c_double, C.c_double, C.c_uint64, _vp, _vp]
_lib.tg_nsdf_probe.argtypes = [_vp, _vp, _i32, _vp, _i32, _vp, C.c_int64, C.POINTER(C.c_double),
                               C.POINTER(C.c_double), _vp]
_lib.tg_nsdf_last_error.restype = C.c_char_p
_lib.tg_temp_create.argtypes = [C.POINTER(TempDesc), C.POINTER(_vp)]
_lib.tg_temp_destroy.argtypes = [_vp]
_lib.tg_temp_destroy.restype = None
_lib.tg_temp_reset.argtypes = [_vp, _vp, _vp]
_lib.tg_temp_set.argtypes = [_vp, _vp, _vp, _vp]
_lib.tg_temp_step.argtypes = [_vp, C.POINTER(TempInputs), _vp]
_lib.tg_temp_read.argtypes = [_vp, _i32, _vp, _sz, _vp]
_lib.tg_temp_buffer.argtypes = [_vp, _i32, C.POINTER(_vp)]
_lib.tg_contact_area.argtypes = [_vp, _vp, _vp, _i32, _i32, C.c_double, _vp, _vp]
_lib.tg_temp_last_error.restype = C.c_char_p
_lib.tg_mesh_bvh_create.argtypes = [_vp, _i32, _vp, _i32, C.POINTER(_vp)]
_lib.tg_mesh_bvh_destroy.argtypes = [_vp]
_lib.tg_mesh_bvh_destroy.restype = None
_lib.tg_raycast_depth.argtypes = [_vp, _vp, _vp, C.c_int64, C.c_double, _vp, _vp, _vp, _vp]
_lib.tg_mesh_bvh_last_error.restype = C.c_char_p
for _f in ("tg_create_scene", "tg_upload_objects", "tg_reset_envs", "tg_step_sensors", "tg_read_taxels",
           "tg_get_buffer", "tg_sync", "tg_save_state", "tg_load_state", "tg_bake_grid", "tg_mesh_sdf",
           "tg_profile_enable", "tg_profile_read", "tg_mesh_sdf_noalloc", "tg_graph_capture", "tg_graph_launch",
           "tg_graph_seek", "tg_graph_release", "tg_set_schedule", "tg_get_schedule", "tg_autotune", "tg_object_info",
           "tg_set_sensor_threads", "tg_get_sensor_threads", "tg_nsdf_create", "tg_nsdf_set_params",
           "tg_nsdf_get_params", "tg_nsdf_eval", "tg_nsdf_loss_grad",
           "tg_nsdf_train", "tg_nsdf_probe", "tg_temp_create", "tg_temp_reset", "tg_temp_set", "tg_temp_step",
           "tg_temp_read", "tg_temp_buffer", "tg_contact_area", "tg_mesh_bvh_create", "tg_raycast_depth"):
    getattr(_lib, _f).restype = C.c_int

EXPORTED = ["tg_create_scene", "tg_destroy_scene", "tg_max_link_taxels", "tg_upload_objects", "tg_reset_envs",
            "tg_step_sensors", "tg_read_taxels", "tg_channel_bytes", "tg_get_buffer", "tg_sync", "tg_last_error",
            "tg_save_state", "tg_load_state", "tg_bake_grid", "tg_mesh_sdf", "tg_profile_enable", "tg_profile_read",
            "tg_mesh_sdf_noalloc", "tg_graph_capture", "tg_graph_launch", "tg_graph_seek", "tg_graph_release",
            "tg_set_schedule", "tg_get_schedule", "tg_set_sensor_threads", "tg_get_sensor_threads", "tg_autotune",
            "tg_object_info", "tg_nsdf_create",
            "tg_nsdf_destroy", "tg_nsdf_set_params", "tg_nsdf_get_params", "tg_nsdf_eval", "tg_nsdf_loss_grad",
            "tg_nsdf_train", "tg_nsdf_probe", "tg_nsdf_last_error", "tg_temp_create", "tg_temp_destroy",
            "tg_temp_reset", "tg_temp_set", "tg_temp_step", "tg_temp_read", "tg_temp_buffer", "tg_contact_area",
            "tg_temp_last_error", "tg_mesh_bvh_create", "tg_mesh_bvh_destroy", "tg_raycast_depth",
            "tg_mesh_bvh_last_error"]
NOALLOC_MAX_FACES = 65536


def lib():
    return _lib


def _check(status, scene_handle=None):
    if status != TG_OK:
        msg = _lib.tg_last_error(scene_handle)
        raise TGError(status, msg.decode() if msg else "")


def _ptr(a):
    """Raw pointer of a numpy array (host) or a torch tensor (host or device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"], "arrays must be C-contiguous"
        return a.ctypes.data
    assert a.is_contiguous(), "tensors must be contiguous"
    return a.data_ptr()


def _stream(stream):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    import torch

    if torch.cuda.is_available() and torch.cuda.is_initialized():
        return torch.cuda.current_stream().cuda_stream
    return None


def _fill_params(params: dict) -> Params:
    P = Params()
    for k in ("k", "c", "alpha", "k_t", "k_omega", "eta_on", "eta_off", "dt", "p_dead", "chi", "xt_sigma"):
        setattr(P, k, float(params[k]))
    mu = params["mu"]
    P.mu = -1.0 if mu is None or np.isinf(mu) else float(mu)
    P.seed = int(params["seed"])
    P.prox_rays = int(params.get("prox_rays", 0))
    P.prox_range = float(params.get("prox_range", 0.05))
    P.prox_cone = float(params.get("prox_cone", np.radians(30.0)))
    dr = params.get("dr")
    P.dr_on = 1 if dr else 0
    if dr:
        for k in ("mu", "k", "scale"):
            getattr(P, "dr_" + k)[0] = float(dr[k][0])
            getattr(P, "dr_" + k)[1] = float(dr[k][1])
    P.nsdf_max_err_mm = float(params.get("nsdf_max_err_mm", 0.2))
    P.probe_radius_noise = float(params.get("rho", 0.0))
    # point-cloud ProximityTaxel (the paper's experiment values by default)
    P.pc_radius = float(params.get("pc_radius", 0.01))
    P.pc_k = float(params.get("pc_k", 300.0))
    P.pc_ks = float(params.get("pc_ks", 10.0))
    P.pc_density = float(params.get("pc_density", 100.0))
    P.read_delay = int(params.get("read_delay", 0))
    P.read_jitter = int(params.get("read_jitter", 0))
    P.depth_backend = {"sdf": 0, "raycast": 1}[params.get("depth_backend", "sdf")]
    for g in ("depth", "ft", "prox"):
        grp = getattr(P, g)
        for k in NoiseGroup._fields_:
            setattr(grp, k[0], float(params["noise"][g][k[0]]))
    return P


class _CudaView:
    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def object_desc(o, keep: list) -> ObjectDesc:
    """tg_object_desc of a workload ObjectSpec (arrays kept alive in `keep`)."""
    d = ObjectDesc()
    kind = {"sphere": TG_OBJ_SPHERE, "box": TG_OBJ_BOX, "plane": TG_OBJ_PLANE, "mesh": TG_OBJ_MESH,
            "grid": TG_OBJ_GRID, "neural": TG_OBJ_NEURAL}[o.kind]
    d.kind = kind
    d.radius = float(o.radius)
    d.half[:] = [float(h) for h in o.half]
    if kind == TG_OBJ_MESH:
        V = np.ascontiguousarray(o.verts, np.float32); F = np.ascontiguousarray(o.faces, np.int32)
        keep += [V, F]
        d.n_verts, d.n_faces = len(V), len(F)
        d.verts, d.faces = _ptr(V), _ptr(F)
    if kind == TG_OBJ_NEURAL:
        net = o.net if isinstance(o.net, Nsdf) else Nsdf.from_params(o.nsdf_lo, o.nsdf_hi, o.nsdf_table,
                                                                     o.nsdf_weights)
        keep.append(net)
        d.nsdf = net.h
        d.nsdf_err_mm = float(o.nsdf_err_mm)
    if kind in (TG_OBJ_GRID, TG_OBJ_NEURAL):
        vals = o.values
        if isinstance(vals, np.ndarray):
            vals = np.ascontiguousarray(vals, np.uint16 if o.fp16 else np.float32)
        keep.append(vals)
        d.dims[:] = [int(v) for v in o.dims]
        d.lo[:] = [float(v) for v in o.lo]
        d.hi[:] = [float(v) for v in o.hi]
        d.fp16 = 1 if o.fp16 else 0
        d.values = _ptr(vals)
    cloud = getattr(o, "cloud", None)
    if cloud is not None and len(cloud):
        c = np.ascontiguousarray(cloud, np.float32).reshape(-1, 3)
        keep.append(c)
        d.cloud, d.n_cloud = _ptr(c), len(c)
    return d


class Scene:
    """A tg_scene: the taxel geometry, state and outputs of E envs."""

    def __init__(self, geom: dict, params: dict, sensors: int = 0, taxel_gid0: int = 0, env_gid0: int = 0,
                 pads: dict | None = None):
        keep = {}
        off = np.ascontiguousarray(geom["taxel_offsets"], np.int64)
        E = len(off) - 1
        rows = np.ascontiguousarray(geom["link_rows"], np.int32)
        L = len(rows) // E
        keep["off"] = off
        keep["rows"] = rows
        keep["cols"] = np.ascontiguousarray(geom["link_cols"], np.int32)
        keep["wrap"] = np.ascontiguousarray(geom["link_wrap"], np.uint8)
        d = SceneDesc()
        d.n_envs, d.max_links = E, L
        d.taxel_offsets, d.link_rows = _ptr(off), _ptr(rows)
        d.link_cols, d.link_wrap = _ptr(keep["cols"]), _ptr(keep["wrap"])
        for k in ("x", "y", "z", "nx", "ny", "nz", "R"):
            a = geom[k]
            if isinstance(a, np.ndarray):
                a = np.ascontiguousarray(a, np.float32)
            keep[k] = a
            setattr(d, k, _ptr(a))
        d.params = _fill_params(params)
        d.sensors = sensors
        d.taxel_gid0 = int(taxel_gid0)
        d.env_gid0 = int(env_gid0)
        self.pads = pads
        if pads is not None:
            keep["pad_link"] = np.ascontiguousarray(pads["pad_link"], np.int32)
            keep["pad_frame"] = np.ascontiguousarray(pads["pad_frame"], np.float32)
            pd = d.pads
            pd.pads_per_env, pd.rows, pd.cols = int(pads["pads_per_env"]), int(pads["rows"]), int(pads["cols"])
            pd.pitch = float(pads["pitch"])
            pd.pad_link, pd.pad_frame = _ptr(keep["pad_link"]), _ptr(keep["pad_frame"])
            for k in ("s_d", "alpha", "lambda_d", "c", "eps"):
                setattr(pd, k, float(pads[k]))
            pd.radius = int(pads["radius"])
            # shear anchors: on when pads carries shear_points > 0
            pd.shear_points = int(pads.get("shear_points", 0))
            for k, dflt in (("s_s", 100.0), ("lambda_s", 2000.0), ("eta_enter", 1e-5), ("eta_exit", 1e-4),
                            ("thickness", 2e-3)):
                setattr(pd, k, float(pads.get(k, dflt)))
        h = C.c_void_p()
        _check(_lib.tg_create_scene(C.byref(d), C.byref(h)), None)
        self.h = h
        self.n_envs, self.max_links, self.n_taxels = E, L, int(off[-1])
        self.sensors = sensors
        self._keep_inputs = None

    @classmethod
    def from_workload(cls, wl, sensors: int = 0):
        if wl.params.get("prox_rays", 0) > 0:
            sensors |= TG_SENSOR_PROX
        if wl.pads is not None:
            sensors |= TG_SENSOR_MARKERS
        return cls(wl.geom(), wl.params, sensors=sensors, pads=wl.pads)

    def close(self):
        if getattr(self, "h", None):
            _lib.tg_destroy_scene(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def upload_objects(self, objects):
        keep = []
        arr = (ObjectDesc * len(objects))(*[object_desc(o, keep) for o in objects])
        _check(_lib.tg_upload_objects(self.h, arr, len(objects)), self.h)

    def reset(self, episode: int, env_mask=None, stream=None):
        _check(_lib.tg_reset_envs(self.h, _ptr(env_mask), int(episode), _stream(stream)), self.h)

    def _inputs(self, inputs: dict):
        I = StepInputs()
        keep = {}
        for k, dt in (("link_pose", np.float32), ("link_vel", np.float32), ("obj_pose", np.float32),
                      ("obj_vel", np.float32), ("obj_id", np.int32), ("env_params", np.float32)):
            a = inputs.get(k)
            if a is None:
                continue
            if isinstance(a, np.ndarray):
                a = np.ascontiguousarray(a, dt)
            keep[k] = a
            setattr(I, k, _ptr(a))
        I.pose_dt = float(inputs.get("pose_dt", 0.0))
        I.step = int(inputs.get("step", 0))
        return I, keep

    def step(self, inputs: dict, stream=None):
        """inputs: link_pose, link_vel, obj_pose, obj_vel, obj_id, optional env_params (numpy = host,
        torch = host or device), pose_dt (s), step (RNG counter)."""
        I, keep = self._inputs(inputs)
        self._keep_inputs = keep  # host sources must outlive the async copies
        _check(_lib.tg_step_sensors(self.h, C.byref(I), _stream(stream)), self.h)

    def graph_capture(self, inputs: dict, pose_dt_per_step: float, stream=None):
        """Capture one step into a CUDA graph; inputs must be device tensors that stay in place."""
        I, keep = self._inputs(inputs)
        self._graph_inputs = keep
        _check(_lib.tg_graph_capture(self.h, C.byref(I), float(pose_dt_per_step), _stream(stream)), self.h)

    def graph_launch(self, n_steps: int = 1, stream=None):
        _check(_lib.tg_graph_launch(self.h, int(n_steps), _stream(stream)), self.h)

    def graph_seek(self, step: int, pose_dt: float, pose_dt_per_step: float, stream=None):
        _check(_lib.tg_graph_seek(self.h, int(step), float(pose_dt), float(pose_dt_per_step), _stream(stream)),
               self.h)

    def graph_release(self):
        _check(_lib.tg_graph_release(self.h), self.h)
        self._graph_inputs = None

    def object_info(self, i: int):
        """(kind in use, probe error mm) of uploaded object i."""
        k, e = _i32(), C.c_double()
        _check(_lib.tg_object_info(self.h, int(i), C.byref(k), C.byref(e)), self.h)
        return int(k.value), float(e.value)

    def set_schedule(self, schedule="grid", sorted: bool = True):
        """schedule: a name of SCHEDULES or its index."""
        k = SCHEDULES.index(schedule) if isinstance(schedule, str) else int(schedule)
        _check(_lib.tg_set_schedule(self.h, k, int(bool(sorted))), self.h)

    def schedule(self):
        p, s = _i32(), _i32()
        _check(_lib.tg_get_schedule(self.h, C.byref(p), C.byref(s)), self.h)
        return {"schedule": SCHEDULES[int(p.value)], "sorted": int(s.value)}

    def set_sensor_threads(self, kernel, threads: int):
        """Threads per CTA (128, 256 or 512) of a sensor kernel (a name of SENSOR_KERNELS or its index)."""
        k = SENSOR_KERNELS.index(kernel) if isinstance(kernel, str) else int(kernel)
        _check(_lib.tg_set_sensor_threads(self.h, k, int(threads)), self.h)

    def sensor_threads(self):
        out = {}
        for k, name in enumerate(SENSOR_KERNELS):
            t = _i32()
            _check(_lib.tg_get_sensor_threads(self.h, k, C.byref(t)), self.h)
            out[name] = int(t.value)
        return out

    def autotune(self, inputs: dict, steps: int = 3, stream=None):
        """Time every step schedule on these inputs and keep the fastest, then
        every launch shape of each sensor kernel the scene runs; returns the
        report as a dict (step candidates under "candidates", the sensor
        kernels' under "sensor_candidates")."""
        I, keep = self._inputs(inputs)
        self._keep_inputs = keep
        R = TuneReport()
        _check(_lib.tg_autotune(self.h, C.byref(I), int(steps), C.byref(R), _stream(stream)), self.h)
        step_c, sensor_c = [], []
        for i in range(R.n):
            c = R.cand[i]
            if c.kernel < 0:
                step_c.append({"schedule": SCHEDULES[c.schedule], "sorted": c.sorted, "threads": c.threads,
                               "ms_per_step": c.ms_per_step})
            else:
                sensor_c.append({"kernel": SENSOR_KERNELS[c.kernel], "threads": c.threads,
                                 "ms_per_step": c.ms_per_step})
        chosen_sensor = {SENSOR_KERNELS[k]: R.cand[R.sensor_chosen[k]].threads
                         for k in range(3) if R.sensor_chosen[k] >= 0}
        return {"candidates": step_c, "chosen": step_c[R.chosen], "sensor_candidates": sensor_c,
                "sensor_chosen": chosen_sensor}

    def channel_bytes(self, ch: int) -> int:
        return int(_lib.tg_channel_bytes(self.h, ch))

    def _shape_dtype(self, ch):
        T, EL = self.n_taxels, self.n_envs * self.max_links
        return {CH_CONTACT: ((T,), np.uint8), CH_DEPTH: ((T,), np.float32), CH_DIST: ((T,), np.float32),
                CH_FORCE_TORQUE: ((6, T), np.float32), CH_LINK_WRENCH: ((EL, LINK_REC), np.float32),
                CH_LINK_COUNT: ((EL, 2), np.int32), CH_STATE_FLAGS: ((T,), np.uint8),
                CH_PROX: ((T,), np.float32),
                CH_MARKER: ((self._n_markers(), 3), np.float32), CH_PC_FT: ((6, T), np.float32),
                CH_SHEAR_ANCHORS: ((self._n_pads(),), np.int32)}[ch]

    def _n_pads(self):
        p = self.pads
        return 0 if p is None else self.n_envs * int(p["pads_per_env"])

    def _n_markers(self):
        p = self.pads
        return 0 if p is None else self.n_envs * int(p["pads_per_env"]) * int(p["rows"]) * int(p["cols"])

    def read(self, ch: int, noisy: bool = False, out=None, stream=None):
        """Copy a channel into `out` (numpy = host, torch tensor = host or device); returns it."""
        shape, dt = self._shape_dtype(ch)
        if out is None:
            out = np.empty(shape, dt)
        # the destination's own size: the library rejects one that does not match the channel
        nbytes = out.nbytes if isinstance(out, np.ndarray) else out.numel() * out.element_size()
        _check(_lib.tg_read_taxels(self.h, ch, int(noisy), _ptr(out), int(nbytes), _stream(stream)), self.h)
        if isinstance(out, np.ndarray):
            self.sync(stream)
        return out

    def buffer(self, ch: int, noisy: bool = False):
        """Zero-copy torch view of a library-owned device buffer."""
        import torch

        p, n = C.c_void_p(), C.c_size_t()
        _check(_lib.tg_get_buffer(self.h, ch, int(noisy), C.byref(p), C.byref(n)), self.h)
        shape, dt = self._shape_dtype(ch)
        typestr = {np.float32: "<f4", np.int32: "<i4", np.uint8: "|u1"}[dt]
        return torch.as_tensor(_CudaView(p.value, shape, typestr), device="cuda")

    def sync(self, stream=None):
        _check(_lib.tg_sync(self.h, _stream(stream)), self.h)

    def profile(self, on: bool = True):
        _check(_lib.tg_profile_enable(self.h, int(on)), self.h)

    def profile_read(self):
        """(pose kernel ms, step kernel ms, steps) summed since the last read."""
        a, b, n = C.c_double(), C.c_double(), C.c_int64()
        _check(_lib.tg_profile_read(self.h, C.byref(a), C.byref(b), C.byref(n)), self.h)
        return a.value, b.value, n.value

    def save_state(self) -> bytes:
        n = C.c_size_t()
        _check(_lib.tg_save_state(self.h, None, C.byref(n)), self.h)
        buf = C.create_string_buffer(n.value)
        _check(_lib.tg_save_state(self.h, buf, C.byref(n)), self.h)
        return buf.raw

    def load_state(self, data: bytes):
        buf = C.create_string_buffer(data, len(data))
        _check(_lib.tg_load_state(self.h, buf, len(data)), self.h)


def bake_grid(verts, faces, dims, lo, hi, fp16=False, stream=None):
    """Exact mesh SDF at the grid nodes on the GPU; returns a torch tensor [z][y][x]
    (float32, or int16 holding binary16 bits when fp16)."""
    import torch

    V = np.ascontiguousarray(verts, np.float32); F = np.ascontiguousarray(faces, np.int32)
    d = np.ascontiguousarray(dims, np.int32)
    lo = np.ascontiguousarray(lo, np.float32); hi = np.ascontiguousarray(hi, np.float32)
    out = torch.empty((int(d[2]), int(d[1]), int(d[0])), dtype=torch.float16 if fp16 else torch.float32, device="cuda")
    _check(_lib.tg_bake_grid(_ptr(V), len(V), _ptr(F), len(F), _ptr(d), _ptr(lo), _ptr(hi), int(fp16),
                             out.data_ptr(), _stream(stream)), None)
    return out


def _ncheck(status):
    if status != 0:
        msg = _lib.tg_nsdf_last_error()
        raise TGError(status, msg.decode() if msg else "")


class Nsdf:
    """A learned SDF (tg_nsdf): hash-encoding table and bfloat16 MLP on the device."""

    def __init__(self, lo, hi, seed: int = 0):
        lo = np.ascontiguousarray(lo, np.float32); hi = np.ascontiguousarray(hi, np.float32)
        self.lo, self.hi = lo, hi
        h = _vp()
        _ncheck(_lib.tg_nsdf_create(_ptr(lo), _ptr(hi), int(seed), C.byref(h)))
        self.h = h.value

    @classmethod
    def from_params(cls, lo, hi, table, weights):
        n = cls(lo, hi, 0)
        n.set_params(table, weights)
        return n

    def close(self):
        if getattr(self, "h", None):
            _lib.tg_nsdf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, table, weights):
        t = np.ascontiguousarray(table, np.uint16).reshape(-1)
        w = np.ascontiguousarray(weights, np.uint16).reshape(-1)
        assert t.size == 2 * NSDF_TABLE_ENTRIES and w.size == NSDF_WEIGHTS
        _ncheck(_lib.tg_nsdf_set_params(self.h, _ptr(t), _ptr(w)))

    def params(self):
        """(table uint16 [16][65536][2] binary16 bits, weights uint16 [6208] bfloat16 bits)"""
        t = np.zeros((16, 65536, 2), np.uint16)
        w = np.zeros(NSDF_WEIGHTS, np.uint16)
        _ncheck(_lib.tg_nsdf_get_params(self.h, _ptr(t), _ptr(w)))
        return t, w

    def eval(self, points, grad=False, stream=None):
        import torch

        pts = points.contiguous()
        n = pts.shape[0]
        phi = torch.empty(n, dtype=torch.float32, device=pts.device)
        g = torch.empty((n, 3), dtype=torch.float32, device=pts.device) if grad else None
        _ncheck(_lib.tg_nsdf_eval(self.h, pts.data_ptr(), n, phi.data_ptr(), g.data_ptr() if grad else None,
                                  _stream(stream)))
        return (phi, g) if grad else phi

    def loss_grad(self, points, labels_mm, stream=None):
        import torch

        pts, lab = points.contiguous(), labels_mm.contiguous()
        gw = torch.empty(NSDF_WEIGHTS, dtype=torch.float32, device=pts.device)
        gt = torch.empty((16, 65536, 2), dtype=torch.float32, device=pts.device)
        loss = C.c_double()
        _ncheck(_lib.tg_nsdf_loss_grad(self.h, pts.data_ptr(), lab.data_ptr(), pts.shape[0], C.byref(loss),
                                       gw.data_ptr(), gt.data_ptr(), _stream(stream)))
        return loss.value, gw, gt

    def train(self, points, labels_mm, steps: int, batch: int = 1 << 14, lr0: float = 1e-2, lr_final: float = 1e-3,
              seed: int = 0, record_losses: bool = True, stream=None):
        pts, lab = points.contiguous(), labels_mm.contiguous()
        losses = np.zeros(max(steps, 1), np.float32) if record_losses else None
        _ncheck(_lib.tg_nsdf_train(self.h, pts.data_ptr(), lab.data_ptr(), pts.shape[0], int(steps), int(batch),
                                   float(lr0), float(lr_final), int(seed),
                                   _ptr(losses) if record_losses else None, _stream(stream)))
        return losses[:steps] if record_losses else None

    def probe(self, verts, faces, points, stream=None):
        """(max, mean) |phi_net - phi_mesh| in mm over device probe points."""
        V = np.ascontiguousarray(verts, np.float32); F = np.ascontiguousarray(faces, np.int32)
        pts = points.contiguous()
        mx, mean = C.c_double(), C.c_double()
        _ncheck(_lib.tg_nsdf_probe(self.h, _ptr(V), len(V), _ptr(F), len(F), pts.data_ptr(), pts.shape[0],
                                   C.byref(mx), C.byref(mean), _stream(stream)))
        return mx.value, mean.value


def mesh_sdf(verts, faces, points, with_grad=True, stream=None):
    """Exact mesh SDF (and unit gradient) at device points [n][3]."""
    import torch

    V = np.ascontiguousarray(verts, np.float32); F = np.ascontiguousarray(faces, np.int32)
    pts = points.contiguous()
    n = pts.shape[0]
    phi = torch.empty(n, dtype=torch.float32, device=pts.device)
    grad = torch.empty((n, 3), dtype=torch.float32, device=pts.device) if with_grad else None
    _check(_lib.tg_mesh_sdf(_ptr(V), len(V), _ptr(F), len(F), pts.data_ptr(), n, phi.data_ptr(),
                            grad.data_ptr() if grad is not None else None, _stream(stream)), None)
    return phi, grad


def mesh_sdf_noalloc(verts, faces, points, phi, grad=None, stream=None):
    """tg_mesh_sdf_noalloc: exact mesh SDF at device points into caller-owned
    device tensors, with no device allocation inside the library (for callers
    that cannot allocate).  verts (float32 [nv][3]), faces (int32 [nf][3]),
    points, phi and grad must be contiguous CUDA tensors."""
    _check(_lib.tg_mesh_sdf_noalloc(verts.data_ptr(), verts.shape[0], faces.data_ptr(), faces.shape[0],
                                    points.data_ptr(), points.shape[0], phi.data_ptr(),
                                    grad.data_ptr() if grad is not None else None, _stream(stream)), None)


def _tcheck(status):
    if status != 0:
        msg = _lib.tg_temp_last_error()
        raise TGError(status, msg.decode() if msg else "")


class TempGrid:
    """TemperatureGrid sensors (tg_temp): G grids of nx x ny x nz cells on the device.

    voxel: [G][3] voxel sizes (m); material: [G][7] k, rho, c_p, emissivity, h,
    tau, base temperature.  Fields are [G][nx][ny][nz] float32."""

    def __init__(self, dims, voxel, material, k2_floor: float = 1e-12):
        voxel = np.ascontiguousarray(voxel, np.float32).reshape(-1, 3)
        material = np.ascontiguousarray(material, np.float32).reshape(-1, 7)
        assert len(voxel) == len(material)
        self.G, self.dims = len(voxel), tuple(int(n) for n in dims)
        d = TempDesc()
        d.n_grids = self.G
        d.nx, d.ny, d.nz = self.dims
        d.voxel, d.material, d.k2_floor = _ptr(voxel), _ptr(material), float(k2_floor)
        h = _vp()
        _tcheck(_lib.tg_temp_create(C.byref(d), C.byref(h)))
        self.h = h.value

    def close(self):
        if getattr(self, "h", None):
            _lib.tg_temp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def cells(self):
        return self.dims[0] * self.dims[1] * self.dims[2]

    def reset(self, grid_mask=None, stream=None):
        m = None if grid_mask is None else np.ascontiguousarray(grid_mask, np.uint8)
        _tcheck(_lib.tg_temp_reset(self.h, _ptr(m) if m is not None else None, _stream(stream)))

    def set(self, field, measured=None, stream=None):
        f = np.ascontiguousarray(field, np.float32)
        m = None if measured is None else np.ascontiguousarray(measured, np.float32)
        assert f.size == self.G * self.cells
        _tcheck(_lib.tg_temp_set(self.h, _ptr(f), _ptr(m) if m is not None else None, _stream(stream)))
        self.sync(stream)

    def step(self, dt: float, t_amb: float, source=None, contacts=None, stream=None):
        """source: device tensor [G][cells] (W/m^2) or None.  contacts: None or a
        dict of offsets [G+1], cell [C], temp [C], k [C], area [C] (numpy arrays
        or device tensors)."""
        inp = TempInputs()
        inp.dt, inp.t_amb = float(dt), float(t_amb)
        inp.source = source.data_ptr() if source is not None else None
        keep = []
        if contacts is not None and len(contacts["cell"]) > 0:
            inp.n_contacts = len(contacts["cell"])
            for key, field, dt_ in (("offsets", "contact_offsets", np.int32), ("cell", "contact_cell", np.int32),
                                    ("temp", "contact_temp", np.float32), ("k", "contact_k", np.float32),
                                    ("area", "contact_area", np.float32)):
                v = contacts[key]
                if hasattr(v, "data_ptr"):
                    setattr(inp, field, v.data_ptr())
                else:
                    a = np.ascontiguousarray(v, dt_)
                    keep.append(a)
                    setattr(inp, field, _ptr(a))
        _tcheck(_lib.tg_temp_step(self.h, C.byref(inp), _stream(stream)))

    def read(self, measured: bool = False, stream=None):
        out = np.zeros((self.G,) + self.dims, np.float32)
        _tcheck(_lib.tg_temp_read(self.h, int(measured), _ptr(out), out.nbytes, _stream(stream)))
        self.sync(stream)
        return out

    def buffer(self, measured: bool = False):
        """Device view of T or T_meas as a torch tensor [G][nx][ny][nz] (no copy)."""
        import torch

        p = _vp()
        _tcheck(_lib.tg_temp_buffer(self.h, int(measured), C.byref(p)))
        return torch.as_tensor(_CudaView(p.value, (self.G,) + self.dims, "<f4"), device="cuda")

    def sync(self, stream=None):
        import torch

        torch.cuda.synchronize()


def contact_area(points, n_points, depth, d_w: float = 1.0, stream=None):
    """tg_contact_area on device tensors: points [P][M][3], n_points int32 [P], depth [P]; returns area [P]."""
    import torch

    pts, n, dl = points.contiguous(), n_points.contiguous(), depth.contiguous()
    area = torch.empty(pts.shape[0], dtype=torch.float32, device=pts.device)
    _tcheck(_lib.tg_contact_area(pts.data_ptr(), n.data_ptr(), dl.data_ptr(), pts.shape[0], pts.shape[1],
                                 float(d_w), area.data_ptr(), _stream(stream)))
    return area


def _bcheck(status):
    if status != 0:
        msg = _lib.tg_mesh_bvh_last_error()
        raise TGError(status, msg.decode() if msg else "")


class MeshBvh:
    """tg_mesh_bvh: a bounding volume hierarchy over one triangle mesh, for the raycast depth backend."""

    def __init__(self, verts, faces):
        V = np.ascontiguousarray(verts, np.float32).reshape(-1, 3)
        F = np.ascontiguousarray(faces, np.int32).reshape(-1, 3)
        h = _vp()
        _bcheck(_lib.tg_mesh_bvh_create(_ptr(V), len(V), _ptr(F), len(F), C.byref(h)))
        self.h = h.value

    def close(self):
        if getattr(self, "h", None):
            _lib.tg_mesh_bvh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def depth(self, probes, radius, scale: float = 1.0, stream=None):
        """(depth [n], normal [n][3], face [n]) at device probes [n][3] (mesh frame) with radii [n]."""
        import torch

        q, r = probes.contiguous(), radius.contiguous()
        n = q.shape[0]
        d = torch.empty(n, dtype=torch.float32, device=q.device)
        nn = torch.empty((n, 3), dtype=torch.float32, device=q.device)
        f = torch.empty(n, dtype=torch.int32, device=q.device)
        _bcheck(_lib.tg_raycast_depth(self.h, q.data_ptr(), r.data_ptr(), n, float(scale), d.data_ptr(),
                                      nn.data_ptr(), f.data_ptr(), _stream(stream)))
        return d, nn, f
