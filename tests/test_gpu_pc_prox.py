"""The point-cloud ProximityTaxel on the GPU against the oracle's brute force
(Appendix A "ProximityTaxel"): every taxel's link-frame force and torque from
the tracked surface points within its sensing sphere."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2606_22332_gb300 import workload as W
from _scenes import bake_objects_oracle, oracle_scene

PC = {"pc_radius": 0.01, "pc_k": 300.0, "pc_ks": 10.0, "pc_density": 100.0}


@pytest.fixture(scope="module")
def tg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_22332_gb300.tg as tg
    return tg


def _check(tg, wl, steps=2, dr=None):
    wl.params = dict(wl.params, **PC)
    if dr:
        wl.params["dr"] = dr
    sc = tg.Scene.from_workload(wl, sensors=tg.TG_SENSOR_PCPROX)
    sc.upload_objects(wl.objects)
    osc = oracle_scene(wl)
    ost = osc.new_state()
    osc.reset(ost, 0)
    clouds = [o.cloud if o.cloud is not None else np.zeros((0, 3), np.float32) for o in wl.objects]
    worst = 0.0
    for s in range(steps):
        inp = wl.inputs(s)
        sc.step(inp)
        g = sc.read(tg.CH_PC_FT).astype(np.float64)
        sc.sync()
        osc.step(ost, inp)
        o = osc.pc_prox(clouds, inp, PC["pc_radius"], PC["pc_k"], PC["pc_ks"], PC["pc_density"])
        for rows in (slice(0, 3), slice(3, 6)):
            ref = np.abs(o[rows]).max()
            err = np.abs(g[rows] - o[rows]).max()
            assert err <= 2e-4 * ref + 1e-7, (s, rows, err, ref)
            worst = max(worst, err / max(ref, 1e-30))
        assert (np.linalg.norm(o[:3], axis=0) > 0).mean() > 0.05  # the sensor sees the object
    sc.close()
    return worst


def test_config0_sphere_and_mesh_moving(tg):
    wl = W.add_clouds(W.config0(seed=41, n_envs=10), n=3000)
    print("config0 worst relative error", _check(tg, wl))


def test_grid_objects_with_domain_randomised_scale(tg):
    wl = W.config1(n_envs=12, n_objects=3, n_grid=24, steps=3)
    wl.objects = bake_objects_oracle(wl.objects)
    wl = W.add_clouds(wl, n=5000)
    print("grid worst relative error", _check(tg, wl, dr={"mu": (0.4, 1.2), "k": (5e3, 2e4), "scale": (0.8, 1.2)}))


def test_object_without_a_cloud_reads_zero(tg):
    wl = W.add_clouds(W.config0(seed=42, n_envs=4), n=1000)
    wl.objects[0].cloud = None
    wl.params = dict(wl.params, **PC)
    sc = tg.Scene.from_workload(wl, sensors=tg.TG_SENSOR_PCPROX)
    sc.upload_objects(wl.objects)
    sc.step(wl.inputs(0))
    g = sc.read(tg.CH_PC_FT)
    sc.sync()
    env_obj = np.repeat(wl.obj_id, np.diff(wl.taxel_offsets))
    assert np.all(g[:, env_obj == 0] == 0.0)
    sc.close()


def test_sensor_parameters_are_checked(tg):
    wl = W.config0(seed=43, n_envs=2)
    for bad in ({"pc_radius": 0.0}, {"pc_radius": 0.2}, {"pc_density": -1.0}, {"pc_k": float("inf")}):
        wl.params = dict(W.config0(seed=43, n_envs=2).params, **dict(PC, **bad))
        with pytest.raises(tg.TGError):
            tg.Scene.from_workload(wl, sensors=tg.TG_SENSOR_PCPROX)
