"""Batching and launch through the C-ABI: per-step domain randomisation,
work schedules, CUDA-graph replay and the autotuner, each against the FP64
oracle (or, where results must not depend on the choice, bit for bit
against the other choice).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2606_22332_gb300 import workload as W
from _compare import compare_step, gpu_outputs
from _scenes import bake_objects_oracle, oracle_scene

DR = {"mu": (0.4, 1.2), "k": (5e3, 2e4), "scale": (0.8, 1.2)}


@pytest.fixture(scope="module")
def tg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_22332_gb300.tg as tg
    return tg


def _grid_workload(n_envs=20, steps=4):
    wl = W.config1(n_envs=n_envs, n_objects=4, n_grid=24, steps=steps)
    wl.objects = bake_objects_oracle(wl.objects)
    return wl


def _uneven_workload(n_envs=14, steps=3):
    """Uneven envs (200-1,000 taxels over 10-20 links, lattices padded with
    fillers) on FP16 grids: items of several lattices, ragged lengths."""
    rng = np.random.default_rng(31)
    objs = bake_objects_oracle(W.config1_objects(rng, 3, n_grid=24, fp16=True, faces=(800, 1200)))
    lat = W.uneven_lattices(rng, n_envs)
    return W._assemble("uneven", rng, objs, rng.integers(0, 3, n_envs), lat, W.default_params(77), steps=steps,
                       max_links=20, arc=W.PAD_ARC)


def _device_inputs(wl, step):
    inp = wl.inputs(step)
    out = dict(pose_dt=inp["pose_dt"], step=inp["step"])
    for k in ("link_pose", "link_vel", "obj_pose", "obj_vel", "obj_id"):
        out[k] = torch.from_numpy(np.ascontiguousarray(inp[k])).cuda()
    return out


def _all_channels(tg, sc):
    chans = [tg.CH_STATE_FLAGS, tg.CH_DEPTH, tg.CH_FORCE_TORQUE, tg.CH_LINK_WRENCH, tg.CH_LINK_COUNT]
    out = []
    for ch in chans:
        for noisy in ((False, True) if ch in (tg.CH_DEPTH, tg.CH_FORCE_TORQUE) else (False,)):
            out.append(sc.read(ch, noisy).copy())
    sc.sync()
    return out


def test_domain_randomisation_matches_oracle(tg):
    for wl in (W.config0(n_envs=16), _grid_workload(12, 3)):
        wl.params = dict(wl.params, dr=DR)
        sc = tg.Scene.from_workload(wl, sensors=tg.TG_SENSOR_DIST)
        sc.upload_objects(wl.objects)
        osc = oracle_scene(wl)
        ost = osc.new_state(); osc.reset(ost, 0)
        for s in range(3):
            inp = wl.inputs(s)
            sc.step(inp)
            g = gpu_outputs(sc)
            sc.sync()
            o = osc.step(ost, inp)
            compare_step(g, o, ost, wl.params, wl, where=f"{wl.name} dr step {s}")
        sc.close()


def test_env_params_with_domain_randomisation_is_rejected(tg):
    wl = W.config0(n_envs=2)
    wl.params = dict(wl.params, dr=DR)
    sc = tg.Scene.from_workload(wl)
    sc.upload_objects(wl.objects)
    inp = wl.inputs(0)
    inp["env_params"] = np.tile(np.array([[0.8, 1e4, 1.0]], np.float32), (2, 1))
    with pytest.raises(tg.TGError):
        sc.step(inp)
    sc.close()


SCHEDULES = ("grid", "persistent", "pipe1024", "pipe768", "pipe512", "grid384", "persistent384")


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("sorted_", [1, 0])
@pytest.mark.parametrize("uneven", [0, 1])
def test_schedules_give_identical_results(tg, schedule, sorted_, uneven):
    """Every schedule and item order gives the grid schedule's outputs bit for
    bit, with the surface-distance output on: envs of one lattice (1,000
    taxels, 20 links) and uneven envs (items of several lattices, fillers)."""
    wl = _uneven_workload() if uneven else _grid_workload(30, 3)
    ref = tg.Scene.from_workload(wl, sensors=tg.TG_SENSOR_DIST)
    ref.upload_objects(wl.objects)
    ref.set_schedule("grid", sorted=True)
    sc = tg.Scene.from_workload(wl, sensors=tg.TG_SENSOR_DIST)
    sc.upload_objects(wl.objects)
    sc.set_schedule(schedule, sorted=bool(sorted_))
    assert sc.schedule() == {"schedule": schedule, "sorted": sorted_}
    for s in range(3):
        ref.step(wl.inputs(s))
        sc.step(wl.inputs(s))
        for a, b in zip(_all_channels(tg, ref), _all_channels(tg, sc)):
            assert np.array_equal(a.view(np.uint8), b.view(np.uint8))
        ref.sync(); sc.sync()
    ref.close(); sc.close()


@pytest.mark.parametrize("schedule", ["grid", "persistent", "pipe1024", "grid384"])
def test_graph_replay_matches_oracle_and_seek(tg, schedule):
    wl = _grid_workload(16, 6)
    sc = tg.Scene.from_workload(wl, sensors=tg.TG_SENSOR_DIST)
    sc.upload_objects(wl.objects)
    sc.set_schedule(schedule, sorted=True)
    dev = _device_inputs(wl, 0)
    sc.graph_capture(dev, pose_dt_per_step=wl.params["dt"])
    osc = oracle_scene(wl)
    ost = osc.new_state(); osc.reset(ost, 0)
    for s in range(3):
        sc.graph_launch(1)
        g = gpu_outputs(sc)
        sc.sync()
        o = osc.step(ost, wl.inputs(s))
        compare_step(g, o, ost, wl.params, wl, where=f"graph replay {s}")
    # seek: the next replay runs step 9 with pose_dt = 9 dt
    sc.graph_seek(9, 9 * wl.params["dt"], wl.params["dt"])
    sc.graph_launch(2)
    o = osc.step(ost, wl.inputs(9))
    o = osc.step(ost, wl.inputs(10))
    g = gpu_outputs(sc)
    sc.sync()
    compare_step(g, o, ost, wl.params, wl, where="graph after seek")
    with pytest.raises(tg.TGError):
        sc.set_schedule("grid")  # fixed while a graph is held
    sc.graph_release()
    with pytest.raises(tg.TGError):
        sc.graph_launch(1)
    sc.close()


def test_graph_capture_rejects_host_inputs(tg):
    wl = _grid_workload(4, 1)
    sc = tg.Scene.from_workload(wl)
    sc.upload_objects(wl.objects)
    with pytest.raises(tg.TGError):
        sc.graph_capture(wl.inputs(0), pose_dt_per_step=wl.params["dt"])
    sc.close()


def test_autotune_restores_state_and_keeps_parity(tg):
    wl = _grid_workload(24, 6)
    sc = tg.Scene.from_workload(wl, sensors=tg.TG_SENSOR_DIST)
    sc.upload_objects(wl.objects)
    osc = oracle_scene(wl)
    ost = osc.new_state(); osc.reset(ost, 0)
    for s in range(2):
        sc.step(wl.inputs(s))
        osc.step(ost, wl.inputs(s))
    before = sc.save_state()
    rep = sc.autotune(wl.inputs(2), steps=2)
    assert len(rep["candidates"]) == 2 * len(SCHEDULES)
    assert {c["schedule"] for c in rep["candidates"]} == set(SCHEDULES)
    assert all(c["ms_per_step"] > 0 for c in rep["candidates"])
    assert sc.save_state() == before
    chosen = sc.schedule()
    assert chosen == {"schedule": rep["chosen"]["schedule"], "sorted": rep["chosen"]["sorted"]}
    for s in range(2, 5):
        sc.step(wl.inputs(s))
        g = gpu_outputs(sc)
        sc.sync()
        o = osc.step(ost, wl.inputs(s))
        compare_step(g, o, ost, wl.params, wl, where=f"after autotune step {s}")
    sc.close()


def test_graph_replays_are_timed_one_by_one(tg):
    wl = _grid_workload(8, 1)
    sc = tg.Scene.from_workload(wl)
    sc.upload_objects(wl.objects)
    sc.profile(True)
    sc.graph_capture(_device_inputs(wl, 0), pose_dt_per_step=wl.params["dt"])
    assert sc.profile_read()[2] == 0  # capturing is not a step
    sc.graph_launch(5)
    pose_ms, step_ms, n = sc.profile_read()
    assert n == 5 and pose_ms > 0 and step_ms > 0
    sc.graph_launch(2)
    assert sc.profile_read()[2] == 2
    sc.graph_release()
    sc.close()


def test_object_sort_beyond_the_cached_item_count_is_bit_identical(tg):
    """90,000 single-link envs: more items than the ordering kernel keeps in
    shared memory (2 bytes each within 160 KB), so it re-reads each item's
    object; the sorted schedule must give the unsorted results bit for bit."""
    wl = W.config1(n_envs=90000, n_links=1, rows=2, cols=4, n_objects=4, n_grid=24, steps=2)
    wl.objects = bake_objects_oracle(wl.objects)
    assert wl.n_envs * 2 + 4 * 4 > 160 * 1024
    outs = []
    for schedule, sorted_ in (("grid", False), ("grid", True), ("pipe1024", True)):
        sc = tg.Scene.from_workload(wl)
        sc.upload_objects(wl.objects)
        sc.set_schedule(schedule, sorted=sorted_)
        for s in range(2):
            sc.step(wl.inputs(s))
        outs.append(_all_channels(tg, sc))
        sc.close()
    assert float((outs[0][1] > 0).mean()) > 0.01  # some taxels penetrate
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            assert np.array_equal(a, b)
