"""Read delay with jitter on the GPU against the oracle (paper, "Sensor Noise
Model", base noise: the noisy readout is formed from y_{t - Delta_read}).

A grid workload whose links move every step (so the delayed readout differs
from the current one) runs with a delay of 2 steps and a jitter of 1 step,
through the grid and the pipelined schedules and through graph replays; every
step is compared with the oracle at the usual bounds, including the reported
(delayed) noisy contact bits.  A checkpoint taken mid-run carries the delayed
history: restoring it and stepping again gives the same outputs bit for bit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2606_22332_gb300 import workload as W
from _compare import compare_step, gpu_outputs
from _scenes import bake_objects_oracle, oracle_scene


@pytest.fixture(scope="module")
def tg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_22332_gb300.tg as tg
    return tg


def _workload():
    wl = W.config1(n_envs=12, n_objects=3, n_grid=24, steps=8)
    wl.objects = bake_objects_oracle(wl.objects)
    wl.params = dict(wl.params, read_delay=2, read_jitter=1)
    return wl


@pytest.mark.parametrize("schedule", ["grid", "persistent", "pipe1024", "pipe512"])
def test_read_delay_matches_oracle(tg, schedule):
    wl = _workload()
    sc = tg.Scene.from_workload(wl)
    sc.upload_objects(wl.objects)
    sc.set_schedule(schedule)
    osc = oracle_scene(wl)
    ost = osc.new_state()
    osc.reset(ost, 0)
    differs = 0
    for s in range(8):
        inp = wl.inputs(s)
        sc.step(inp)
        g = gpu_outputs(sc)
        sc.sync()
        o = osc.step(ost, inp)
        compare_step(g, o, ost, wl.params, wl, where=f"{schedule} delayed step {s}")
        differs += int((o["contact_noisy"] != (o["contact_clean"] & ~((ost["flags"] >> 1) & 1))).sum())
    assert differs > 0, "the delayed contact bits never differed from the current ones"
    sc.close()


def test_read_delay_through_graph_replays_and_checkpoints(tg):
    wl = _workload()
    sc = tg.Scene.from_workload(wl)
    sc.upload_objects(wl.objects)
    sc.set_schedule("pipe1024")
    dev = {k: torch.from_numpy(np.ascontiguousarray(getattr(wl, k))).cuda()
           for k in ("link_pose", "link_vel", "obj_pose", "obj_vel", "obj_id")}
    sc.graph_capture(dict(dev, pose_dt=0.0, step=0), pose_dt_per_step=wl.params["dt"])
    osc = oracle_scene(wl)
    ost = osc.new_state()
    osc.reset(ost, 0)
    for s in range(4):
        sc.graph_launch(1)
        g = gpu_outputs(sc)
        sc.sync()
        compare_step(g, osc.step(ost, wl.inputs(s)), ost, wl.params, wl, where=f"replay {s}")
    saved = sc.save_state()
    sc.graph_launch(2)
    a = [sc.read(ch, noisy) for ch, noisy in ((tg.CH_DEPTH, True), (tg.CH_FORCE_TORQUE, True), (tg.CH_CONTACT, True))]
    sc.sync()
    sc.load_state(saved)
    sc.graph_seek(4, 4 * wl.params["dt"], wl.params["dt"])
    sc.graph_launch(2)
    b = [sc.read(ch, noisy) for ch, noisy in ((tg.CH_DEPTH, True), (tg.CH_FORCE_TORQUE, True), (tg.CH_CONTACT, True))]
    sc.sync()
    for x, y in zip(a, b):
        assert np.array_equal(x.view(np.uint8), y.view(np.uint8))
    sc.graph_release()
    sc.close()
