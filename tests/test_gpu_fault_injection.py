"""Failure detection with faults made on the host (no GPU fault is caused).

- A NaN link pose from the host: the taxels of that link get non-finite
  signed distances, which the step kernels count on the device (the taxels
  read as clear of the surface, nothing is indexed by a NaN); tg_sync
  returns TG_ERR_NUMERIC with the count and clears it, and after a reset the
  next clean step matches the oracle again.
- An object index outside the uploaded objects, passed in host memory: the
  step is rejected on the host with TG_ERR_INVALID_ARG before anything runs,
  and the scene keeps working.
- Bad sizes: reads into buffers of the wrong size (host and device), a
  scene whose lattices do not add up to its taxel counts, and a mesh over
  the no-alloc query's face limit are rejected with TG_ERR_INVALID_ARG.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2606_22332_gb300 import workload as W
from _compare import compare_step, gpu_outputs
from _scenes import bake_objects_oracle, oracle_scene

TG_ERR_INVALID_ARG, TG_ERR_NUMERIC = 1, 6


@pytest.fixture(scope="module")
def tg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_22332_gb300.tg as tg
    return tg


def _workload():
    wl = W.config1(n_envs=8, n_objects=3, n_grid=24, steps=3)
    wl.objects = bake_objects_oracle(wl.objects)
    return wl


@pytest.mark.parametrize("schedule", ["grid", "pipe1024"])
def test_nan_pose_is_reported_then_a_clean_step_recovers(tg, schedule):
    wl = _workload()
    sc = tg.Scene.from_workload(wl)
    sc.upload_objects(wl.objects)
    sc.set_schedule(schedule)
    bad = wl.inputs(0)
    bad["link_pose"] = wl.link_pose.copy()
    e, l = 3, 7
    bad["link_pose"][e, l, 0] = np.nan           # one link's position
    sc.step(bad)
    with pytest.raises(tg.TGError) as err:
        sc.sync()
    n_link = int(wl.link_rows[e * wl.max_links + l] * wl.link_cols[e * wl.max_links + l])
    assert err.value.status == TG_ERR_NUMERIC
    assert f"({n_link} taxel queries)" in str(err.value)
    sc.sync()                                    # the count was cleared
    # the link's taxels read as clear of the surface; nothing non-finite reaches the outputs
    t0 = int(wl.taxel_offsets[e]) + l * n_link
    ft = sc.read(tg.CH_FORCE_TORQUE)
    assert np.all(ft[:, t0:t0 + n_link] == 0) and np.isfinite(ft).all()
    assert np.isfinite(sc.read(tg.CH_DEPTH, True)).all()
    # recovery: a fresh episode and a clean step match the oracle
    sc.reset(1)
    osc = oracle_scene(wl)
    ost = osc.new_state()
    osc.reset(ost, 1)
    inp = wl.inputs(1)
    sc.step(inp)
    g = gpu_outputs(sc)
    sc.sync()
    compare_step(g, osc.step(ost, inp), ost, wl.params, wl, where="after the NaN step")
    sc.close()


def test_nan_pose_is_reported_with_the_raycast_backend(tg):
    """The raycast backend's pre-pass hands a NaN distance to the step for a
    probe with a non-finite pose, so the count reaches tg_sync as with the
    signed-distance backend."""
    wl = W.config0(seed=41, n_envs=6)
    wl.params = dict(wl.params, depth_backend="raycast")
    e = int(np.flatnonzero([wl.objects[k].kind == "mesh" for k in wl.obj_id])[0])
    sc = tg.Scene.from_workload(wl)
    sc.upload_objects(wl.objects)
    bad = wl.inputs(0)
    bad["link_pose"] = wl.link_pose.copy()
    bad["link_pose"][e, 2, 1] = np.nan
    sc.step(bad)
    with pytest.raises(tg.TGError) as err:
        sc.sync()
    L = wl.max_links
    n_link = int(wl.link_rows[e * L + 2] * wl.link_cols[e * L + 2])
    n_act = int((wl.R[int(wl.taxel_offsets[e]) + sum(int(wl.link_rows[e * L + k] * wl.link_cols[e * L + k])
                                                      for k in range(2)):][:n_link] > 0).sum())
    assert err.value.status == TG_ERR_NUMERIC and f"({n_act} taxel queries)" in str(err.value)
    assert np.isfinite(sc.read(tg.CH_FORCE_TORQUE)).all()
    sc.close()


def test_object_index_out_of_range_is_rejected_on_the_host(tg):
    wl = _workload()
    sc = tg.Scene.from_workload(wl)
    sc.upload_objects(wl.objects)
    for bad_id in (len(wl.objects), -1):
        inp = wl.inputs(0)
        inp["obj_id"] = wl.obj_id.copy()
        inp["obj_id"][5] = bad_id
        with pytest.raises(tg.TGError) as err:
            sc.step(inp)
        assert err.value.status == TG_ERR_INVALID_ARG and "obj_id[5]" in str(err.value)
    # nothing ran: the scene still steps and matches the oracle
    osc = oracle_scene(wl)
    ost = osc.new_state()
    osc.reset(ost, 0)
    sc.step(wl.inputs(0))
    g = gpu_outputs(sc)
    sc.sync()
    compare_step(g, osc.step(ost, wl.inputs(0)), ost, wl.params, wl, where="after the rejected steps")
    sc.close()


def test_bad_sizes_are_rejected(tg):
    wl = _workload()
    sc = tg.Scene.from_workload(wl)
    sc.upload_objects(wl.objects)
    sc.step(wl.inputs(0))
    for out in (np.empty(wl.n_taxels - 1, np.float32), torch.empty(wl.n_taxels + 1, device="cuda")):
        with pytest.raises(tg.TGError) as err:
            sc.read(tg.CH_DEPTH, out=out)
        assert err.value.status == TG_ERR_INVALID_ARG
    sc.sync()
    sc.close()
    # a lattice that does not add up to the env's taxel count
    geom = wl.geom()
    geom["link_rows"] = geom["link_rows"].copy()
    geom["link_rows"][0] += 1
    with pytest.raises(tg.TGError) as err:
        tg.Scene(geom, wl.params)
    assert err.value.status == TG_ERR_INVALID_ARG
    # a mesh over the no-alloc query's face limit
    V = torch.zeros((3, 3), dtype=torch.float32, device="cuda")
    F = torch.zeros((tg.NOALLOC_MAX_FACES + 1, 3), dtype=torch.int32, device="cuda")
    pts = torch.zeros((2, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(tg.TGError) as err:
        tg.mesh_sdf_noalloc(V, F, pts, torch.empty(2, dtype=torch.float32, device="cuda"))
    assert err.value.status == TG_ERR_INVALID_ARG
