"""The CUDA path at full size, in the bench's launch configuration, against
the oracle on sampled envs.

20,480 envs x 20 links x 50 taxels and 64 objects as 96^3 binary16 grids
(the headline workload's sizes); the objects are low-poly hulls so that the
oracle bakes the very grids the GPU reads.  As bench.py does, the schedule
is picked by the autotuner and the steps run as replays of a captured CUDA
graph.  Envs are independent, so the oracle steps a sample of envs (a
subset scene keeping their global taxel and env ids) and every output of
those envs is compared element by element.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2606_22332_gb300 import workload as W
from _compare import compare_step
from _scenes import low_poly_grid_objects, oracle_scene

E, L, N_OBJ = 20480, 20, 64


@pytest.fixture(scope="module")
def tg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_22332_gb300.tg as tg
    return tg


def _gather(tg, sc, off, sub, envs):
    """The sampled envs' outputs, gathered on the device in subset order
    (off: the full scene's taxel offsets)."""
    T = sub.taxel_offsets[-1]
    idx = torch.from_numpy(np.concatenate([np.arange(off[e], off[e + 1]) for e in envs])).cuda()
    lidx = torch.from_numpy((envs[:, None] * L + np.arange(L)[None, :]).reshape(-1)).cuda()
    flags = sc.buffer(tg.CH_STATE_FLAGS)[idx].cpu().numpy()
    out = {
        "flags": flags,
        "contact_clean": (flags & 1).astype(np.uint8),
        "contact_noisy": ((flags >> 2) & 1).astype(np.uint8),
        "depth_clean": sc.buffer(tg.CH_DEPTH, False)[idx].cpu().numpy(),
        "depth_noisy": sc.buffer(tg.CH_DEPTH, True)[idx].cpu().numpy(),
        "ft_clean": sc.buffer(tg.CH_FORCE_TORQUE, False).reshape(6, -1)[:, idx].cpu().numpy(),
        "ft_noisy": sc.buffer(tg.CH_FORCE_TORQUE, True).reshape(6, -1)[:, idx].cpu().numpy(),
        "link_sums": sc.buffer(tg.CH_LINK_WRENCH).reshape(E * L, -1)[lidx].cpu().numpy(),
        "link_counts": sc.buffer(tg.CH_LINK_COUNT).reshape(E * L, 2)[lidx].cpu().numpy(),
        "dist": None,
    }
    assert len(out["depth_clean"]) == T
    return out


def test_full_size_sampled_parity_in_the_bench_launch_configuration(tg):
    rng = np.random.default_rng(20260003)
    objs = low_poly_grid_objects(rng, N_OBJ, 96, fp16=True)
    wl = W._assemble("metric_run_lowpoly", rng, objs, rng.integers(0, N_OBJ, E), [[(5, 10, 50)] * L] * E,
                     W.default_params(20260003), steps=3, arc=W.PAD_ARC)
    assert wl.n_active == E * 1000
    sc = tg.Scene(wl.geom(), wl.params)
    sc.upload_objects(wl.objects)
    dt = wl.params["dt"]
    d_in = {k: torch.as_tensor(getattr(wl, k)).cuda() for k in ("link_pose", "link_vel", "obj_pose", "obj_vel",
                                                                "obj_id")}
    rep = sc.autotune(dict(d_in, pose_dt=0.0, step=0), steps=2)
    sc.graph_capture(dict(d_in, pose_dt=0.0, step=0), pose_dt_per_step=dt)

    envs = np.sort(rng.choice(E, 48, replace=False))
    sub = wl.subset(envs)
    osc = oracle_scene(sub)
    ost = osc.new_state()
    osc.reset(ost, 0)
    for s in range(3):
        sc.graph_launch(1)
        torch.cuda.synchronize()
        g = _gather(tg, sc, wl.taxel_offsets, sub, envs)
        o = osc.step(ost, sub.inputs(s))
        st = compare_step(g, o, ost, sub.params, sub, where=f"full size, replay {s}")
    pen = float((o["depth_clean"] > 0).mean())
    worst = {k: v for k, v in st.items() if k != "outliers"}
    print(f"schedule {rep['chosen']}; sampled taxels {sub.n_active}, penetrating share {pen:.3f}; {worst}")
    assert pen > 0.02
    sc.graph_release()
    sc.sync()
    sc.close()
