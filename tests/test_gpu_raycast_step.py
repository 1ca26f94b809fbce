"""The raycast contact-depth backend inside the sensor step on the GPU
against the oracle (paper, "Probe geometry and contact-depth query", two
contact-depth backends): a mesh's depth is R minus the distance from the
probe centre to the nearest triangle within R, its contact normal that
triangle's normal.

Workload: the capsule links of the plain-method scene (spheres and ~2,000-
face hulls), several steps with moving links, the full noise model, through
the grid and the pipelined schedules, and a run with per-env scale
randomisation.  Depth, surface distance and contact bits are compared at the
usual bounds.  Where the deepest feature is an edge or a vertex shared by
faces with different normals (the oracle flags it), either face's normal is
a valid answer: such taxels, and every later reading of them (their force
enters the hysteresis state), are left out of the force/torque checks and
enter their links' sums with the error they show; so do their 3x3
crosstalk neighbours on the lattice, whose noisy readout mixes in the tie
taxel's force.  One pre-pass launch per step answers every mesh taxel.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2606_22332_gb300 import workload as W
from _compare import compare_step, gpu_outputs
from _scenes import oracle_scene


@pytest.fixture(scope="module")
def tg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_22332_gb300.tg as tg
    return tg


def _with_crosstalk_neighbours(wl, mask):
    """`mask` grown by one lattice cell in every direction on each link (the
    columns wrap on a wrapped link), the reach of the 3x3 crosstalk."""
    out = mask.copy()
    L = wl.max_links
    for e in range(wl.n_envs):
        t0 = int(wl.taxel_offsets[e])
        for l in range(L):
            r, c = int(wl.link_rows[e * L + l]), int(wl.link_cols[e * L + l])
            if r * c == 0:
                continue
            m = mask[t0:t0 + r * c].reshape(r, c)
            if m.any():
                g = m.copy()
                for dr in (-1, 0, 1):
                    for dc in (-1, 0, 1):
                        src = np.zeros_like(m)
                        rs, rd = (slice(max(dr, 0), r + min(dr, 0)), slice(max(-dr, 0), r + min(-dr, 0)))
                        if wl.link_wrap[e * L + l]:
                            sh = np.roll(m, -dc, axis=1)
                            src[rd] = sh[rs]
                        else:
                            cs, cd = (slice(max(dc, 0), c + min(dc, 0)), slice(max(-dc, 0), c + min(-dc, 0)))
                            src[rd, cd] = m[rs, cs]
                        g |= src
                out[t0:t0 + r * c] = g.reshape(-1)
            t0 += r * c
    return out


def _run(tg, wl, schedule, steps):
    sc = tg.Scene.from_workload(wl, sensors=tg.TG_SENSOR_DIST)
    sc.upload_objects(wl.objects)
    sc.set_schedule(schedule)
    osc = oracle_scene(wl)
    ost = osc.new_state()
    osc.reset(ost, 0)
    ties = np.zeros(len(wl.R), bool)
    mesh_env = np.array([wl.objects[int(k)].kind == "mesh" for k in wl.obj_id])
    in_mesh = np.repeat(mesh_env, np.diff(wl.taxel_offsets)) & (wl.R > 0)
    n_contact = 0
    for s in range(steps):
        inp = wl.inputs(s)
        sc.step(inp)
        g = gpu_outputs(sc)
        sc.sync()
        o = osc.step(ost, inp)
        ties |= o["depth_tie"].astype(bool)
        st = compare_step(g, o, ost, wl.params, wl, where=f"raycast {schedule} step {s}",
                          exclude=_with_crosstalk_neighbours(wl, ties))
        n_contact += int((o["contact_clean"] & in_mesh).sum())
    sc.close()
    assert n_contact > 0, "no mesh taxel ever touched"
    assert ties.sum() <= 0.01 * in_mesh.sum(), ties.sum()
    return st, int(ties.sum())


@pytest.mark.parametrize("schedule", ["grid", "persistent", "pipe1024", "pipe512"])
def test_raycast_step_matches_oracle(tg, schedule):
    wl = W.config0(seed=41, n_envs=12)
    wl.params = dict(wl.params, depth_backend="raycast")
    st, nt = _run(tg, wl, schedule, steps=4)
    print(schedule, "ties", nt, {k: v for k, v in st.items() if k != "outliers"})


def test_raycast_step_with_scale_randomisation(tg):
    wl = W.config0(seed=42, n_envs=10)
    wl.params = dict(wl.params, depth_backend="raycast",
                     dr={"mu": (0.6, 1.0), "k": (5e3, 2e4), "scale": (0.9, 1.2)})
    _run(tg, wl, "grid", steps=3)


def test_raycast_and_sdf_agree_outside_the_mesh(tg):
    """Outside a closed mesh the nearest triangle's distance is the signed
    distance: taxels whose probe centre is outside (positive signed
    distance) read the same depth through either backend."""
    wl = W.config0(seed=43, n_envs=8)
    wl.params = dict(wl.params, p_dead=0.0)
    outs = {}
    for backend in ("sdf", "raycast"):
        wl.params = dict(wl.params, depth_backend=backend)
        sc = tg.Scene.from_workload(wl, sensors=tg.TG_SENSOR_DIST)
        sc.upload_objects(wl.objects)
        sc.step(wl.inputs(0))
        outs[backend] = gpu_outputs(sc)
        sc.sync()
        sc.close()
    R = wl.R.astype(np.float64)
    outside = (outs["sdf"]["dist"] > -R) & (R > 0)       # phi = dist + R > 0
    assert outside.sum() > 0
    d = np.abs(outs["sdf"]["depth_clean"][outside].astype(np.float64) - outs["raycast"]["depth_clean"][outside])
    assert d.max() <= 2e-6, d.max()


def test_raycast_backend_rejects_probe_radius_noise(tg):
    wl = W.config0(seed=44, n_envs=2)
    wl.params = dict(wl.params, depth_backend="raycast", rho=1e-4)
    with pytest.raises(tg.TGError):
        tg.Scene.from_workload(wl)
