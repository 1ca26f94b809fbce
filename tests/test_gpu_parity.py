"""CUDA path against the FP64 oracle, element by element, through the C-ABI.

Covers: the plain method with analytic spheres and exact meshes (every query
of the 64-env workload), batched FP32 and FP16 grids over several steps with
the pose advance, uneven CSR layouts with envs split over several work items,
fillers, empty envs, resets of env subsets, checkpoints, host versus device
inputs, determinism, and the exact-mesh bake.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle
from paper_2606_22332_gb300 import workload as W
from _compare import compare_step, gpu_outputs
from _scenes import bake_objects_oracle, oracle_scene, pad_workload, quiet_params


@pytest.fixture(scope="module")
def tg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_22332_gb300.tg as tg
    return tg


def run_both(tg, wl, steps, sensors=0, step0=0):
    scene = tg.Scene.from_workload(wl, sensors=sensors)
    scene.upload_objects(wl.objects)
    osc = oracle_scene(wl)
    ost = osc.new_state()
    osc.reset(ost, 0)
    all_stats = []
    for s in range(step0, step0 + steps):
        inp = wl.inputs(s)
        scene.step(inp)
        g = gpu_outputs(scene)
        scene.sync()
        o = osc.step(ost, inp)
        all_stats.append(compare_step(g, o, ost, wl.params, wl, where=f"{wl.name} step {s}"))
    scene.close()
    return all_stats


def test_config0_sphere_and_mesh_every_query(tg):
    wl = W.config0()
    stats = run_both(tg, wl, steps=3, sensors=tg.TG_SENSOR_DIST)
    print("config0", stats)


def test_grid_fp32_batched_multi_step(tg):
    rng = np.random.default_rng(11)
    wl = W.config1(n_envs=24, n_objects=4, n_grid=24, steps=6)
    wl.objects = bake_objects_oracle(wl.objects)
    stats = run_both(tg, wl, steps=6, sensors=tg.TG_SENSOR_DIST)
    print("grid32", stats[-1])


def test_grid_fp16_uneven_split_items(tg):
    rng = np.random.default_rng(12)
    objs = bake_objects_oracle(W.config1_objects(rng, 3, n_grid=20, fp16=True, faces=(1500, 2500)))
    lat = W.uneven_lattices(rng, 14, taxels=(200, 1000), links=(10, 20))
    lat += W.uneven_lattices(rng, 3, taxels=(1100, 2600), links=(3, 6), cols=16)  # envs over one work item
    lat.insert(5, [])                                                              # an env without taxels
    env_obj = rng.integers(0, len(objs), len(lat))
    wl = W._assemble("uneven16", rng, objs, env_obj, lat, W.default_params(99), steps=4, max_links=20,
                     arc=W.PAD_ARC)
    assert wl.taxel_offsets[6] == wl.taxel_offsets[5]
    stats = run_both(tg, wl, steps=4)
    print("grid16", stats[-1])


def test_plate_force_on_gpu(tg):
    rng = np.random.default_rng(3)
    depths = rng.uniform(-1e-3, 3e-3, (7, 9))
    wl = pad_workload(depths, 7, 9, params=W.default_params(5), link_vel=(0.05, -0.02, 0.1, 0.3, -0.2, 0.5))
    run_both(tg, wl, steps=5)


def test_fillers_and_paper_parameters(tg):
    p = W.default_params(8)
    p.update(alpha=1.2, k=500.0, c=1.0, mu=None)          # the paper's KinematicTaxel values, no clamp
    p["noise"]["depth"] = W.noise_group(beta=0.5, tau=0.05, sigma_white=2e-4, quant=1e-4, gain_lo=0.85, gain_hi=1.15)
    p["noise"]["ft"] = W.noise_group(beta=0.5, tau=0.05, sigma_white=5e-3, sigma_rw=1e-4, gain_lo=0.85, gain_hi=1.15,
                                     stuck_lo=-0.1, stuck_hi=0.1)
    p["p_dead"] = 0.05
    wl = W.config0(seed=77, n_envs=8)
    wl.params = p
    wl.R[::7] = 0.0                                          # fillers scattered through every lattice
    run_both(tg, wl, steps=3)


def test_determinism_and_checkpoint(tg):
    wl = W.config1(n_envs=6, n_objects=2, n_grid=16, steps=5)
    wl.objects = bake_objects_oracle(wl.objects)
    sc = tg.Scene.from_workload(wl)
    sc.upload_objects(wl.objects)
    for s in range(3):
        sc.step(wl.inputs(s))
    blob = sc.save_state()
    outs = []
    for s in (3, 4):
        sc.step(wl.inputs(s))
        outs.append(gpu_outputs(sc))
    sc.load_state(blob)
    for k, s in enumerate((3, 4)):
        sc.step(wl.inputs(s))
        again = gpu_outputs(sc)
        for key in ("flags", "depth_noisy", "ft_noisy", "link_sums"):
            assert np.array_equal(again[key], outs[k][key]), key
    sc.close()


def test_host_and_device_inputs_agree(tg):
    wl = W.config0(n_envs=8)
    a = tg.Scene.from_workload(wl); a.upload_objects(wl.objects)
    b = tg.Scene.from_workload(wl); b.upload_objects(wl.objects)
    inp = wl.inputs(2)
    dev = {k: (torch.as_tensor(v).cuda() if isinstance(v, np.ndarray) else v) for k, v in inp.items()}
    a.step(inp)
    b.step(dev)
    ga, gb = gpu_outputs(a), gpu_outputs(b)
    for k in ga:
        if ga[k] is not None:
            assert np.array_equal(ga[k], gb[k]), k
    # device views equal the copies
    import paper_2606_22332_gb300.tg as T
    assert np.array_equal(b.buffer(T.CH_FORCE_TORQUE, True).cpu().numpy(), gb["ft_noisy"])
    a.close(); b.close()


def test_reset_subset_of_envs(tg):
    wl = W.config0(n_envs=10)
    wl.params = dict(wl.params, p_dead=0.3)
    sc = tg.Scene.from_workload(wl); sc.upload_objects(wl.objects)
    osc = oracle_scene(wl); ost = osc.new_state(); osc.reset(ost, 0)
    mask = np.zeros(10, np.uint8); mask[[1, 4, 7]] = 1
    sc.step(wl.inputs(0)); osc.step(ost, wl.inputs(0))
    before = gpu_outputs(sc)
    sc.reset(5, env_mask=mask); osc.reset(ost, 5, env_mask=mask)
    # a reset env's clean depth and force/torque read zero until its next
    # step (they carry the hysteresis x_{t-1}); the other envs keep theirs
    after = gpu_outputs(sc); sc.sync()
    in_reset = np.repeat(mask.astype(bool), np.diff(wl.taxel_offsets))
    for k in ("depth_clean", "ft_clean"):
        assert not after[k][..., in_reset].any(), k
        assert np.array_equal(after[k][..., ~in_reset], before[k][..., ~in_reset]), k
    for s in (1, 2):
        sc.step(wl.inputs(s))
        g = gpu_outputs(sc); sc.sync()
        o = osc.step(ost, wl.inputs(s))
        compare_step(g, o, ost, wl.params, wl, where=f"reset step {s}")
    sc.close()


def test_bake_matches_oracle(tg):
    rng = np.random.default_rng(21)
    for fp16 in (False, True):
        V, F = W.hull_mesh(rng, 96, 0.04, min_faces=1000)
        lo, hi = W.grid_box(V)
        dims = (17, 19, 18)
        ref = oracle.bake_grid(V, F, dims, lo.astype(np.float64), hi.astype(np.float64), fp16=fp16)
        got = tg.bake_grid(V, F, dims, lo, hi, fp16=fp16).cpu().numpy()
        if fp16:
            got = got.view(np.uint16)
            same = got == ref
            refv = ref.view(np.float16).astype(np.float64)
        else:
            same = got == ref
            refv = ref.astype(np.float64)
        # a node may round differently only when its exact value sits on a rounding tie
        # (or on the surface, where the sign of a ~0 value is arbitrary)
        bad = ~same & (np.abs(refv) > 1e-7)
        assert bad.sum() <= max(1, 1e-4 * ref.size), (fp16, int(bad.sum()))


def test_mesh_sdf_points_match_oracle(tg):
    rng = np.random.default_rng(22)
    V, F = W.hull_mesh(rng, 64, 0.04, min_faces=500)
    q = rng.uniform(-0.03, 0.03, (4000, 3)).astype(np.float32)
    phi, grad = tg.mesh_sdf(V, F, torch.as_tensor(q).cuda())
    ophi, og = oracle.Obj.mesh(V, F).sdf(q.astype(np.float64))
    # the float32 output is the compensated distance rounded once: within half an ulp
    assert (np.abs(phi.cpu().numpy() - ophi) <= 6e-8 * np.abs(ophi) + 1e-12).all()
    far = np.abs(ophi) > 1e-6
    assert np.abs(grad.cpu().numpy()[far] - og[far]).max() < 1e-4


def test_maximum_sizes(tg):
    """A link of tg_max_link_taxels() taxels (one whole work item), an env of
    33 links (split by the 32-link item limit), one-taxel links and a
    one-taxel env."""
    rng = np.random.default_rng(21)
    assert tg.lib().tg_max_link_taxels() == 1024
    objs = bake_objects_oracle(W.config1_objects(rng, 2, n_grid=24, fp16=True, faces=(1500, 2500)))
    lat = [[(32, 32, 1024)], [(2, 3, 6)] * 33, [(32, 32, 1024), (1, 1, 1), (4, 5, 20)], [(1, 1, 1)]]
    wl = W._assemble("maxsize", rng, objs, rng.integers(0, 2, len(lat)), lat, W.default_params(7), steps=3,
                     max_links=34, arc=W.PAD_ARC)
    stats = run_both(tg, wl, steps=3)
    print("maxsize", stats[-1])


@pytest.mark.parametrize("case", ["config0", "grid16", "paper_noisy"])
def test_probe_radius_noise(tg, case):
    """Probe-radius noise (rho): the noisy readout's depth, contact bit and
    force/torque from max(0, R + eps) against the oracle, every query."""
    if case == "config0":
        wl = W.config0(seed=31, n_envs=12)
        wl.params = dict(wl.params, rho=3e-4)
        sensors = tg.TG_SENSOR_DIST
    elif case == "grid16":
        wl = W.config1(n_envs=16, n_objects=3, n_grid=24, steps=4)
        wl.objects = bake_objects_oracle(wl.objects)
        wl.params = dict(wl.params, rho=5e-4)
        sensors = 0
    else:
        p = W.default_params(9)
        p.update(alpha=1.2, k=500.0, c=1.0, mu=None, rho=3e-4, p_dead=0.05)
        p["noise"]["depth"] = W.noise_group(beta=0.5, tau=0.05, sigma_white=2e-4, quant=1e-4, gain_lo=0.85,
                                            gain_hi=1.15)
        p["noise"]["ft"] = W.noise_group(beta=0.5, tau=0.05, sigma_white=5e-3, sigma_rw=1e-4, gain_lo=0.85,
                                         gain_hi=1.15, stuck_lo=-0.1, stuck_hi=0.1)
        wl = W.config0(seed=78, n_envs=10)
        wl.params = p
        sensors = 0
    stats = run_both(tg, wl, steps=3, sensors=sensors)
    print(case, stats[-1])


def test_probe_radius_noise_bounds_are_checked(tg):
    wl = W.config0(seed=32, n_envs=2)
    for bad in (-1e-6, 6e-4, float("nan")):
        with pytest.raises(tg.TGError):
            tg.Scene.from_workload(dict_params(wl, rho=bad))


def dict_params(wl, **over):
    wl.params = dict(wl.params, **over)
    return wl
