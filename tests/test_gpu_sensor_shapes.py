"""Launch shapes of the sensor kernels (proximity rays, point-cloud
proximity, elastomer markers with shear anchors): 128, 256 or 512 threads
per CTA give bit-identical outputs, and the autotuner times every shape of
every sensor kernel the scene runs, keeps the fastest and leaves the run's
state as it found it.

Each taxel's proximity reading sums its rays in ray order, each point-cloud
sum is a warp's fixed-order reduction over its candidates, and each
marker's shear sums the contributing points in point order across chunks of
CTA size: none of them depends on the CTA size, so equality is exact.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2606_22332_gb300 import workload as W
from _scenes import bake_objects_oracle

PC = {"pc_radius": 0.01, "pc_k": 300.0, "pc_ks": 10.0, "pc_density": 100.0}
SH = dict(shear_points=1000, s_s=100.0, lambda_s=2000.0, eta_enter=1e-5, eta_exit=1e-4, thickness=2e-3)


@pytest.fixture(scope="module")
def tg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_22332_gb300.tg as tg
    return tg


@pytest.fixture(scope="module")
def wl():
    w = W.config2(n_envs=16, n_objects=3, n_grid=24, faces=(1500, 2500), seed=91)
    w.objects = bake_objects_oracle(w.objects)
    W.add_clouds(w, 1000, seed=7)
    w.params = dict(w.params, **PC)
    w.pads = dict(w.pads, **SH)
    return w


def _outputs(tg, wl, threads=None, tune=False, steps=3):
    sc = tg.Scene.from_workload(wl, sensors=tg.TG_SENSOR_PCPROX)
    sc.upload_objects(wl.objects)
    for k, t in (threads or {}).items():
        sc.set_sensor_threads(k, t)
    rep = None
    if tune:
        sc.step(wl.inputs(0))
        sc.reset(0)
        rep = sc.autotune(wl.inputs(0), steps=1)
        sc.reset(0)
    out = []
    for s in range(steps):
        sc.step(wl.inputs(s))
        out.append({"prox_clean": sc.read(tg.CH_PROX, False), "prox_noisy": sc.read(tg.CH_PROX, True),
                    "markers": sc.read(tg.CH_MARKER), "pc_ft": sc.read(tg.CH_PC_FT),
                    "anchors": sc.read(tg.CH_SHEAR_ANCHORS), "ft_noisy": sc.read(tg.CH_FORCE_TORQUE, True)})
    shape = sc.sensor_threads()
    sc.sync()
    sc.close()
    return out, rep, shape


@pytest.fixture(scope="module")
def reference(tg, wl):
    out, _, shape = _outputs(tg, wl)
    assert shape == {"prox": 256, "pc_prox": 256, "markers": 256}
    assert any((o["anchors"] > 0).any() for o in out), "no anchored point: the shear path would not be exercised"
    assert any((np.abs(o["pc_ft"]) > 0).any() for o in out)
    return out


@pytest.mark.parametrize("kernel", ["prox", "pc_prox", "markers"])
@pytest.mark.parametrize("threads", [128, 512])
def test_sensor_launch_shapes_give_identical_results(tg, wl, reference, kernel, threads):
    out, _, shape = _outputs(tg, wl, {kernel: threads})
    assert shape[kernel] == threads
    for s, (a, b) in enumerate(zip(out, reference)):
        for key in a:
            assert np.array_equal(a[key].view(np.uint8), b[key].view(np.uint8)), f"{kernel}/{threads} step {s} {key}"


def test_autotune_times_every_sensor_shape(tg, wl, reference):
    out, rep, shape = _outputs(tg, wl, tune=True)
    assert len(rep["candidates"]) == 2 * len(tg.SCHEDULES)
    got = {(c["kernel"], c["threads"]) for c in rep["sensor_candidates"]}
    assert got == {(k, t) for k in ("prox", "pc_prox", "markers") for t in (128, 256, 512)}
    assert all(c["ms_per_step"] > 0 for c in rep["sensor_candidates"])
    assert shape == rep["sensor_chosen"]
    for k in ("prox", "pc_prox", "markers"):
        best = min((c for c in rep["sensor_candidates"] if c["kernel"] == k), key=lambda c: c["ms_per_step"])
        assert shape[k] == best["threads"]
    print("sensor shapes", rep["sensor_candidates"], "chosen", shape)
    # tuning leaves no trace in the run's results
    for s, (a, b) in enumerate(zip(out, reference)):
        for key in a:
            assert np.array_equal(a[key].view(np.uint8), b[key].view(np.uint8)), f"after autotune step {s} {key}"


def test_sensor_shape_arguments_are_checked(tg, wl):
    sc = tg.Scene.from_workload(wl)
    for bad in ((0, 64), (0, 1024), (3, 256), (-1, 256)):
        with pytest.raises(tg.TGError):
            sc.set_sensor_threads(*bad)
    sc.close()
