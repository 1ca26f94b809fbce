"""ElastomerTaxel shear anchors (Eqs. 19-20): CUDA path against the FP64 oracle.

Workload: 12 envs of the full-sensor scene (uneven fingertip links, five
16 x 16 marker pads per env on the fingertips, objects as FP16 grids pressed
into them and moving with their poses), every object carrying 1,000 tracked
surface points (the paper's N_pc), s_s = 100, lambda_s = 2000, eta_enter =
1e-5 m, eta_exit = 1e-4 m, a 2 mm elastomer.

Anchors are set and released on float comparisons of the points' elastomer
SDF; the oracle reports, per pad and step, how far the SDF of each point is
from the threshold it faces.  A pad whose margin falls below 1e-6 m (50x the
~2e-8 m error of the float pad coordinates) is set aside from that step on;
every other pad must match the oracle's anchor count exactly and its
displacements within 1e-5 |u| + 1e-7 drag, drag = s_s sum (h + |z - e|) over
the points in or near contact (a coordinate error eps moves a point's term by
at most s_s eps (2 h + |z - e|)).  The shear part is checked with the
dilation scale s_d = 0, so that the marker output is the shear alone; one
run with dilation on checks their sum.
"""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2606_22332_gb300 import workload as W
from _scenes import bake_objects_oracle, oracle_scene

SH = dict(s_s=100.0, lambda_s=2000.0, eta_enter=1e-5, eta_exit=1e-4, thickness=2e-3)
N_PC = 1000
BAND = 1e-6


@pytest.fixture(scope="module")
def tg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_22332_gb300.tg as tg
    return tg


@pytest.fixture(scope="module")
def base_wl():
    wl = W.config2(n_envs=12, n_objects=3, n_grid=24, faces=(1500, 2500), seed=77)
    wl.objects = bake_objects_oracle(wl.objects)
    W.add_clouds(wl, N_PC, seed=5)
    return wl


def _with_shear(wl, s_d):
    wl.pads = dict(wl.pads, shear_points=N_PC, s_d=s_d, **SH)
    return wl


class _Pair:
    """GPU scene and oracle side by side over steps."""

    def __init__(self, tg, wl):
        self.tg, self.wl = tg, wl
        self.sc = tg.Scene.from_workload(wl)
        self.sc.upload_objects(wl.objects)
        self.osc = oracle_scene(wl)
        self.P = wl.pads["pads_per_env"]
        self.ost = self.osc.new_shear_state(self.P, N_PC)
        self.clouds = [o.cloud for o in wl.objects]
        self.amb = np.zeros(wl.n_envs * self.P, bool)
        self.worst = 0.0

    def step(self, inp, dilation=False):
        tg, sc = self.tg, self.sc
        sc.step(inp)
        mu = sc.read(tg.CH_MARKER).astype(np.float64).reshape(self.wl.n_envs * self.P, -1, 3)
        na = sc.read(tg.CH_SHEAR_ANCHORS)
        sc.sync()
        us, no, mg, dg = self.osc.shear_step(self.wl.pads, self.clouds, SH, inp, self.ost, drag=True)
        uo = us.reshape(mu.shape)
        tol_pad = 1e-7 * dg.reshape(-1)[:, None, None]
        if dilation:
            ud, _ = self.osc.markers(self.wl.pads, inp)
            ud = ud.reshape(mu.shape)
            uo = uo + ud
            tol_pad = tol_pad + 1e-4 * np.abs(ud) + 1e-7
        self.amb |= mg.reshape(-1) < BAND
        ok = ~self.amb
        no = no.reshape(-1)
        assert np.array_equal(na[ok], no[ok]), f"anchor counts differ on {np.flatnonzero(ok & (na != no))}"
        err = np.abs(mu - uo)
        tol = 1e-5 * np.abs(uo) + tol_pad
        bad = (err > tol) & ok[:, None, None]
        assert not bad.any(), f"marker err {err[bad].max():.3e} on pads {np.unique(np.nonzero(bad)[0])}"
        self.worst = max(self.worst, float((err / np.maximum(tol, 1e-30))[ok].max()) if ok.any() else 0.0)
        return na, no, uo

    def close(self):
        self.sc.close()


def test_shear_anchors_against_the_oracle(tg, base_wl):
    wl = _with_shear(base_wl, s_d=0.0)
    pr = _Pair(tg, wl)
    live = 0
    for s in range(6):
        na, no, uo = pr.step(wl.inputs(s))
        sheared = (np.abs(uo).reshape(len(na), -1).max(1) > 0) & ~pr.amb
        live += int(sheared.sum())
    pr.close()
    print(f"worst err / tol {pr.worst:.3f}; pads set aside {int(pr.amb.sum())} of {pr.amb.size}; "
          f"sheared pad-steps compared {live}")
    assert pr.amb.sum() <= 0.25 * pr.amb.size
    assert live >= 60, "too few sheared pads: the test would not exercise the shear sum"


def test_shear_adds_to_the_dilation(tg, base_wl):
    wl = _with_shear(base_wl, s_d=1.0)
    pr = _Pair(tg, wl)
    for s in range(3):
        pr.step(wl.inputs(s), dilation=True)
    pr.close()


def test_reset_and_object_change_clear_the_anchors(tg, base_wl):
    wl = _with_shear(base_wl, s_d=0.0)
    pr = _Pair(tg, wl)
    for s in range(2):
        pr.step(wl.inputs(s))
    # reset envs 0..3: their anchors are gone (the oracle's state alike)
    mask = np.zeros(wl.n_envs, np.uint8)
    mask[:4] = 1
    pr.sc.reset(0, env_mask=mask)
    pr.ost["anchors"][:4] = np.nan
    pr.ost["anchor_obj"][:4] = -1
    na, no, _ = pr.step(wl.inputs(2))
    # a reset env's points re-anchor where they are: no shear on the step after a reset
    u0 = pr.sc.read(tg.CH_MARKER).reshape(wl.n_envs, -1, 3)[:4]
    assert np.all(u0 == 0.0)
    # envs 4..7 switch objects
    inp = dict(wl.inputs(3))
    oid = inp["obj_id"].copy()
    oid[4:8] = (oid[4:8] + 1) % len(wl.objects)
    inp["obj_id"] = oid
    pr.step(inp)
    u1 = pr.sc.read(tg.CH_MARKER).reshape(wl.n_envs, -1, 3)[4:8]
    assert np.all(u1 == 0.0)
    pr.close()


def test_checkpoint_keeps_the_anchors(tg, base_wl):
    wl = _with_shear(base_wl, s_d=0.0)
    sc = tg.Scene.from_workload(wl)
    sc.upload_objects(wl.objects)
    for s in range(2):
        sc.step(wl.inputs(s))
    blob = sc.save_state()
    sc.step(wl.inputs(2))
    a = sc.read(tg.CH_MARKER).copy()
    sc.load_state(blob)
    sc.step(wl.inputs(2))
    b = sc.read(tg.CH_MARKER)
    sc.sync()
    sc.close()
    assert np.array_equal(a, b) and np.abs(a).max() > 0


def test_shear_arguments_are_checked(tg, base_wl):
    wl = _with_shear(base_wl, s_d=0.0)
    # clouds larger than the anchor slots
    wl2 = dataclasses.replace(wl, pads=dict(wl.pads, shear_points=N_PC - 1))
    sc = tg.Scene.from_workload(wl2)
    with pytest.raises(tg.TGError):
        sc.upload_objects(wl.objects)
    sc.close()
    for bad in (dict(thickness=0.0), dict(eta_enter=-1e-5), dict(shear_points=70000), dict(s_s=float("nan"))):
        wl2.pads = dict(wl.pads, **bad)
        with pytest.raises(tg.TGError):
            tg.Scene.from_workload(wl2)
