"""TemperatureGrid on the GPU against the FP64 oracle (Appendix
"TemperatureGrid Sensor Model").

Grids of 8 x 8 x 16 cells (2.5 mm voxels). Materials are silicone-like, or
aluminium-like in a third of the grids, where diffusion damps the high modes
strongly. Contacts fall on the grids' faces, the internal source is on in
some steps, and the fields start from random 22..45 C values.

The GPU diffuses through orthonormal DCT-II transforms in FP32. Each transform
is three contractions of length <= 16 on values within ~25 C of the first
cell, so one step's round-off is bounded by ~6 x 16 x 2^-24 x 25 C = 1.4e-4 C
in the worst case. The test allows 1.5e-4 C per step.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import temperature as TO
from paper_2606_22332_gb300 import workload as W

DIMS = (8, 8, 16)
TOL_PER_STEP = 1.5e-4


@pytest.fixture(scope="module")
def tg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_22332_gb300.tg as tg
    return tg


def _oracle_step(wl, T, Tm, dt, t_amb, source, contacts):
    To, Tmo = np.empty_like(T), np.empty_like(Tm)
    for g in range(wl["G"]):
        m = wl["material"][g].astype(np.float64)
        mat = dict(k=m[0], rho=m[1], cp=m[2], emissivity=m[3], h=m[4], tau=m[5])
        cs = []
        if contacts is not None:
            for c in range(contacts["offsets"][g], contacts["offsets"][g + 1]):
                cs.append((int(contacts["cell"][c]), float(contacts["temp"][c]), float(contacts["k"][c]),
                           float(contacts["area"][c])))
        q = None if source is None else source[g].astype(np.float64)
        To[g], Tmo[g] = TO.step(T[g], Tm[g], wl["voxel"][g].astype(np.float64), mat, dt, t_amb, source=q,
                                contacts=cs)
    return To, Tmo


@pytest.mark.parametrize("device_contacts", [False, True])
def test_temperature_steps_against_the_oracle(tg, device_contacts):
    rng = np.random.default_rng(7)
    wl = W.temperature_grids(seed=3, n_envs=8, links_per_env=3, dims=DIMS, metal_share=0.34)
    G = wl["G"]
    tg_ = tg.TempGrid(DIMS, wl["voxel"], wl["material"])
    T = (22 + 23 * rng.random((G,) + DIMS)).astype(np.float32).astype(np.float64)
    Tm = (T - rng.random(T.shape)).astype(np.float32).astype(np.float64)
    tg_.set(T.astype(np.float32), Tm.astype(np.float32))
    dt, t_amb = 0.02, 22.0
    worst = 0.0
    for s in range(6):
        contacts = W.temperature_contacts(rng, G, DIMS, share=0.6)
        source = (rng.uniform(0, 2e3, (G,) + DIMS).astype(np.float32) if s % 2 else None)
        src_d = torch.as_tensor(source.reshape(G, -1), device="cuda") if source is not None else None
        cd = contacts
        if device_contacts:
            cd = {k: torch.as_tensor(v, device="cuda") for k, v in contacts.items()}
        tg_.step(dt, t_amb, source=src_d, contacts=cd)
        Tg, Tmg = tg_.read(False), tg_.read(True)
        T, Tm = _oracle_step(wl, T, Tm, dt, t_amb, source, contacts)
        err = max(np.abs(Tg - T).max(), np.abs(Tmg - Tm).max())
        worst = max(worst, err)
        assert err <= TOL_PER_STEP * (s + 1), (s, err)
    # the step did move the fields: diffusion, contacts and surface loss are all exercised
    assert np.abs(T - T.mean(axis=(1, 2, 3), keepdims=True)).max() > 0.1
    print(f"worst |T_gpu - T_oracle| over 6 steps: {worst:.2e} C")
    tg_.close()


def test_uniform_grids_stay_at_base_and_reset(tg):
    wl = W.temperature_grids(seed=4, n_envs=4, links_per_env=2, dims=DIMS)
    tg_ = tg.TempGrid(DIMS, wl["voxel"], wl["material"])
    base = wl["material"][:, 6]
    T0 = tg_.read()
    assert np.array_equal(T0, np.broadcast_to(base[:, None, None, None], T0.shape))
    for _ in range(3):
        tg_.step(0.005, float(base[0]))  # ambient = base: nothing moves
    assert np.allclose(tg_.read(), T0, atol=2e-5)
    hot = np.full(T0.shape, 40.0, np.float32)
    tg_.set(hot)
    mask = np.zeros(wl["G"], np.uint8)
    mask[::2] = 1
    tg_.reset(mask)
    T1 = tg_.read()
    assert np.array_equal(T1[::2], T0[::2]) and np.all(T1[1::2] == 40.0)
    tg_.close()


def test_contact_area_against_the_oracle(tg):
    rng = np.random.default_rng(11)
    P, M = 200, 8
    pts = np.zeros((P, M, 3), np.float32)
    npts = rng.integers(1, M + 1, P).astype(np.int32)
    depth = rng.uniform(1e-5, 1e-3, P).astype(np.float32)
    for p in range(P):
        R = np.linalg.qr(rng.standard_normal((3, 3)))[0]
        uv = rng.uniform(-5e-3, 5e-3, (M, 2))
        local = np.concatenate([uv, rng.normal(0, 1e-5, (M, 1))], 1)  # nearly planar patches
        pts[p] = (local @ R.T + rng.uniform(-0.1, 0.1, 3)).astype(np.float32)
    area = tg.contact_area(torch.as_tensor(pts, device="cuda"), torch.as_tensor(npts, device="cuda"),
                           torch.as_tensor(depth, device="cuda"), d_w=1.0).cpu().numpy()
    ref = np.array([TO.contact_area(pts[p, :npts[p]].astype(np.float64), float(depth[p]), 1.0) for p in range(P)])
    assert np.allclose(area, ref, rtol=2e-4, atol=0), np.abs(area / ref - 1).max()
    assert (npts < 3).any() and (ref > np.pi * depth.astype(np.float64) ** 2 * 1.01).any()


def test_temperature_arguments_are_checked(tg):
    wl = W.temperature_grids(seed=5, n_envs=2, links_per_env=1, dims=DIMS)
    for dims in ((6, 8, 16), (12, 8, 16), (8, 8, 64), (0, 8, 8)):
        with pytest.raises(tg.TGError):
            tg.TempGrid(dims, wl["voxel"], wl["material"])
    bad = wl["material"].copy()
    bad[0, 1] = -1.0
    with pytest.raises(tg.TGError):
        tg.TempGrid(DIMS, wl["voxel"], bad)
    tg_ = tg.TempGrid(DIMS, wl["voxel"], wl["material"])
    with pytest.raises(tg.TGError):
        tg_.step(0.0, 22.0)
    c = W.temperature_contacts(np.random.default_rng(0), wl["G"], DIMS, share=1.0)
    c["cell"] = c["cell"].copy()
    c["cell"][0] = 8 * 8 * 16
    with pytest.raises(tg.TGError):
        tg_.step(0.005, 22.0, contacts=c)
    tg_.close()
