"""Structure of the seeded input generators (they hold none of the method's
arithmetic, only the shapes and distributions of the workloads)."""
import numpy as np

from paper_2606_22332_gb300 import workload as W


def test_temperature_grids_and_contacts_are_well_formed():
    wl = W.temperature_grids(seed=1, n_envs=50, links_per_env=5, dims=(8, 8, 16), metal_share=0.3)
    G = wl["G"]
    assert G == 250 and wl["voxel"].shape == (G, 3) and wl["material"].shape == (G, 7)
    assert np.allclose(wl["voxel"], [0.0025, 0.0025, 0.0025])
    m = wl["material"]
    assert np.all(m[:, 0] > 0) and np.all(m[:, 1] > 0) and np.all(m[:, 2] > 0)
    assert np.all((m[:, 3] >= 0) & (m[:, 3] <= 1)) and np.all(m[:, 6] == 22.0)
    assert 0.15 < np.mean(m[:, 0] > 100) < 0.45  # the metal share
    rng = np.random.default_rng(2)
    c = W.temperature_contacts(rng, G, (8, 8, 16), share=0.4, max_per_grid=4)
    off = c["offsets"]
    assert off[0] == 0 and off[-1] == len(c["cell"]) and np.all(np.diff(off) >= 0) and np.all(np.diff(off) <= 4)
    assert 0.25 < np.mean(np.diff(off) > 0) < 0.55
    i, r = np.divmod(c["cell"], 8 * 16)
    j, k = np.divmod(r, 16)
    on_face = (i == 0) | (i == 7) | (j == 0) | (j == 7) | (k == 0) | (k == 15)
    assert np.all(on_face) and np.all((c["cell"] >= 0) & (c["cell"] < 1024))
    assert np.all(c["k"] > 0) and np.all(c["area"] > 0)
    hot = c["temp"] == 45.0
    assert 0 < hot.mean() < 0.4 and np.all(np.abs(c["temp"][~hot] - 22.0) <= 0.5)


def test_object_clouds_lie_on_their_objects():
    rng = np.random.default_rng(3)
    sph = W.ObjectSpec(kind="sphere", radius=0.03)
    p = W.object_cloud(rng, sph, 2000)
    assert p.shape == (2000, 3) and np.allclose(np.linalg.norm(p, axis=1), 0.03, rtol=1e-6)
    box = W.ObjectSpec(kind="box", half=(0.01, 0.02, 0.03))
    b = W.object_cloud(rng, box, 3000).astype(np.float64)
    on = np.isclose(np.abs(b), [0.01, 0.02, 0.03], rtol=1e-6, atol=1e-9).any(axis=1)
    assert np.all(on) and np.all(np.abs(b) <= np.array([0.01, 0.02, 0.03]) + 1e-7)
    assert W.object_cloud(rng, W.ObjectSpec(kind="plane"), 10) is None


def test_marker_pads_have_orthonormal_frames_on_present_links():
    wl = W.config2(n_envs=6, n_objects=2, n_grid=8, faces=(300, 500), seed=9)
    P = wl.pads["pads_per_env"]
    fr = wl.pads["pad_frame"].reshape(-1, 9).astype(np.float64)
    n, t = fr[:, 3:6], fr[:, 6:9]
    assert np.allclose(np.linalg.norm(n, axis=1), 1) and np.allclose(np.linalg.norm(t, axis=1), 1)
    assert np.allclose(np.einsum("ij,ij->i", n, t), 0)
    rows = wl.link_rows.reshape(wl.n_envs, wl.max_links)
    for e in range(wl.n_envs):
        for p in range(P):
            assert rows[e, wl.pads["pad_link"][e, p]] > 0
