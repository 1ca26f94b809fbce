"""Raycast depth backend on the GPU against the FP64 oracle ("Two
contact-depth backends").

Meshes: a superquadric and a convex hull of 1,500-2,500 faces. Probes start
from surface samples, moved along the face normal by U(-R, 2R) with a
tangential jitter. Radii are U(0.5, 3) mm, the mesh scale is 1 or 1.3, and
some probes are inactive (R = 0).

The depth is unique and must match within 2e-7 m (FP32 coordinates of
~5 cm objects). The winning face is not unique: a probe nearest an edge or a
vertex is equally near two or more faces. So the GPU's face must be valid:
that face alone reaches the oracle's depth within the same tolerance, and the
returned normal is its unit normal.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle
from paper_2606_22332_gb300 import workload as W

TOL = 2e-7


@pytest.fixture(scope="module")
def tg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_22332_gb300.tg as tg
    return tg


def _probes(rng, V, F, n):
    p, nrm = W.surface_samples(rng, V, F, n)
    R = rng.uniform(0.5e-3, 3e-3, n)
    t = rng.standard_normal((n, 3)) * 3e-4
    q = p + nrm * (rng.uniform(-1, 2, n) * R)[:, None] + t
    R[rng.random(n) < 0.05] = 0.0
    return q, R


@pytest.mark.parametrize("scale", [1.0, 1.3])
def test_raycast_depth_against_the_oracle(tg, scale):
    rng = np.random.default_rng(5)
    objs = W.config1_objects(rng, 2, n_grid=8, faces=(1500, 2500))
    for o in objs:
        V, F = o.verts.astype(np.float32), o.faces.astype(np.int32)
        bvh = tg.MeshBvh(V, F)
        q, R = _probes(rng, V.astype(np.float64) * scale, F, 1500)
        q32 = q.astype(np.float32)
        d, n, f = bvh.depth(torch.as_tensor(q32, device="cuda"), torch.as_tensor(R.astype(np.float32), device="cuda"),
                            scale=scale)
        d, n, f = d.cpu().numpy().astype(np.float64), n.cpu().numpy(), f.cpu().numpy()
        u = -np.ones_like(q)  # the sensing direction only enters the oracle's ray test
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        do, no, fo, _ = oracle.raycast_depth(V, F, scale, q32.astype(np.float64), u,
                                             R.astype(np.float32).astype(np.float64))
        assert np.all(np.abs(d - do) <= TOL), np.abs(d - do).max()
        hit = d > TOL
        assert np.all(f[~(d > 0)] == -1) and np.all(n[~(d > 0)] == 0)
        assert 0.2 < hit.mean() < 0.9
        for i in np.flatnonzero(hit):
            # the GPU's face alone reaches the depth; its normal is that face's normal
            di, ni, _, _ = oracle.raycast_depth(V, F[f[i]:f[i] + 1], scale, q32[i:i + 1].astype(np.float64),
                                                u[i:i + 1], float(np.float32(R[i])))
            assert di[0] >= do[i] - TOL
            assert np.allclose(n[i], ni[0], atol=1e-5)
        bvh.close()


def test_raycast_arguments_are_checked(tg):
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    with pytest.raises(tg.TGError):
        tg.MeshBvh(V, np.array([[0, 1, 3]], np.int32))
    with pytest.raises(tg.TGError):
        tg.MeshBvh(np.array([[0, 0, np.nan], [1, 0, 0], [0, 1, 0]], np.float32), np.array([[0, 1, 2]], np.int32))
    b = tg.MeshBvh(V, np.array([[0, 1, 2]], np.int32))
    q = torch.zeros((1, 3), device="cuda")
    with pytest.raises(tg.TGError):
        b.depth(q, torch.ones(1, device="cuda"), scale=0.0)
    d, n, f = b.depth(torch.tensor([[0.2, 0.2, 5e-4]], device="cuda"), torch.tensor([1e-3], device="cuda"))
    assert abs(float(d[0]) - 5e-4) < 1e-9 and int(f[0]) == 0 and np.allclose(n[0].cpu().numpy(), [0, 0, 1])
    b.close()
