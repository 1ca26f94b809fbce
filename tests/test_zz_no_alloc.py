"""tg_mesh_sdf_noalloc: the mesh distance query for callers that cannot
allocate device memory (an application whose own allocator owns the GPU's
memory, or a path that cannot take cudaMalloc's device-wide synchronisation).

Checked through the C-ABI against tg_mesh_sdf, which allocates its triangle
list per call: two calls in a row on different meshes and point sets (the
second call must not see anything of the first in the shared array), the
size limit, and invalid faces (an out-of-range index or a zero-area face
make every result NaN; the next valid call is unaffected).  This file is
collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2606_22332_gb300 import workload as W


@pytest.fixture(scope="module")
def tg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_22332_gb300.tg as tg
    return tg


def _case(tg, seed, n_points, hull_points, min_faces):
    rng = np.random.default_rng(seed)
    V, F = W.hull_mesh(rng, hull_points, 0.04, min_faces=min_faces)
    q = rng.uniform(-0.035, 0.035, (n_points, 3)).astype(np.float32)
    pts = torch.as_tensor(q).cuda()
    ref_phi, ref_grad = tg.mesh_sdf(V, F, pts)
    Vd = torch.as_tensor(V).cuda().contiguous()
    Fd = torch.as_tensor(F).cuda().contiguous()
    phi = torch.empty(n_points, dtype=torch.float32, device="cuda")
    grad = torch.empty((n_points, 3), dtype=torch.float32, device="cuda")
    tg.mesh_sdf_noalloc(Vd, Fd, pts, phi, grad)
    torch.cuda.synchronize()
    return ref_phi.cpu().numpy(), ref_grad.cpu().numpy(), phi.cpu().numpy(), grad.cpu().numpy()


def test_noalloc_matches_allocating_query_twice(tg):
    # a large mesh, then a smaller one: the second call reuses the shared array
    for seed, npts, hp, mf in ((31, 5000, 200, 6000), (32, 3000, 40, 300)):
        rp, rg, p, g = _case(tg, seed, npts, hp, mf)
        # same kernel, same triangles: the distances are bit-identical
        assert np.array_equal(p.view(np.uint32), rp.view(np.uint32))
        # unit gradients: equal, except where a gradient is a face normal (normalised in
        # FP32 here, in FP64 by the allocating query), which may differ in the last bits
        assert np.abs(g - rg).max() <= 1e-6


def test_noalloc_rejects_meshes_over_the_limit(tg):
    nf = tg.NOALLOC_MAX_FACES + 1
    V = torch.zeros((3, 3), dtype=torch.float32, device="cuda")
    F = torch.zeros((nf, 3), dtype=torch.int32, device="cuda")
    pts = torch.zeros((4, 3), dtype=torch.float32, device="cuda")
    phi = torch.empty(4, dtype=torch.float32, device="cuda")
    with pytest.raises(tg.TGError) as err:
        tg.mesh_sdf_noalloc(V, F, pts, phi)
    assert err.value.status == 1  # TG_ERR_INVALID_ARG


def _run(tg, V, F, q):
    Vd = torch.as_tensor(V).cuda().contiguous()
    Fd = torch.as_tensor(F).cuda().contiguous()
    pts = torch.as_tensor(q).cuda()
    phi = torch.zeros(len(q), dtype=torch.float32, device="cuda")
    grad = torch.zeros((len(q), 3), dtype=torch.float32, device="cuda")
    tg.mesh_sdf_noalloc(Vd, Fd, pts, phi, grad)
    torch.cuda.synchronize()
    return phi.cpu().numpy(), grad.cpu().numpy()


def test_noalloc_invalid_faces_give_nan_then_valid_calls_recover(tg):
    rng = np.random.default_rng(33)
    V, F = W.hull_mesh(rng, 64, 0.04, min_faces=500)
    q = rng.uniform(-0.03, 0.03, (700, 3)).astype(np.float32)
    ref_phi, _ = tg.mesh_sdf(V, F, torch.as_tensor(q).cuda())
    ref_phi = ref_phi.cpu().numpy()
    bad_index = F.copy()
    bad_index[17, 1] = len(V) + 5                 # out of range
    degenerate = F.copy()
    degenerate[3, 2] = degenerate[3, 1]           # two equal corners: zero area
    for Fb in (bad_index, degenerate):
        phi, grad = _run(tg, V, Fb, q)
        assert np.isnan(phi).all() and np.isnan(grad).all()
        # the counter is cleared by the next call: a valid mesh gives the allocating query's distances
        phi, grad = _run(tg, V, F, q)
        assert np.array_equal(phi.view(np.uint32), ref_phi.view(np.uint32))
        assert np.isfinite(grad).all()
