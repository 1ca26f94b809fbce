"""Oracle pins for the raycast contact-depth backend inside the sensor step
(paper, "Probe geometry and contact-depth query", two contact-depth
backends): a mesh object can answer with the raycast backend (the deepest
penetration over the triangles within R of the probe, with that triangle's
normal) instead of its signed distance.

A pad of probes is pressed onto the top face of a cube mesh whose top face
lies where the half-space of the plain pad tests lies:
- over the face interior the raycast step equals the half-space step (depth,
  contact, force) to rounding;
- a probe whose centre is more than R inside the cube has no triangle within
  R: the raycast backend reads no contact, the signed-distance backend reads
  a depth above R;
- at the cube's top edge the deepest feature is shared by two faces with
  different normals: the step flags the tie, reports R minus the distance to
  the edge, and its force lies along one of the two face normals.
"""
import numpy as np

from paper_2606_22332_gb300 import workload as W
from _scenes import oracle_scene, pad_workload
from test_oracle_geometry import cube_mesh

H = 0.02  # half side of the cube


def _top_cube():
    V, F = cube_mesh(H)
    V = W.f32(V - np.array([0.0, 0.0, H], np.float32))   # top face at z = 0
    return W.ObjectSpec(kind="mesh", verts=V, faces=F)


def _params(backend):
    p = W.default_params(7)
    p.update(p_dead=0.0, depth_backend=backend)
    return p


def _step(wl):
    osc = oracle_scene(wl)
    st = osc.new_state()
    osc.reset(st, 0)
    return osc.step(st, wl.inputs(0))


def test_face_interior_matches_the_half_space():
    depths = np.linspace(0.05e-3, 0.95e-3, 20).reshape(4, 5)
    plane = _step(pad_workload(depths, 4, 5, params=_params("sdf")))
    ray = _step(pad_workload(depths, 4, 5, params=_params("raycast"), obj=_top_cube()))
    assert np.allclose(ray["depth_clean"], plane["depth_clean"], rtol=0, atol=1e-15)
    assert np.array_equal(ray["contact_clean"], plane["contact_clean"])
    assert np.allclose(ray["ft_clean"], plane["ft_clean"], rtol=1e-12, atol=1e-15)
    assert np.allclose(ray["depth_clean"], depths.reshape(-1), rtol=0, atol=2e-8)  # float32 probe positions
    assert not ray["depth_tie"].any()


def test_a_probe_deep_inside_has_no_triangle_within_reach():
    depths = np.full((2, 2), 3e-3)              # centres 2 mm below the face, R = 1 mm
    ray = _step(pad_workload(depths, 2, 2, params=_params("raycast"), obj=_top_cube()))
    sdf = _step(pad_workload(depths, 2, 2, params=_params("sdf"), obj=_top_cube()))
    assert np.all(ray["depth_clean"] == 0) and not ray["contact_clean"].any() and np.all(ray["ft_clean"] == 0)
    assert np.allclose(sdf["depth_clean"], 3e-3, atol=1e-12) and sdf["contact_clean"].all()


def test_a_probe_at_the_top_edge_is_a_tie_between_two_normals():
    wl = pad_workload(0.0, 1, 1, params=_params("raycast"), obj=_top_cube())
    off = 0.3e-3                                 # outside the side face and above the top face
    h_link = float(wl.link_pose[0, 0, 2])
    wl.x = W.f32([H + off]); wl.y = W.f32([0.0]); wl.z = W.f32([off - h_link])
    out = _step(wl)
    pen = 1e-3 - np.sqrt(2.0) * off
    assert out["depth_tie"][0] == 1
    assert np.isclose(out["depth_clean"][0], pen, rtol=0, atol=1e-8)  # float32 probe position
    f = out["ft_clean"][:3, 0]
    k = wl.params["k"]
    assert np.isclose(np.linalg.norm(f), k * out["depth_clean"][0], rtol=1e-9)
    assert np.allclose(f / np.linalg.norm(f), [0, 0, 1], atol=1e-9) or np.allclose(f / np.linalg.norm(f), [1, 0, 0],
                                                                                     atol=1e-9)
