"""Pins of the oracle's learned SDF (multiresolution hash encoding + bfloat16
ReLU MLP, output in mm) against facts that do not come from the oracle:

- bfloat16 rounding against torch's float -> bfloat16 conversion;
- level resolutions against the exact integer form of floor(16 * 2^(l/3));
- dense indexing is a bijection, hashed indexing spreads uniformly and
  matches hand-worked products of the encoding's published primes;
- trilinear interpolation is exact at vertices and reproduces affine tables
  on dense levels (read out through a network that passes one feature);
- the MLP is positively homogeneous and invariant to hidden-unit permutation
  (a transposed or misindexed weight matrix breaks these);
- the input gradient and the loss gradients against finite differences (the
  network is piecewise linear in each weight and table entry, so differences
  over one bfloat16 / binary16 spacing are exact away from kinks);
- outside the box, phi(q) = phi(clamp q) + |q - clamp q|;
- Adam against its closed form under a constant gradient.
"""
import numpy as np
import pytest

import oracle
from oracle import NSDF_HIDDEN as H, NSDF_IN as NI, NSDF_LEVELS as NL, NSDF_TABLE as TT

torch = pytest.importorskip("torch")


def f32_to_bf16_bits(x):
    t = torch.tensor(np.asarray(x, np.float32)).to(torch.bfloat16)
    return t.view(torch.int16).numpy().view(np.uint16)


def bf16_bits(a):
    return f32_to_bf16_bits(np.asarray(a, np.float32))


def bf16_vals(bits):
    return (np.asarray(bits, np.uint32) << 16).view(np.float32).astype(np.float64)


def random_net(rng, lo=(-0.02, -0.02, -0.02), hi=(0.02, 0.025, 0.03), table_scale=1.0, out_scale=20.0):
    table = rng.uniform(-table_scale, table_scale, (NL, TT, 2)).astype(np.float16).view(np.uint16)
    w1 = bf16_bits(rng.uniform(-1, 1, (H, NI)) * np.sqrt(6 / (NI + H)))
    w2 = bf16_bits(rng.uniform(-1, 1, (H, H)) * np.sqrt(6 / (2 * H)))
    w3 = bf16_bits(rng.uniform(-1, 1, H) * np.sqrt(6 / (H + 1)) * out_scale)
    return oracle.Nsdf(lo, hi, table, w1, w2, w3)


def inside_points(rng, net, n):
    lo, hi = np.array(net.s.lo[:]), np.array(net.s.hi[:])
    return lo + (hi - lo) * rng.uniform(0.02, 0.98, (n, 3))


# ---------------------------------------------------------------- bfloat16
def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(size=4000) * 10.0 ** rng.integers(-30, 30, 4000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, -3.1415926, 1e-40, 3e38]]).astype(np.float32)
    # exact ties at the bfloat16 spacing (lower 16 bits 0x8000)
    ties = (rng.integers(0, 2 ** 31, 200).astype(np.uint32) & 0xFFFF0000) | 0x8000
    x = np.concatenate([x, ties.view(np.float32)])
    x = x[np.isfinite(x)]
    ref = f32_to_bf16_bits(x)
    got = np.array([oracle.double_to_bf16(float(v)) for v in x], np.uint16)
    assert np.array_equal(got, ref)
    back = np.array([oracle.bf16_to_double(int(b)) for b in ref])
    assert np.array_equal(back, bf16_vals(ref))


# ---------------------------------------------------------------- encoding geometry
def test_resolutions_are_the_exact_geometric_series():
    got = [oracle.nsdf_resolution(l) for l in range(NL)]
    assert got[0] == 16 and got[-1] == 512
    for l, n in enumerate(got):
        # floor(16 * 2^(l/3)) = floor(cbrt(4096 * 2^l)) in exact integers
        assert n ** 3 <= 4096 * 2 ** l < (n + 1) ** 3


def test_dense_levels_are_bijections_hashed_levels_spread():
    for l in range(NL):
        n1 = oracle.nsdf_resolution(l) + 1
        if n1 ** 3 <= TT:
            idx = {oracle.nsdf_index(l, i, j, k) for i in range(n1) for j in range(n1) for k in range(n1)}
            assert len(idx) == n1 ** 3 and max(idx) < n1 ** 3
    # hand-worked hashes at level 4 (the first hashed level): primes 1, 2654435761, 805459861
    assert oracle.nsdf_index(4, 0, 0, 0) == 0
    assert oracle.nsdf_index(4, 1, 0, 0) == 1
    assert oracle.nsdf_index(4, 0, 1, 0) == 0x79B1          # 0x9E3779B1 mod 2^16
    assert oracle.nsdf_index(4, 0, 0, 1) == 0x5795          # 0x30025795 mod 2^16
    assert oracle.nsdf_index(4, 3, 0, 0) == 3
    assert oracle.nsdf_index(4, 1, 1, 0) == 0x79B0          # 1 xor 0x79B1
    rng = np.random.default_rng(1)
    v = rng.integers(0, 513, (20000, 3))
    idx = np.array([oracle.nsdf_index(15, *t) for t in v])
    assert idx.max() < TT
    counts = np.bincount(idx >> 10, minlength=64)
    from scipy import stats
    assert stats.chisquare(counts).pvalue > 1e-4


def _feature_probe_net(lo, hi, table, level, f):
    """A network whose output is enc[2 level + f] when that value is positive."""
    w1 = np.zeros((H, NI), np.float32); w1[0, 2 * level + f] = 1.0
    w2 = np.zeros((H, H), np.float32); w2[0, 0] = 1.0
    w3 = np.zeros(H, np.float32); w3[0] = 1.0
    return oracle.Nsdf(lo, hi, table, bf16_bits(w1), bf16_bits(w2), bf16_bits(w3))


def test_trilinear_exact_at_vertices_and_affine_on_dense_levels():
    rng = np.random.default_rng(2)
    lo, hi = np.array([-0.01, -0.02, 0.0]), np.array([0.03, 0.02, 0.05])
    table = np.zeros((NL, TT, 2), np.float16)
    for l in range(4):                       # dense: feature 0 = 1 + i/64 + j/128 + k/256
        n1 = oracle.nsdf_resolution(l) + 1
        i, j, k = np.meshgrid(np.arange(n1), np.arange(n1), np.arange(n1), indexing="ij")
        e = (i + n1 * (j + n1 * k)).reshape(-1)
        table[l, e, 0] = (1 + i / 64 + j / 128 + k / 256).reshape(-1)
        table[l, e, 1] = (2 - i / 256).reshape(-1)
    table[4:] = rng.uniform(0.5, 2.0, table[4:].shape)
    bits = table.view(np.uint16)
    for l in (0, 2, 3):
        N = oracle.nsdf_resolution(l)
        net = _feature_probe_net(lo, hi, bits, l, 0)
        u = rng.uniform(0, 1, (50, 3))
        phi = net.eval(lo + u * (hi - lo), round=False) * 1e3
        p = u * N
        assert np.allclose(phi, 1 + p[:, 0] / 64 + p[:, 1] / 128 + p[:, 2] / 256, rtol=0, atol=1e-12)
    for l in (4, 9, 15):                     # hashed: exact at vertices
        N = oracle.nsdf_resolution(l)
        net = _feature_probe_net(lo, hi, bits, l, 0)
        v = rng.integers(0, N + 1, (40, 3))
        q = lo + (v / N) * (hi - lo)
        phi = net.eval(q, round=False) * 1e3
        expect = [table[l, oracle.nsdf_index(l, *t), 0].astype(np.float64) for t in v]
        assert np.allclose(phi, expect, rtol=1e-12, atol=0)


# ---------------------------------------------------------------- MLP
def test_mlp_homogeneity_and_permutation_invariance():
    rng = np.random.default_rng(3)
    net = random_net(rng)
    q = inside_points(rng, net, 200)
    base = net.eval(q, round=True)
    n2 = oracle.Nsdf(net.s.lo, net.s.hi, net.table, net.w1, net.w2,
                     bf16_bits(2.0 * bf16_vals(net.w3)))
    assert np.array_equal(n2.eval(q, round=True), 2.0 * base)
    perm1, perm2 = rng.permutation(H), rng.permutation(H)
    n3 = oracle.Nsdf(net.s.lo, net.s.hi, net.table, net.w1[perm1], net.w2[perm2][:, perm1], net.w3[perm2])
    assert np.allclose(n3.eval(q, round=False), net.eval(q, round=False), rtol=1e-12, atol=1e-15)
    assert np.array_equal(n3.eval(q, round=True), base)
    # scaling a hidden unit's input weights by 2 and its output weights by 1/2 changes nothing
    w1 = bf16_vals(net.w1).copy(); w2 = bf16_vals(net.w2).copy()
    w1[5] *= 2.0; w2[:, 5] *= 0.5
    n4 = oracle.Nsdf(net.s.lo, net.s.hi, net.table, bf16_bits(w1), bf16_bits(w2), net.w3)
    assert np.allclose(n4.eval(q, round=False), net.eval(q, round=False), rtol=1e-12, atol=1e-15)


def test_rounding_changes_little():
    rng = np.random.default_rng(4)
    net = random_net(rng)
    q = inside_points(rng, net, 500)
    a, b = net.eval(q, round=True) * 1e3, net.eval(q, round=False) * 1e3
    assert np.max(np.abs(a - b)) < 0.05 * np.max(np.abs(b)) + 1e-3
    assert np.any(a != b)


def test_outside_extension():
    rng = np.random.default_rng(5)
    net = random_net(rng)
    lo, hi = np.array(net.s.lo[:]), np.array(net.s.hi[:])
    q = lo + (hi - lo) * rng.uniform(-0.8, 1.8, (300, 3))
    c = np.clip(q, lo, hi)
    assert np.allclose(net.eval(q, round=True), net.eval(c, round=True) + np.linalg.norm(q - c, axis=1),
                       rtol=0, atol=1e-15)


# ---------------------------------------------------------------- gradients
def test_input_gradient_against_finite_differences():
    rng = np.random.default_rng(6)
    net = random_net(rng)
    q = inside_points(rng, net, 100)
    _, g = net.eval(q, round=False, grad=True)
    h = 1e-9
    bad = 0
    for a in range(3):
        e = np.zeros(3); e[a] = h
        fd = (net.eval(q + e, round=False) - net.eval(q - e, round=False)) / (2 * h)
        ok = np.isclose(fd, g[:, a], rtol=1e-5, atol=1e-9)
        bad += int((~ok).sum())
    assert bad <= 3  # a difference straddling a cell face or a ReLU kink is not a derivative


def _bf16_step(bits, d):
    """the bfloat16 value d spacings away (same sign region)."""
    return np.uint16(int(bits) + d) if bf16_vals([bits])[0] >= 0 else np.uint16(int(bits) - d)


def test_loss_gradients_against_exact_differences():
    rng = np.random.default_rng(7)
    net = random_net(rng)
    q = inside_points(rng, net, 64)
    y = net.eval(q, round=False) * 1e3 + rng.choice([-1, 1], 64) * rng.uniform(0.5, 2.0, 64)
    loss, g1, g2, g3, gt = net.loss_grad(q, y, round=False)

    def loss_with(**over):
        parts = dict(table=net.table, w1=net.w1, w2=net.w2, w3=net.w3)
        parts.update(over)
        n = oracle.Nsdf(net.s.lo, net.s.hi, **parts)
        return n.loss_grad(q, y, round=False)[0]

    checked = 0
    for name, grad, arr in (("w1", g1, net.w1), ("w2", g2, net.w2), ("w3", g3, net.w3)):
        flat = arr.reshape(-1)
        for idx in rng.choice(flat.size, 12, replace=False):
            vals = []
            for d in (-1, 1):
                b = flat.copy(); b[idx] = _bf16_step(flat[idx], d)
                vals.append((bf16_vals([b[idx]])[0], loss_with(**{name: b.reshape(arr.shape)})))
            (wm, lm), (wp, lp) = vals
            w0 = bf16_vals([flat[idx]])[0]
            sl, sr = (loss - lm) / (w0 - wm), (lp - loss) / (wp - w0)
            if not np.isclose(sl, sr, rtol=1e-6, atol=1e-12):
                continue  # a kink between the neighbours
            # (loss differences of ~1e-6 on a loss of ~1 leave ~1e-9 relative of FP64 cancellation)
            assert np.isclose(grad.reshape(-1)[idx], sr, rtol=1e-6, atol=1e-12), (name, idx)
            checked += 1
    # table entries touched by the batch: one binary16 spacing either way
    touched = np.argwhere(gt != 0)
    for l, e, f in touched[rng.choice(len(touched), 20, replace=False)]:
        h0 = net.table[l, e, f].view(np.float16)
        res = []
        for d in (-np.inf, np.inf):
            t2 = net.table.copy()
            hv = np.nextafter(h0, np.float16(d))
            t2[l, e, f] = hv.view(np.uint16)
            res.append((float(hv), loss_with(table=t2)))
        (hm, lm), (hp, lp) = res
        h0 = float(h0)
        sl, sr = (loss - lm) / (h0 - hm), (lp - loss) / (hp - h0)
        if not np.isclose(sl, sr, rtol=1e-6, atol=1e-12):
            continue
        assert np.isclose(gt[l, e, f], sr, rtol=1e-6, atol=1e-12)
        checked += 1
    assert checked >= 30


# ---------------------------------------------------------------- Adam
def test_adam_constant_gradient_closed_form():
    rng = np.random.default_rng(8)
    n = 50
    theta = rng.normal(size=n); t0 = theta.copy()
    m = np.zeros(n); v = np.zeros(n)
    g = rng.normal(size=n) * 10.0 ** rng.integers(-6, 2, n)
    lr, eps = 1e-2, 1e-15
    for t in range(1, 11):
        oracle.adam_step(theta, m, v, g, lr, 0.9, 0.99, eps, t)
    assert np.allclose(theta, t0 - 10 * lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-14)
    # zero gradient, zero state: nothing moves
    th = rng.normal(size=n); th0 = th.copy(); z = np.zeros(n)
    oracle.adam_step(th, np.zeros(n), np.zeros(n), z, lr, 0.9, 0.99, eps, 1)
    assert np.array_equal(th, th0)


def test_contact_normal_stencil_is_exact_on_affine_fields():
    rng = np.random.default_rng(9)
    lo, hi = np.array([-0.01, -0.02, 0.0]), np.array([0.03, 0.02, 0.05])
    table = np.zeros((NL, TT, 2), np.float16)
    n1 = oracle.nsdf_resolution(2) + 1
    i, j, k = np.meshgrid(np.arange(n1), np.arange(n1), np.arange(n1), indexing="ij")
    table[2, (i + n1 * (j + n1 * k)).reshape(-1), 0] = (1 + i / 64 + j / 128 + k / 256).reshape(-1)
    net = _feature_probe_net(lo, hi, table.view(np.uint16), 2, 0)
    N = oracle.nsdf_resolution(2)
    q = lo + (hi - lo) * rng.uniform(0.05, 0.95, (30, 3))
    g = net.normal(q, round=False)
    # phi (m) = 1e-3 (1 + p_x / 64 + p_y / 128 + p_z / 256), p = N (q - lo) / (hi - lo)
    expect = 1e-3 * N * np.array([1 / 64, 1 / 128, 1 / 256]) / (hi - lo)
    assert np.allclose(g, expect[None], rtol=1e-9)


def test_scene_uses_the_network_only_within_1mm_of_contact():
    """A learned-SDF object: grid phi = z (a plane, exact for trilinear
    interpolation), network with zero weights (phi_net = 0).  Probes whose
    grid distance is beyond R + 1 mm read the grid, the others the network."""
    from paper_2606_22332_gb300 import workload as W
    from _scenes import oracle_scene, pad_workload, quiet_params

    lo = np.array([-0.02, -0.02, -0.005], np.float32)
    hi = np.array([0.02, 0.02, 0.02], np.float32)
    dims = (9, 9, 26)
    zs = np.linspace(float(lo[2]), float(hi[2]), dims[2])
    grid = np.broadcast_to(zs[:, None, None], (dims[2], dims[1], dims[0])).astype(np.float32).copy()
    obj = W.ObjectSpec(kind="neural", dims=dims, lo=lo, hi=hi, fp16=False, values=grid, nsdf_lo=lo, nsdf_hi=hi,
                       nsdf_table=np.zeros((NL, TT, 2), np.uint16), nsdf_weights=np.zeros(6208, np.uint16),
                       nsdf_err_mm=0.0)
    heights_over_R = np.array([[5e-3, 2e-3, 1.2e-3, 0.8e-3, 0.3e-3, -0.5e-3]])   # probe height minus R
    wl = pad_workload(-heights_over_R, 1, 6, params=quiet_params(), obj=obj)
    osc = oracle_scene(wl)
    st = osc.new_state(); osc.reset(st, 0)
    o = osc.step(st, wl.inputs(0))
    R = 1e-3
    far = heights_over_R[0] > 1e-3
    h = W.f32(wl.z).astype(np.float64) + 0.01                  # probe height above the plane
    assert np.allclose(o["dist"][far], h[far] - float(np.float32(R)), atol=1e-12)
    assert np.allclose(o["dist"][~far], -float(np.float32(R)), atol=1e-12)   # phi_net = 0
    assert np.allclose(o["depth_clean"][~far], float(np.float32(R)), atol=1e-12)
    assert np.all(o["depth_clean"][far] == 0)
