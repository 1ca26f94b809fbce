"""Oracle pins for the read delay (paper, "Sensor Noise Model", base noise:
the noisy readout is formed from y_{t - Delta_read}, with optional uniform
jitter).

A flat pad over the half-space is lifted and pressed step by step, so the
clean readings change every step; then:
- with every other knob off, the noisy depth, force/torque and contact bit
  are the clean ones of exactly Delta steps earlier, and the reset state
  (0) before the episode's first Delta steps;
- with gains, hysteresis and crosstalk on, the delayed chain equals the
  undelayed chain shifted by Delta (the chain is linear and time-invariant),
  and a dead taxel reads its stuck value from the first step (the dead
  override is not delayed);
- the jitter draws delays uniform on {Delta .. Delta + J}, one per env and
  step, and the readout follows the drawn delay;
- a reset clears the delayed history.
"""
import numpy as np
from scipy import stats

import oracle
from paper_2606_22332_gb300 import workload as W
from _scenes import oracle_scene, pad_workload

ROWS, COLS, STEPS = 4, 5, 14


def _quiet(seed=5, **kw):
    p = W.default_params(seed)
    p.update(p_dead=0.0, chi=0.0, noise=dict(depth=W.noise_group(), ft=W.noise_group(), prox=W.noise_group()))
    p.update(kw)
    return p


def _heights(rng):
    # link heights: the probes (R = 1 mm) go from 0.5 mm clear to 2 mm deep
    return 0.01 + rng.uniform(-2e-3, 0.5e-3, STEPS)


def _run(params, heights, episode=0, reset_at=None):
    wl = pad_workload(np.linspace(0, 1e-3, ROWS * COLS).reshape(ROWS, COLS), ROWS, COLS, params=params)
    osc = oracle_scene(wl)
    st = osc.new_state()
    osc.reset(st, episode)
    outs = []
    for t, h in enumerate(heights):
        if reset_at is not None and t == reset_at:
            osc.reset(st, episode)
        inp = wl.inputs(t)
        inp["link_pose"] = wl.link_pose.copy()
        inp["link_pose"][0, 0, 2] = h
        o = osc.step(st, inp)
        outs.append({k: np.array(o[k], copy=True) for k in ("depth_clean", "depth_noisy", "ft_clean", "ft_noisy",
                                                             "contact_clean", "contact_noisy")})
    return outs, st


def test_readout_lags_by_exactly_delta():
    rng = np.random.default_rng(1)
    h = _heights(rng)
    for delta in (1, 3):
        outs, _ = _run(_quiet(read_delay=delta), h)
        assert any(o["depth_clean"].max() > 0 for o in outs) and any(o["contact_clean"].any() for o in outs)
        for t, o in enumerate(outs):
            if t < delta:
                assert np.all(o["depth_noisy"] == 0) and np.all(o["ft_noisy"] == 0)
                assert not o["contact_noisy"].any()
            else:
                src = outs[t - delta]
                assert np.array_equal(o["depth_noisy"], src["depth_clean"])
                assert np.array_equal(o["ft_noisy"], src["ft_clean"])
                assert np.array_equal(o["contact_noisy"], src["contact_clean"])
            # the clean readout is never delayed
            assert np.array_equal(o["depth_clean"], _run(_quiet(), h[: t + 1])[0][t]["depth_clean"])


def test_delayed_chain_is_the_undelayed_chain_shifted():
    rng = np.random.default_rng(2)
    h = _heights(rng)
    groups = dict(depth=W.noise_group(beta=0.1, tau=0.05, gain_lo=0.8, gain_hi=1.2),
                  ft=W.noise_group(beta=0.1, tau=0.05, gain_lo=0.8, gain_hi=1.2, stuck_lo=0.3, stuck_hi=0.7),
                  prox=W.noise_group())
    base = _quiet(seed=11, chi=0.05, p_dead=0.25, noise=groups)
    a, st = _run(base, h)
    b, _ = _run(dict(base, read_delay=3), h)
    dead = ((st["flags"] >> 1) & 1).astype(bool)
    assert 0 < dead.sum() < ROWS * COLS
    for t in range(STEPS):
        # dead taxels: the stuck readout from the first step, delay or not
        assert np.array_equal(b[t]["ft_noisy"][:, dead], a[t]["ft_noisy"][:, dead])
        if t >= 3:
            assert np.array_equal(b[t]["depth_noisy"][~dead], a[t - 3]["depth_noisy"][~dead])
            assert np.array_equal(b[t]["ft_noisy"][:, ~dead], a[t - 3]["ft_noisy"][:, ~dead])
            assert np.array_equal(b[t]["contact_noisy"], a[t - 3]["contact_noisy"])
        else:
            assert np.all(b[t]["depth_noisy"][~dead] == 0)


def test_jitter_draws_uniform_delays_and_the_readout_follows_them():
    p = _quiet(read_delay=1, read_jitter=2)
    d = np.array([[oracle.read_delay(p, e, t) for t in range(200)] for e in range(50)])
    assert set(np.unique(d)) == {1, 2, 3}
    counts = np.bincount(d.ravel(), minlength=4)[1:]
    assert stats.chisquare(counts).pvalue > 1e-4
    # one draw per env and step: consecutive steps are not all equal
    assert (np.diff(d[0]) != 0).any()
    h = _heights(np.random.default_rng(3))
    outs, _ = _run(p, h)
    for t, o in enumerate(outs):
        dt = oracle.read_delay(p, 0, t)
        want = outs[t - dt]["depth_clean"] if t >= dt else np.zeros(ROWS * COLS)
        assert np.array_equal(o["depth_noisy"], want)


def test_reset_clears_the_delayed_history():
    h = _heights(np.random.default_rng(4))
    outs, _ = _run(_quiet(read_delay=2), h, reset_at=6)
    assert np.any(outs[5]["depth_noisy"] > 0) or np.any(outs[4]["depth_clean"] > 0)
    for t in (6, 7):
        assert np.all(outs[t]["depth_noisy"] == 0) and not outs[t]["contact_noisy"].any()
    assert np.array_equal(outs[8]["depth_noisy"], outs[6]["depth_clean"])
