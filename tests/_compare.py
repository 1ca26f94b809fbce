"""Element-by-element comparison of the CUDA path with the FP64 oracle.

Tolerances (stated for the hot path):
  contact flags, dead masks, RNG-driven bits   bit-exact
  depth, noisy depth, surface distance         |d_gpu - d_ora| <= 1e-5 m
  force/torque (clean and noisy)               per 3-vector (force, torque):
                                               |f_gpu - f_ora| <= 1e-4 |f_ora| + 1e-6
                                               (Euclidean norms; a float32 component of
                                               a 20 N vector is itself only resolved to
                                               ~2e-6 N, so the bound is on the vector)
  per-link sums                                the per-taxel bound summed over the
                                               link: 1e-4 sum|f_j| + 1e-6 n_link
Contact bits are decided by the depth against eta_on / eta_off; a taxel
whose oracle depth lies within BAND of a threshold may legitimately differ
(the two sides round differently) and is counted instead of failed; the
count must stay below 1e-4 of the active taxels.
"""
from __future__ import annotations

import numpy as np

F_REL, F_ABS, D_ABS = 1e-4, 1e-6, 1e-5
BAND = 1e-9


def gpu_outputs(scene):
    import paper_2606_22332_gb300.tg as tg

    return {
        "flags": scene.read(tg.CH_STATE_FLAGS),
        "contact_clean": scene.read(tg.CH_CONTACT, False),
        "contact_noisy": scene.read(tg.CH_CONTACT, True),
        "depth_clean": scene.read(tg.CH_DEPTH, False),
        "depth_noisy": scene.read(tg.CH_DEPTH, True),
        "ft_clean": scene.read(tg.CH_FORCE_TORQUE, False),
        "ft_noisy": scene.read(tg.CH_FORCE_TORQUE, True),
        "link_sums": scene.read(tg.CH_LINK_WRENCH),
        "link_counts": scene.read(tg.CH_LINK_COUNT),
        "dist": scene.read(tg.CH_DIST) if scene.sensors & tg.TG_SENSOR_DIST else None,
    }


def compare_step(gpu, ora, ostate, params, wl, active=None, where="", tol=None, exclude=None, ambiguous=None):
    """Assert the CUDA step matches the oracle step; returns error statistics.

    tol overrides the bounds (keys d_abs, f_rel, f_abs, band, band_noisy,
    agg_d) where the path has a larger stated error, e.g. a learned SDF's
    bfloat16 roundings; each value is a scalar or a per-taxel array, so the
    taxels of grid-object envs keep the bounds above while those of
    learned-SDF envs get their own.  tol["f_outliers"] is the fraction of
    active taxels whose force / torque may exceed its bound (normals that are
    discontinuous at the point, as a learned SDF's are at every hash-grid
    cell face); those taxels are returned in stats["outliers"], counted in
    stats["n_outliers"], and, like the taxels in `exclude` (earlier
    outliers, whose state carries the difference), enter their links' sums
    with their own bound widened to the error they show.  No link is skipped.
    `ambiguous` marks taxels on a decision boundary of the method where the
    two sides may legitimately take different branches (a learned SDF's
    near-field switch, decided in FP32 on the GPU and FP64 here): they are
    left out of every per-taxel check, counted in stats["ambiguous"], enter
    their links' sums with the error they show, and the oracle adopts their
    contact bits."""
    t = {"d_abs": D_ABS, "f_rel": F_REL, "f_abs": F_ABS, "band": BAND, "agg_d": 0.0, "f_outliers": 0.0}
    t.update(tol or {})
    stats = {}
    R = wl.R
    T = len(R)

    def per_taxel(v):
        return np.broadcast_to(np.asarray(v, np.float64), (T,))

    D_ABS_, F_REL_, F_ABS_, BAND_ = (per_taxel(t[k]) for k in ("d_abs", "f_rel", "f_abs", "band"))
    AGG_D = per_taxel(t["agg_d"])
    amb = np.zeros(T, bool) if ambiguous is None else np.asarray(ambiguous, bool)
    stats["ambiguous"] = int(amb.sum()) if ambiguous is not None else 0
    act = R > 0 if active is None else active
    n_act = int(act.sum())
    # dead masks: bit-exact
    assert np.array_equal((gpu["flags"] >> 1) & 1, (ostate["flags"] >> 1) & 1), f"{where}: dead masks differ"
    # contact bits, with the threshold band
    d_or = ora["depth_clean"]
    band = (np.abs(d_or - params["eta_on"]) < BAND_) | (np.abs(d_or - params["eta_off"]) < BAND_)
    # the noisy bit decides on the noisy readout's depth (with probe-radius noise up to rho from the
    # clean one): tol["band_noisy"] widens its band where the path's phi carries a stated error
    bn = per_taxel(t.get("band_noisy", t["band"]))
    band_n = (np.abs(d_or - params["eta_on"]) < bn) | (np.abs(d_or - params["eta_off"]) < bn)
    for k, b in (("contact_clean", band), ("contact_noisy", band_n)):
        bad = (gpu[k] != ora[k]) & ~b & ~amb
        if bad.any():
            i = np.flatnonzero(bad)[:5]
            raise AssertionError(f"{where}: {k} differs at {i}: gpu {gpu[k][i]} oracle {ora[k][i]} oracle depth "
                                 f"{d_or[i]} gpu depth {gpu['depth_clean'][i]} band {BAND_[i]} "
                                 f"oracle flags {ostate['flags'][i]} gpu flags {gpu['flags'][i]}")
    mis = (gpu["contact_clean"] != ora["contact_clean"]) & band & ~amb
    nb = int(mis.sum())
    # the 1e-4 share applies to the plain bound's band; a wider stated band
    # (a learned SDF's) tolerates its mismatches and counts them
    nb_plain = int((mis & (BAND_ <= BAND)).sum())
    assert nb_plain <= max(1, 1e-4 * n_act), f"{where}: {nb_plain} banded contact mismatches"
    stats["banded"] = nb
    # the oracle adopts the GPU's contact bits where they differ inside the
    # band, so both sides' Schmitt states stay in step (the next step decides
    # from the previous bit)
    for bit, k, b in ((1, "contact_clean", band), (4, "contact_noisy", band_n)):
        sync = (gpu[k] != ora[k]) & (b | amb)
        if sync.any():
            ostate["flags"][sync] = (ostate["flags"][sync] & ~np.uint8(bit)) | (gpu["flags"][sync] & np.uint8(bit))
    # depth
    for k in ("depth_clean", "depth_noisy"):
        err = np.where(amb, 0.0, np.abs(gpu[k].astype(np.float64) - ora[k]))
        stats[k] = float(err.max()) if err.size else 0.0
        over = err > D_ABS_
        assert not over.any(), f"{where}: {k} err {err[over].max():.3e} > bound at {np.flatnonzero(over)[:5]}"
    if gpu.get("dist") is not None:
        err = np.where(amb, 0.0, np.abs(gpu["dist"].astype(np.float64) - ora["dist"]))
        stats["dist"] = float(err.max()) if err.size else 0.0
        over = err > D_ABS_
        assert not over.any(), f"{where}: dist err {err[over].max():.3e} > bound"
    # force/torque, per 3-vector
    skip = (np.zeros(T, bool) if exclude is None else exclude.copy()) | amb
    bad = np.zeros(T, bool)
    bound = {}  # per (readout, part): each taxel's share of its link-sum bound
    for k in ("ft_clean", "ft_noisy"):
        g, o = gpu[k].astype(np.float64), ora[k]
        for part, rows in (("force", slice(0, 3)), ("torque", slice(3, 6))):
            err = np.linalg.norm(g[rows] - o[rows], axis=0)
            tol_ = F_REL_ * np.linalg.norm(o[rows], axis=0) + F_ABS_
            ratio = np.where(skip, 0.0, err / tol_)
            key = f"{k}_{part}"
            stats[key] = float(ratio.max()) if ratio.size else 0.0
            stats[key + "_abs"] = float(err.max()) if err.size else 0.0
            bad |= ratio > 1.0
            bound[(k, part)] = (tol_, err)
    stats["outliers"] = bad
    stats["n_outliers"] = int(bad.sum())
    if bad.sum() > t["f_outliers"] * n_act:
        k = "ft_clean" if (np.linalg.norm(gpu["ft_clean"].astype(np.float64) - ora["ft_clean"], axis=0)[bad] > 0).any() else "ft_noisy"
        i = int(np.flatnonzero(bad)[0])
        raise AssertionError(f"{where}: {int(bad.sum())} taxels outside the force/torque bound, e.g. taxel {i}: "
                             f"gpu {gpu[k][:, i]} oracle {ora[k][:, i]} depth {d_or[i]:.3e}")
    widen = skip | bad
    link_b = {}
    for (k, part), (tol_, err) in bound.items():
        link_b[(k, part)] = np.where(widen, np.maximum(tol_, err), tol_)
    # per-link sums: the per-taxel bounds summed over the link
    L = wl.max_links
    off = wl.taxel_offsets
    ls_g, ls_o = gpu["link_sums"].astype(np.float64), ora["link_sums"]
    worst = 0.0
    for e in range(wl.n_envs):
        t0 = int(off[e])
        for l in range(L):
            r, c = wl.link_rows[e * L + l], wl.link_cols[e * L + l]
            nl = int(r * c)
            if nl == 0:
                continue
            sl = slice(t0, t0 + nl)
            t0 += nl
            rec = e * L + l
            for k, cols_ in (("ft_clean", range(0, 6)), ("ft_noisy", range(6, 12))):
                for j, col in enumerate(cols_):
                    tol = link_b[(k, "force" if j < 3 else "torque")][sl].sum()
                    err = abs(ls_g[rec, col] - ls_o[rec, col])
                    worst = max(worst, err / tol)
                    assert err <= tol, f"{where}: link sum env {e} link {l} col {col}: {ls_g[rec, col]} vs {ls_o[rec, col]}"
            for col, dsrc in ((12, "depth_clean"), (15, "depth_noisy")):
                # an ambiguous taxel adds the depth difference it shows
                d_amb = np.abs(gpu[dsrc][sl].astype(np.float64) - ora[dsrc][sl])[amb[sl]].sum()
                for j in range(3):
                    tol = 1e4 * (AGG_D[sl].sum() + (np.maximum(1e-4, F_REL_[sl]) * np.abs(ora[dsrc][sl])).sum()
                                 + d_amb) + F_ABS_[sl].sum()
                    err = abs(ls_g[rec, col + j] - ls_o[rec, col + j])
                    assert err <= tol, f"{where}: agg_force env {e} link {l}: {ls_g[rec, col + j]} vs {ls_o[rec, col + j]}"
    stats["link_sums"] = worst
    # contact counts: equal on every link without a banded or ambiguous taxel
    if nb == 0:
        link_amb = np.zeros(wl.n_envs * L, bool)
        t0 = 0
        for rec in range(wl.n_envs * L):
            nl = int(wl.link_rows[rec] * wl.link_cols[rec])
            link_amb[rec] = amb[t0:t0 + nl].any()
            t0 += nl
        diff = np.any(gpu["link_counts"] != ora["link_counts"], axis=1) & ~link_amb
        assert not diff.any(), f"{where}: link contact counts differ at links {np.flatnonzero(diff)[:5]}"
    return stats
