"""Comparison of GPU hit records with the FP64 oracle (shared by GPU tests).

Rule (the tolerance the method is held to): a ray's outcome is its hit voxel
or MISS.  Rays the oracle does not flag as ties must match it exactly in
outcome and RGBA, and in entry face; rays whose competing crossings lie within
1e-6 of the volume extent (oracle.classify) may return any outcome reachable
under those near-ties, and those that differ from the oracle's primary answer
are counted and must stay under 1e-5 of the rays.  Hit t must agree within
1e-5 relative (absolute 1e-5 below 1).
"""
import numpy as np

import oracle
import paper_2410_14128_b300 as vx

T_REL = 1e-5
TIE_FRACTION = 1e-5


def gpu_keys(h, dims, layout=vx.HIT_FULL):
    nx, ny, _ = dims
    if layout == vx.HIT_FULL:
        hit = h["status"] == vx.STATUS_HIT
        k = h["x"].astype(np.int64) + nx * (h["y"].astype(np.int64) + ny * h["z"].astype(np.int64))
        return np.where(hit, k, -1), h["status"]
    k = np.where(h["idx"] == 0xFFFFFFFF, -1, h["idx"].astype(np.int64))
    return k, np.where(k >= 0, vx.STATUS_HIT, vx.STATUS_MISS)


def compare(grid, rays, h, layout=vx.HIT_FULL, ref=None, ties=None, palette=None):
    """Returns a dict of counts; raises AssertionError when the rule fails.
    grid: uint32 RGBA grid, or uint8 palette indices with `palette`."""
    nz, ny, nx = grid.shape
    dims = (nx, ny, nz)
    if ref is None:
        ref, _ = oracle.trace(grid, rays) if palette is None else oracle.trace_pal(grid, palette, rays)
    rk = np.where(ref["status"] == oracle.HIT,
                  ref["x"].astype(np.int64) + nx * (ref["y"].astype(np.int64) + ny * ref["z"].astype(np.int64)), -1)
    gk, gst = gpu_keys(h, dims, layout)
    # invalid rays are reported as such
    inv = ref["status"] == oracle.INVALID
    if layout == vx.HIT_FULL:
        assert np.array_equal(gst[inv], np.full(inv.sum(), vx.STATUS_INVALID)), "invalid rays"
        assert not np.any(gst == vx.STATUS_ERROR), "rays hit the iteration cap"
    mism = (gk != rk) & ~inv
    n_mis = int(mism.sum())
    n_tie = 0
    n_tie_bad = 0
    if n_mis:
        if ties is None:
            ties = oracle.classify(grid, rays) if palette is None else oracle.classify_pal(grid, palette, rays)
        idx = np.nonzero(mism)[0]
        for i in idx:
            if ties["tie"][i]:
                n_tie += 1
                alts = set(ties["alt"][i][: ties["n_alt"][i]].tolist())
                if gk[i] not in alts and not ties["overflow"][i]:
                    n_tie_bad += 1
        non_tie = n_mis - n_tie
        assert non_tie == 0, f"{non_tie} non-tie rays differ from the oracle, e.g. ray {idx[:5].tolist()}"
        assert n_tie_bad == 0, f"{n_tie_bad} tie rays return an unreachable outcome"
        assert n_tie <= max(TIE_FRACTION * len(rays), 0), f"{n_tie} tie rays differ (limit {TIE_FRACTION})"
    both = (gk == rk) & (rk >= 0)
    t_ref = ref["t"][both]
    t_gpu = h["t"][both].astype(np.float64)
    err = np.abs(t_gpu - t_ref) / np.maximum(np.abs(t_ref), 1.0)
    assert err.size == 0 or err.max() <= T_REL, f"t error {err.max()}"
    if layout == vx.HIT_FULL:
        assert np.array_equal(h["rgba"][both], ref["rgba"][both]), "rgba"
        same_face = h["face"][both].astype(np.int64) == ref["face"][both]
        assert same_face.all(), f"{(~same_face).sum()} faces differ"
        miss = (rk == -1) & ~inv
        assert np.all(np.isinf(h["t"][miss]))
    return {"rays": len(rays), "hits": int((rk >= 0).sum()), "mismatch": n_mis, "tie_mismatch": n_tie,
            "t_err_max": float(err.max()) if err.size else 0.0}
