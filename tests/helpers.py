"""Comparison of CUDA search results with the FP64 oracle.

Rule (the parity bar): kept-epoch masks and top-K trajectory indices must match exactly; LH' and
alpha within 1e-4 relative.  LH' is a significance in units of sigma, and FP32 sums of psi that
cancel lose relative accuracy as LH' -> 0, so the relative scale is floored at LH' = 1: the
bound is |dL| <= 1e-4 max(|L|, 1) and, since alpha = L / sqrt(sum phi), |d alpha| <=
1e-4 |alpha| max(1, 1/|L|).  Every selection in the paper's regime (LH' >= 7) is purely relative.

FP32 against FP64 can only disagree on decisions that sit within rounding of a boundary (reading
R6), so a difference is accepted only where the oracle itself shows one:
  * a near-tie: two LH' within 1e-5 relative at the point where the lists differ, or an LH'
    within 1e-5 of lh_min;
  * a clip bound: a trajectory whose lightcurve comes within 1e-5 max(sigma_G, |median|) of a
    clip bound (oracle.clip_margin).  Either keep decision is then correct; where the GPU's mask
    differs from the oracle's, its LH' and alpha must equal the FP64 sums over the GPU's own
    kept epochs.
Such pixels are counted and the test asserts the count stays tiny.  The clip-bound rule needs the
search inputs (ctx); without them any mask difference fails.
"""
import numpy as np

REL = 1e-4
TIE = 1e-5
CLIP_TIE = 1e-5


def _near(a, b, rel=TIE):
    return abs(a - b) <= rel * max(abs(a), abs(b), 1e-30)


def gpu_result_numpy(res):
    out = {}
    for k in ("lh", "flux", "idx", "nvalid", "nkept", "mask"):
        a = res[k].cpu().numpy()
        if k in ("nvalid", "nkept"):
            a = a.view(np.uint16).astype(np.int64)
        if k == "mask":
            a = a.view(np.uint32)
        out[k] = a
    return out


def search_ctx(psi, phi, times, vx, vy, params, window=None):
    """The inputs of a search, for the clip-bound rule: planes, epoch times, velocities, the
    oracle's parameter dict and the (x_lo, x_hi, y_lo, y_hi) window the results cover."""
    T, H, W = psi.shape
    return dict(psi=np.asarray(psi, np.float64), phi=np.asarray(phi, np.float64),
                times=np.asarray(times, np.float64), vx=np.asarray(vx, np.float32),
                vy=np.asarray(vy, np.float32), params=dict(params),
                window=tuple(window) if window is not None else (0, W, 0, H))


def _margin(ctx, y, x, j):
    """oracle.clip_margin of trajectory j at window pixel (y, x)."""
    import oracle
    x_lo, _, y_lo, _ = ctx["window"]
    return oracle.clip_margin(ctx["psi"], ctx["phi"], ctx["times"], x_lo + x, y_lo + y,
                              ctx["vx"][j], ctx["vy"][j], ctx["params"])


def _sums_under_mask(ctx, y, x, j, mask_words):
    """FP64 LH' and alpha of trajectory j at window pixel (y, x) over the epochs of a kept mask."""
    import oracle
    x_lo, _, y_lo, _ = ctx["window"]
    psi, phi, times = ctx["psi"], ctx["phi"], ctx["times"]
    T, H, W = psi.shape
    ox, oy = oracle.track_offsets(times, ctx["vx"][j:j + 1], ctx["vy"][j:j + 1])
    sp = sf = 0.0
    for t in range(T):
        if not (int(mask_words[t >> 5]) >> (t & 31)) & 1:
            continue
        xx, yy = x_lo + x + int(ox[0, t]), y_lo + y + int(oy[0, t])
        sp += psi[t, yy, xx]
        sf += phi[t, yy, xx]
    if not sf > 0:
        return np.nan, np.nan
    return sp / np.sqrt(sf), sp / sf


def _values_ok(gl, ol, gf, of):
    floor = max(abs(ol), 1.0)
    if abs(gl - ol) > REL * floor:
        return False
    scale = max(abs(of) * max(1.0, 1.0 / max(abs(ol), 1e-30)), 1e-30)
    return abs(gf - of) <= REL * scale


def compare_search(g, o, lh_min, max_ambiguous=0.001, ctx=None, counts=None):
    """g: numpy view of the GPU result; o: oracle result; ctx: search_ctx(...) of the same call
    (enables the clip-bound rule).  Returns the number of ambiguous pixels; raises AssertionError
    on a real mismatch.  counts (a dict, optional) receives the ambiguous pixels by kind."""
    assert g["idx"].shape == o["idx"].shape, (g["idx"].shape, o["idx"].shape)
    wy, wx, K = o["idx"].shape
    kinds = {"lh_tie": 0, "clip_bound_list": 0, "clip_bound_mask": 0}
    same = (g["idx"] == o["idx"]).all(axis=2)
    bad = []
    for y, x in zip(*np.nonzero(~same)):
        gi, oi = g["idx"][y, x], o["idx"][y, x]
        gl, ol = g["lh"][y, x], o["lh"][y, x]
        ok = True
        for s in range(K):
            if gi[s] == oi[s]:
                continue
            # accept only a near-tie in the oracle's own values or at the threshold
            cands = [ol[s]] if oi[s] >= 0 else []
            if gi[s] >= 0:
                cands.append(gl[s])
            tie = False
            for L in cands:
                if _near(L, lh_min):
                    tie = True
                for s2 in range(K):
                    if s2 != s and oi[s2] >= 0 and _near(L, ol[s2]):
                        tie = True
            if not tie:
                ok = False
                break
        if ok:
            kinds["lh_tie"] += 1
            continue
        # a trajectory of either list, from the first difference on, at a clip bound
        if ctx is not None:
            first = int(np.argmax(gi != oi))
            trajs = {int(j) for j in np.concatenate([gi[first:], oi[first:]]) if j >= 0}
            if any(_margin(ctx, y, x, j) <= CLIP_TIE for j in trajs):
                kinds["clip_bound_list"] += 1
                continue
        bad.append((y, x, gi.tolist(), oi.tolist(), gl.tolist(), ol.tolist()))
    assert not bad, "top-K mismatch at %d pixels, first: %s" % (len(bad), bad[:3])
    # where the lists agree: values and masks
    f = same[..., None] & (o["idx"] >= 0)
    if f.any():
        mism = (g["mask"] != o["mask"]).any(axis=-1) | (g["nkept"] != o["nkept"])
        mism &= f
        clip_pix = set()
        for y, x, s in zip(*np.nonzero(mism)):
            j = int(o["idx"][y, x, s])
            assert ctx is not None, "kept masks differ at (%d, %d) slot %d" % (y, x, s)
            m = _margin(ctx, y, x, j)
            assert m <= CLIP_TIE, ("kept masks differ at (%d, %d) slot %d, trajectory %d, with "
                                   "no epoch within %g of a clip bound (margin %.3g)"
                                   % (y, x, s, j, CLIP_TIE, m))
            L, A = _sums_under_mask(ctx, y, x, j, g["mask"][y, x, s])
            assert _values_ok(g["lh"][y, x, s], L, g["flux"][y, x, s], A), \
                "LH'/alpha of the GPU's own kept set at (%d, %d) slot %d" % (y, x, s)
            clip_pix.add((int(y), int(x)))
        kinds["clip_bound_mask"] = len(clip_pix)
        f2 = f & ~mism
        gl, ol = g["lh"][f2], o["lh"][f2]
        floor = np.maximum(np.abs(ol), 1.0)
        rel = np.abs(gl - ol) / floor
        assert rel.size == 0 or rel.max() <= REL, "LH' rel err %.3g" % rel.max()
        gf, of = g["flux"][f2], o["flux"][f2]
        scale = np.maximum(np.abs(of) * np.maximum(1.0, 1.0 / np.maximum(np.abs(ol), 1e-30)),
                           1e-30)
        relf = np.abs(gf - of) / scale
        assert relf.size == 0 or relf.max() <= REL, "alpha rel err %.3g" % relf.max()
        assert np.array_equal(g["nvalid"][f], o["nvalid"][f])
    empty = same[..., None] & (o["idx"] < 0)
    assert np.all(np.isneginf(g["lh"][empty]))
    ambiguous = sum(kinds.values())
    if counts is not None:
        counts.update(kinds)
    assert ambiguous <= max(1, max_ambiguous * wy * wx), "too many ambiguous pixels: %s" % kinds
    return ambiguous
