"""Sub-pixel trajectory evaluation, its backward kernel and the Adam refinement, against the FP64
oracle (oracle.traj_eval_subpixel, traj_vjp, refine_adam) and FP64 central finite differences.

Inputs are seeded likelihood planes drawn directly (synth.make_likelihood_stack: movers at real
starts, half of them off the velocity grid); candidate tracks are formed here from the injected
movers (the grid velocity nearest to the truth at the rounded start, as a search reports it, and
perturbed truths) plus random tracks, some reaching past the image edges.  Kept sets are random
masks.  No input comes from the CUDA path.

Tolerances:
  L, alpha       1e-4 relative (floored at |L| = 1 as in the search parity tests).
  dL/dparams     against the oracle gradient: |d| <= 1e-4 max(|L|, 1) per pixel (positions) and
                 per pixel per unit of time x the time span (velocities), the forward tolerance
                 carried to a derivative on the pixel scale; against FP64 central differences
                 (h = 1e-3 px and 1e-3 px per unit time, tracks clear of cell edges): relative
                 error below 1e-3 of max(|fd|, 0.01 max(|L|, 1)).
  dL/dpsi, dphi  accumulated over all candidates with random upstream weights: 1e-5 of the
                 largest entry (float32 atomics sum a handful of terms per pixel).
  refine         after 20 Adam steps the float32 gradient (relative error ~1e-7) can still move an
                 epoch across a bilinear cell edge that FP64 just misses, after which the two
                 ascents follow different pieces; at least 98% of candidates must agree within
                 1e-3 (px, px per unit time), every returned L must be the oracle's L at the
                 returned params, and after one step (a move of exactly +-lr) all must agree.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2109_03296_b300 as kb
from synth import make_likelihood_stack

pytestmark = pytest.mark.gpu


def _d(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _kept_words(keep):
    n, T = keep.shape
    kw = np.zeros((n, (T + 31) // 32), np.uint32)
    for t in range(T):
        kw[:, t // 32] |= keep[:, t].astype(np.uint32) << np.uint32(t % 32)
    return kw


def _case(T=26, H=384, W=768, n_movers=20, n_rand=200, seed=11, keep_frac=0.85):
    psi, phi, times, vx, vy, mv = make_likelihood_stack("decam", H=H, W=W, T=T,
                                                        n_movers=n_movers, seed=seed)
    rng = np.random.default_rng(seed + 1)
    P = []
    for i in range(n_movers):
        g = np.argmin((vx - mv["vx"][i]) ** 2 + (vy - mv["vy"][i]) ** 2)
        P.append([math.floor(mv["x0"][i] + 0.5), math.floor(mv["y0"][i] + 0.5), vx[g], vy[g]])
        P.append([mv["x0"][i] + rng.normal(0, 0.3), mv["y0"][i] + rng.normal(0, 0.3),
                  mv["vx"][i] + rng.normal(0, 1.0), mv["vy"][i] + rng.normal(0, 1.0)])
    for _ in range(n_rand):
        k = rng.integers(len(vx))
        P.append([rng.uniform(-3, W + 2), rng.uniform(-3, H + 2), vx[k], vy[k]])
    P = np.array(P, np.float32)
    kw = _kept_words(rng.random((len(P), T)) < keep_frac)
    return dict(psi=psi, phi=phi, psi64=psi.astype(np.float64), phi64=phi.astype(np.float64),
                times=times, P=P, kw=kw, rng=rng, movers=mv, vx=vx, vy=vy)


@pytest.fixture(scope="module", params=[26, 45], ids=["T26", "T45"])
def case(request):
    return _case(T=request.param)


def _gpu(c):
    return _d(c["psi"]), _d(c["phi"]), _d(c["P"]), _d(c["kw"].view(np.int32))


def test_traj_eval_matches_oracle(cuda_device, case):
    c = case
    psi, phi, P, kw = _gpu(c)
    lh, fl, g = (a.cpu().numpy() for a in kb.traj_eval(psi, phi, c["times"], P, kw, grad=True))
    span = c["times"][-1] - c["times"][0]
    n_nan = 0
    for i in range(len(c["P"])):
        L, A, G = oracle.traj_eval_subpixel(c["psi64"], c["phi64"], c["times"], c["kw"][i],
                                            *c["P"][i].astype(np.float64))
        if not np.isfinite(L):
            assert np.isnan(lh[i]) and np.isnan(fl[i]) and not g[i].any()
            n_nan += 1
            continue
        s = max(abs(L), 1.0)
        assert abs(lh[i] - L) <= 1e-4 * s, (i, lh[i], L)
        assert abs(fl[i] - A) <= 1e-4 * abs(A) * max(1.0, 1.0 / max(abs(L), 1e-30)), (i, fl[i], A)
        tol = 1e-4 * s * np.array([1.0, 1.0, span, span])
        assert np.all(np.abs(g[i] - G) <= tol), (i, g[i], G)
    assert n_nan < 0.1 * len(c["P"])


def test_traj_gradient_against_fp64_finite_differences(cuda_device, case):
    c = case
    psi, phi, P, kw = _gpu(c)
    _, _, g = kb.traj_eval(psi, phi, c["times"], P, kw, grad=True)
    g = g.cpu().numpy()
    h = 1e-3
    dts = c["times"] - c["times"][0]
    checked = 0
    for i in range(len(c["P"])):
        p = c["P"][i].astype(np.float64)
        xs, ys = p[0] + p[2] * dts, p[1] + p[3] * dts
        if min(np.abs(xs - np.round(xs)).min(), np.abs(ys - np.round(ys)).min()) < 4 * h * (
                1 + dts.max()):
            continue
        L0 = oracle.traj_eval_subpixel(c["psi64"], c["phi64"], c["times"], c["kw"][i], *p,
                                       grad=False)[0]
        if not np.isfinite(L0):
            continue
        fd = np.zeros(4)
        for k in range(4):
            pp, pm = p.copy(), p.copy()
            pp[k] += h
            pm[k] -= h
            fd[k] = (oracle.traj_eval_subpixel(c["psi64"], c["phi64"], c["times"], c["kw"][i],
                                               *pp, grad=False)[0] -
                     oracle.traj_eval_subpixel(c["psi64"], c["phi64"], c["times"], c["kw"][i],
                                               *pm, grad=False)[0]) / (2 * h)
        floor = 0.01 * max(abs(L0), 1.0)
        assert np.all(np.abs(g[i] - fd) <= 1e-3 * np.maximum(np.abs(fd), floor)), (i, g[i], fd)
        checked += 1
    assert checked >= 5


def test_traj_backward_matches_oracle_vjp(cuda_device):
    c = _case(T=13, H=96, W=160, n_movers=6, n_rand=60, seed=31)
    psi, phi, P, kw = _gpu(c)
    n = len(c["P"])
    gl = c["rng"].normal(size=n).astype(np.float32)
    ga = c["rng"].normal(size=n).astype(np.float32)
    gp, gpsi, gphi = kb.traj_eval_backward(psi, phi, c["times"], P, kw, _d(gl), _d(ga),
                                           True, True, True)
    gp, gpsi, gphi = gp.cpu().numpy(), gpsi.cpu().numpy(), gphi.cpu().numpy()
    o_psi = np.zeros_like(c["psi64"])
    o_phi = np.zeros_like(c["phi64"])
    for i in range(n):
        r = oracle.traj_vjp(c["psi64"], c["phi64"], c["times"], c["kw"][i],
                            *c["P"][i].astype(np.float64), gL=float(gl[i]), gA=float(ga[i]))
        if r is None:
            assert not gp[i].any()
            continue
        o_p, a, b = r
        o_psi += a
        o_phi += b
        assert np.all(np.abs(gp[i] - o_p) <= 1e-4 * max(np.abs(o_p).max(), 1e-6)), (i, gp[i], o_p)
    assert np.abs(gpsi - o_psi).max() <= 1e-5 * np.abs(o_psi).max()
    assert np.abs(gphi - o_phi).max() <= 1e-5 * np.abs(o_phi).max()
    assert (o_psi != 0).sum() > 100
    # only grad_lh, only one image
    gp2, gpsi2, gphi2 = kb.traj_eval_backward(psi, phi, c["times"], P, kw, _d(gl), None,
                                              True, True, False)
    assert gphi2 is None
    o_psi = np.zeros_like(c["psi64"])
    for i in range(n):
        r = oracle.traj_vjp(c["psi64"], c["phi64"], c["times"], c["kw"][i],
                            *c["P"][i].astype(np.float64), gL=float(gl[i]), gA=0.0)
        if r is not None:
            o_psi += r[1]
    assert np.abs(gpsi2.cpu().numpy() - o_psi).max() <= 1e-5 * np.abs(o_psi).max()


def test_autograd_function_uses_the_backward_kernel(cuda_device):
    c = _case(T=10, H=64, W=96, n_movers=3, n_rand=20, seed=41)
    psi, phi, P, kw = _gpu(c)
    P = P.clone().requires_grad_(True)
    psi = psi.clone().requires_grad_(True)
    phi = phi.clone().requires_grad_(True)
    L, A = kb.traj_likelihood(P, psi, phi, c["times"], kw)
    ok = torch.isfinite(L)
    wl = torch.linspace(0.5, 1.5, L.numel(), device="cuda")
    loss = (wl * torch.where(ok, L, 0.0)).sum() - 0.3 * torch.where(ok, A, 0.0).sum()
    before = kb.launch_count()
    loss.backward()
    assert kb.launch_count() > before
    gl = (wl * ok).float().contiguous()
    ga = (-0.3 * ok.float()).contiguous()
    gp, gpsi, gphi = kb.traj_eval_backward(psi.detach(), phi.detach(), c["times"], P.detach(), kw,
                                           gl, ga, True, True, True)
    assert torch.allclose(P.grad, gp, rtol=1e-6, atol=0)
    assert torch.allclose(psi.grad, gpsi, rtol=1e-5, atol=1e-6)
    assert torch.allclose(phi.grad, gphi, rtol=1e-5, atol=1e-6)
    # the gradient of sum(L) in the params against the oracle
    L2, _ = kb.traj_likelihood(P, psi.detach(), phi.detach(), c["times"], kw)
    P.grad = None
    torch.where(torch.isfinite(L2), L2, 0.0).sum().backward()
    g = P.grad.cpu().numpy()
    span = c["times"][-1] - c["times"][0]
    for i in torch.nonzero(ok).flatten().tolist():
        L0, _, G = oracle.traj_eval_subpixel(c["psi64"], c["phi64"], c["times"], c["kw"][i],
                                             *c["P"][i].astype(np.float64))
        tol = 1e-4 * max(abs(L0), 1.0) * np.array([1.0, 1.0, span, span])
        assert np.all(np.abs(g[i] - G) <= tol)


def _refine_compare(c, rp, min_agree):
    psi, phi, P, kw = _gpu(c)
    pr, L1, A1, L0 = kb.refine(psi, phi, c["times"], P, kw, rp)
    pr, L1, A1, L0 = (a.cpu().numpy() for a in (pr, L1, A1, L0))
    assert torch.equal(P, _d(c["P"]))          # not in place by default
    agree = total = 0
    for i in range(len(c["P"])):
        p0 = c["P"][i].astype(np.float64)
        Ls = oracle.traj_eval_subpixel(c["psi64"], c["phi64"], c["times"], c["kw"][i], *p0,
                                       grad=False)[0]
        po, Lo, Ao = oracle.refine_adam(c["psi64"], c["phi64"], c["times"], c["kw"][i], p0,
                                        rp.n_steps, rp.lr_pos, rp.lr_vel, rp.beta1, rp.beta2,
                                        rp.eps)
        if not np.isfinite(Ls):
            assert np.isnan(L0[i]) and np.isnan(L1[i]) and np.array_equal(pr[i], c["P"][i])
            continue
        assert abs(L0[i] - Ls) <= 1e-4 * max(abs(Ls), 1.0)
        if not np.isfinite(Lo):
            continue
        total += 1
        # the returned L and alpha are the oracle's at the returned params
        Lg, Ag, _ = oracle.traj_eval_subpixel(c["psi64"], c["phi64"], c["times"], c["kw"][i],
                                              *pr[i].astype(np.float64), grad=False)
        assert abs(L1[i] - Lg) <= 1e-4 * max(abs(Lg), 1.0), (i, L1[i], Lg)
        assert abs(A1[i] - Ag) <= 1e-4 * abs(Ag) * max(1.0, 1.0 / max(abs(Lg), 1e-30))
        if np.all(np.abs(pr[i] - po) <= 1e-3):
            agree += 1
    assert total > 0.8 * len(c["P"])
    assert agree >= min_agree * total, (agree, total)
    return pr, L0, L1


def test_refine_one_step_matches_oracle(cuda_device, case):
    _refine_compare(case, kb.RefineParams(n_steps=1), 1.0)


def test_refine_twenty_steps_matches_oracle(cuda_device, case):
    pr, L0, L1 = _refine_compare(case, kb.RefineParams(), 0.98)
    # ascent from the grid starts of the injected movers raises L on most of them
    nm = len(case["movers"]["x0"])
    s, e = L0[0:2 * nm:2], L1[0:2 * nm:2]
    f = np.isfinite(s) & np.isfinite(e)
    assert (e[f] > s[f]).mean() >= 0.8


def test_refine_edge_cases(cuda_device):
    c = _case(T=8, H=48, W=64, n_movers=2, n_rand=10, seed=51)
    psi, phi, P, kw = _gpu(c)
    # n = 0
    e = torch.empty((0, 4), dtype=torch.float32, device="cuda")
    ek = torch.empty((0, 1), dtype=torch.int32, device="cuda")
    pr, L1, A1, L0 = kb.refine(psi, phi, c["times"], e, ek)
    assert pr.numel() == 0 and L1.numel() == 0
    lh, fl = kb.traj_eval(psi, phi, c["times"], e, ek)
    assert lh.numel() == 0
    # NaN params, an empty kept set and a track entirely off the image give NaN and stay put
    bad = torch.tensor([[float("nan")] * 4, [10.0, 10.0, 1.0, 1.0], [-500.0, -500.0, 0.0, 0.0]],
                       device="cuda")
    kb_ = torch.tensor([[0xFF], [0], [0xFF]], dtype=torch.int32, device="cuda")
    lh, fl, g = kb.traj_eval(psi, phi, c["times"], bad, kb_, grad=True)
    assert torch.isnan(lh).all() and torch.isnan(fl).all() and not g.any()
    pr, L1, A1, L0 = kb.refine(psi, phi, c["times"], bad, kb_)
    assert torch.isnan(L1).all() and torch.isnan(L0).all()
    assert torch.equal(pr[1:], bad[1:]) and torch.isnan(pr[0]).all()
    gp, gpsi, gphi = kb.traj_eval_backward(psi, phi, c["times"], bad, kb_,
                                           torch.ones(3, device="cuda"), None, True, True, True)
    assert not gp.any() and not gpsi.any() and not gphi.any()
    # keep=None keeps every epoch
    lh_all, _ = kb.traj_eval(psi, phi, c["times"], P)
    full = torch.full((P.shape[0], 1), 0xFF, dtype=torch.int32, device="cuda")
    lh_full, _ = kb.traj_eval(psi, phi, c["times"], P, full)
    assert torch.equal(torch.nan_to_num(lh_all, 7.0), torch.nan_to_num(lh_full, 7.0))
    # n_steps = 0 returns the start with its L
    pr, L1, A1, L0 = kb.refine(psi, phi, c["times"], P, kw, kb.RefineParams(n_steps=0))
    assert torch.equal(pr, P)
    assert torch.equal(torch.nan_to_num(L1, 7.0), torch.nan_to_num(L0, 7.0))
    # in place
    Q = P.clone()
    kb.refine(psi, phi, c["times"], Q, kw, inplace=True)
    assert not torch.equal(Q, P)
    # invalid refine settings are refused before any launch
    with pytest.raises(kb.KbError):
        kb.refine(psi, phi, c["times"], P, kw, kb.RefineParams(beta1=1.0))
    with pytest.raises(kb.KbError):
        kb.refine(psi, phi, c["times"], P, kw, kb.RefineParams(lr_pos=float("nan")))


def test_candidate_params_gathers_search_survivors(cuda_device):
    rng = np.random.default_rng(61)
    T, H, W = 11, 40, 56
    times = np.sort(rng.uniform(0, 1.0, T))
    times[0] = 0.0
    phi = rng.uniform(0.2, 1.5, (T, H, W)).astype(np.float32)
    psi = (rng.normal(size=(T, H, W)) * np.sqrt(phi) + 2.0 * phi * (rng.random((T, H, W)) < 0.2)
           ).astype(np.float32)
    vx = rng.uniform(-20, 20, 40).astype(np.float32)
    vy = rng.uniform(-20, 20, 40).astype(np.float32)
    sp = kb.SearchParams(k=3, lh_min=1.0, min_obs=3, clip_on=1, window=(3, 50, 2, 37))
    vxd, vyd = _d(vx), _d(vy)
    res = kb.search(_d(psi), _d(phi), times, vxd, vyd, sp)
    pix, slot, count = kb.collect(res, 300)
    params, keep = kb.candidate_params(pix, slot, res, vxd, vyd, window=sp.window)
    x0, y0, cvx, cvy, traj = kb.candidate_tracks(pix, slot, res, vxd, vyd, window=sp.window)
    ok = traj >= 0
    assert int(ok.sum()) == min(int(count.item()), 300) and ok.any()
    assert torch.equal(params[ok, 0], x0[ok].float()) and torch.equal(params[ok, 1], y0[ok].float())
    assert torch.equal(params[ok, 2], cvx[ok]) and torch.equal(params[ok, 3], cvy[ok])
    assert torch.isnan(params[~ok]).all() and not keep[~ok].any()
    wy, wx, K = res["idx"].shape
    flat = res["mask"].reshape(wy * wx * K, -1)
    sel = pix[ok].long() * K + slot[ok].long()
    assert torch.equal(keep[ok], flat[sel])
    # every survivor has a finite start likelihood: its kept epochs have phi > 0 at the rounded
    # position, which is one of the bilinear taps with weight >= 1/4
    _, _, _, L0 = kb.refine(_d(psi), _d(phi), times, params[ok].contiguous(),
                            keep[ok].contiguous(), kb.RefineParams(n_steps=0))
    assert torch.isfinite(L0).all()


def _match_movers(params, lh, movers, times, max_px=2.5):
    """Index of the highest-L candidate whose track stays within max_px of each mover's true
    track at the first and last epoch (-1 if none)."""
    span = times[-1] - times[0]
    P = params.astype(np.float64)
    out = []
    for i in range(len(movers["x0"])):
        tx0, ty0, tvx, tvy = (movers[k][i] for k in ("x0", "y0", "vx", "vy"))
        d0 = np.hypot(P[:, 0] - tx0, P[:, 1] - ty0)
        d1 = np.hypot(P[:, 0] + P[:, 2] * span - (tx0 + tvx * span),
                      P[:, 1] + P[:, 3] * span - (ty0 + tvy * span))
        m = (d0 <= max_px) & (d1 <= max_px) & np.isfinite(lh)
        out.append(int(np.argmax(np.where(m, lh, -np.inf))) if m.any() else -1)
    return np.array(out)


def test_refine_recovers_off_grid_movers_end_to_end(cuda_device):
    """Search -> collect -> candidate_params -> refine on an image stack whose movers have
    sub-pixel starts and velocities between grid points: refinement must raise L and shrink
    the velocity error of the recovered movers against the grid search."""
    from synth import make_stack, search_params_for
    s = make_stack("decam_refine", H=1024, W=2048, n_movers=40)
    sp = kb.SearchParams(**{k: v for k, v in search_params_for("decam_refine").items()
                            if k in ("k", "lh_min", "min_obs", "clip", "n_sigma", "clip_on")})
    img, var = _d(s.img), _d(s.var)
    mask = _d(s.mask)
    psi, phi = kb.make_psi_phi(img, var, mask, _d(s.psf))
    vx, vy = _d(s.vx), _d(s.vy)
    res = kb.search(psi, phi, s.times, vx, vy, sp)
    pix, slot, count = kb.collect(res, 20000)
    params, keep = kb.candidate_params(pix, slot, res, vx, vy)
    pr, L1, A1, L0 = kb.refine(psi, phi, s.times, params, keep)
    torch.cuda.synchronize()
    P0, P1 = params.cpu().numpy(), pr.cpu().numpy()
    L0, L1 = L0.cpu().numpy(), L1.cpu().numpy()
    mv = s.movers
    i0 = _match_movers(P0, L0, mv, s.times)
    i1 = _match_movers(P1, L1, mv, s.times)
    both = (i0 >= 0) & (i1 >= 0)
    assert both.sum() >= 10, both.sum()
    tv = np.stack([mv["vx"], mv["vy"]], 1)
    e0 = np.hypot(*(P0[i0[both], 2:] - tv[both]).T)
    e1 = np.hypot(*(P1[i1[both], 2:] - tv[both]).T)
    assert np.median(e1) < 0.6 * np.median(e0), (np.median(e0), np.median(e1))
    assert np.all(L1[i1[both]] >= L0[i0[both]] - 1e-3 * np.abs(L0[i0[both]]))
