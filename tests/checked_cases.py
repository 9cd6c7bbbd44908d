"""Searches run by tests/test_gpu_checked.py, once with the regular library and once (in a child
process) with the checked build (KB_B300_LIBRARY=checked).  Run as a script it writes the results
and each search's device error flags to the .npz file named on the command line."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _planes(seed, T, H, W, n_traj, spread):
    rng = np.random.default_rng(seed)
    times = np.sort(rng.uniform(0, 1.0, T))
    times[0] = 0.0
    phi = rng.uniform(0.2, 1.5, (T, H, W))
    psi = rng.normal(size=(T, H, W)) * np.sqrt(phi)
    psi += 3.0 * phi * (rng.random((T, H, W)) < 0.05)
    m = rng.random((T, H, W)) < 0.04
    psi[m] = 0.0
    phi[m] = 0.0
    vx = rng.uniform(-spread, spread, n_traj).astype(np.float32)
    vy = rng.uniform(-spread, spread, n_traj).astype(np.float32)
    return psi.astype(np.float32), phi.astype(np.float32), times, vx, vy


# seed, T, H, W, n_traj, velocity spread (px/day), SearchParams fields
CASES = [
    (1, 13, 101, 77, 70, 40.0, dict(k=4, lh_min=1.5, min_obs=3)),
    (2, 26, 150, 190, 96, 60.0, dict(k=8, lh_min=3.0, min_obs=10)),                 # blocks
    (3, 26, 150, 190, 96, 60.0, dict(k=8, lh_min=3.0, min_obs=10, bound_rows=1)),   # rows
    (4, 40, 65, 80, 50, 30.0, dict(k=3, lh_min=2.0, min_obs=10, clip_on=1)),
    (5, 100, 40, 48, 24, 20.0, dict(k=2, lh_min=2.0, min_obs=30)),
    (6, 9, 90, 90, 40, 400.0, dict(k=5, lh_min=1.0, min_obs=2, window=(3, 70, 5, 83))),
]


def run_all():
    """{name: array} of every case's outputs and error flags, plus a batch of cases 1-5 under
    both modes and both tile widths."""
    import torch

    import paper_2109_03296_b300 as kb
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = {}
    stacks = []
    for i, (seed, T, H, W, n, spread, prm) in enumerate(CASES):
        psi, phi, times, vx, vy = _planes(seed, T, H, W, n, spread)
        sp = kb.SearchParams(**prm)
        res = kb.search(d(psi), d(phi), times, d(vx), d(vy), sp)
        torch.cuda.synchronize()
        out["err_%d" % i] = np.array(kb.search_stats(res["workspace"])[3])
        for k in ("lh", "flux", "idx", "nvalid", "nkept", "mask"):
            out["%s_%d" % (k, i)] = res[k].cpu().numpy()
        if i < 5:
            stacks.append(dict(psi=d(psi), phi=d(phi), times=times, vx=d(vx), vy=d(vy),
                               params=sp))
    b = kb.Batch(stacks)
    for mode in (0, 1):
        for cols in (1, 2):
            b.schedule = kb.Schedule(mode=mode, tile_cols=cols)
            res = b.run(graph=True)
            torch.cuda.synchronize()
            out["err_batch_%d_%d" % (mode, cols)] = np.array(b.stats()[1]["err"])
            for i, r in enumerate(res):
                out["idx_batch_%d_%d_%d" % (mode, cols, i)] = r["idx"].cpu().numpy()
                out["lh_batch_%d_%d_%d" % (mode, cols, i)] = r["lh"].cpu().numpy()
    return out


if __name__ == "__main__":
    np.savez(sys.argv[1], **run_all())
