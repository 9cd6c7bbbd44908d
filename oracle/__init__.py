"""FP64 CPU oracle for the KBMOD shift-and-stack search with the in-line sigma-G clip.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline leg are
the only callers.  The product path (``paper_2109_03296_b300``) never imports this package, and
this package never imports the product path.  See ``kb_oracle.c`` for the definitions and the
readings of points the paper leaves open.

Pinning status of each function (what ties it to the paper and to mathematics other than itself;
the pins live in tests/test_oracle_pins.py):
  sigma_g_coeff     closed form 1/(2 sqrt2 erfinv(1/2)) via scipy, and 0.7413 printed in Section 3.1
  percentile        numpy.percentile(method="linear") on random samples
  sigma_g_clip      hand-worked examples, constant lightcurve keeps all, +20 sigma spikes rejected
  track_offsets     numpy float32 arithmetic on random (epochs from 0 and as MJDs) and
                    half-integer cases
  psi_phi           constant variance gives phi = sum P^2/var; delta image gives psi = P/var;
                    scipy.ndimage.correlate of I/var and 1/var with P and P^2 (varying variance)
  search            closed form L = SNR sqrt(T), alpha = F for a noiseless mover; an independent
                    numpy shift-and-stack with numpy.nanpercentile on tiny stacks; invariances;
                    an exactly representable L = 4 at an inclusive threshold
  stamps            mean stamp of a noiseless mover is F P; numpy.median/mean on tiny stacks
  traj_eval_subpixel  L/alpha equal the integer search at integer positions (epochs from 0 and
                    as MJDs); central finite
                    differences of L for the gradient
  traj_vjp          central finite differences of L and alpha in the track parameters and in
                    single psi/phi pixels; tap support; Euler's theorem for the homogeneity
                    degrees of L and alpha in psi and phi; it adds to its output arrays
  stamp_moments     closed forms: a single lit pixel at (dx, dy) gives x = dx, y = dy, xy = dx dy,
                    xx = dx^2, yy = dy^2; a flat stamp with one dark pixel at its centre gives
                    xx = yy = side r(r+1)(2r+1) / (3 (side^2 - 1)) (36.75 > 36.5 for r = 10);
                    invariance to a constant offset; symmetric stamps give zero odd moments; a
                    sampled Gaussian gives its centre and variance; each filter limit rejects
                    at its own moment's magnitude
  cluster           hand-worked cases (identical tracks, a chain where greedy order matters,
                    tracks that part before the last epoch, invalid entries); on random inputs
                    the properties that fix the greedy result uniquely: kept candidates are
                    pairwise distinct, every other valid one duplicates a kept one of lower
                    index and names the first such as its representative
  refine_adam       closed form of Adam's first step; convergence to a noiseless off-grid mover;
                    stop where Phi vanishes
tests/test_oracle_mutants.py plants plausible mistakes in copies of kb_oracle.c and checks that
each one fails a pin.
"""
from .oracle import *  # noqa: F401,F403
