"""The checked build (search kernel compiled with KB_BOUNDS_CHECK=1: every staged-box read, TMA
x coordinate and result slot is tested before the access) runs the searches of
tests/checked_cases.py in a child process: no check may fail (error flags 0), and its results
must equal the regular library's bit for bit (the checks change no arithmetic)."""
import os
import subprocess
import sys

import numpy as np
import pytest

import checked_cases

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.mark.gpu
def test_checked_build_finds_no_violation_and_matches(cuda_device, tmp_path):
    lib = os.path.join(ROOT, "paper_2109_03296_b300", "libkb_b300_checked.so")
    if not os.path.exists(lib):
        from paper_2109_03296_b300 import build
        build.build(checked=True)
    out = str(tmp_path / "checked.npz")
    env = dict(os.environ, KB_B300_LIBRARY="checked")
    subprocess.run([sys.executable, os.path.join(HERE, "checked_cases.py"), out], env=env,
                   check=True, timeout=600)
    got = np.load(out)
    ref = checked_cases.run_all()
    assert set(got.files) == set(ref)
    for k in ref:
        if k.startswith("err"):
            assert int(got[k]) == 0, k
            assert int(ref[k]) == 0, k
        else:
            a, b = got[k], ref[k]
            if a.dtype == np.float32:
                a, b = a.view(np.uint32), b.view(np.uint32)
            assert np.array_equal(a, b), k
