"""Builds libkb_b300.so in-tree from csrc/*.cu for sm_103a (B300) with nvcc.

Each .cu is compiled separately (in parallel) with -gencode arch=compute_103a,code=sm_103a
and linked into one shared library next to this file.  No JIT, no torch extension machinery:
the library exports plain extern "C" entry points (include/kb.h).

build(checked=True) also links libkb_b300_checked.so: the same library with the search kernel
compiled with -DKB_BOUNDS_CHECK=1 (device-side checks of staged-box reads, TMA coordinates and
result slots, reported in the search's error flags).  Setting KB_B300_LIBRARY=checked makes the
binding load it instead of the regular one.
"""
import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libkb_b300.so")
LIB_CHECKED = os.path.join(HERE, "libkb_b300_checked.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include")]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(ROOT, "include",
                                                                                "kb.h")]


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


def _compile(src, verbose, checked=False):
    obj = os.path.join(BUILD, os.path.basename(src) + (".checked.o" if checked else ".o"))
    cmd = [NVCC, *ARCH, *FLAGS, *(["-DKB_BOUNDS_CHECK=1"] if checked else []), "-c", src, "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
    return obj, r.stderr


def _link(out, objs):
    cmd = [NVCC, *ARCH, "-shared", "-o", out, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))


def build(force=False, verbose=False, checked=False):
    if not force and up_to_date() and (not checked or os.path.exists(LIB_CHECKED)):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    jobs = [(s, False) for s in _sources()]
    search = os.path.join(CSRC, "search.cu")
    if checked:
        jobs.append((search, True))
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(lambda j: _compile(j[0], verbose, j[1]), jobs))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    objs = [o for (o, _), (_, chk) in zip(results, jobs) if not chk]
    _link(LIB, objs)
    if checked:
        search_obj = os.path.join(BUILD, "search.cu.o")
        checked_obj = [o for (o, _), (_, chk) in zip(results, jobs) if chk][0]
        _link(LIB_CHECKED, [checked_obj if o == search_obj else o for o in objs])
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                checked="--checked" in sys.argv))
