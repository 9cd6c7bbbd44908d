"""The ncu summaries under profiles/ are short text, run only committed files with options the
bench accepts, lock no clocks, and name only workloads the generator defines."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROF = os.path.join(ROOT, "profiles")


def _files():
    return sorted(os.path.join(PROF, f) for f in os.listdir(PROF))


def test_profiles_are_short_text():
    files = _files()
    assert files
    for p in files:
        assert p.endswith((".md", ".txt")), p
        assert os.path.getsize(p) < 32 * 1024, p


def _commands(text):
    """Command text of a summary: indented code lines (backslash continuations joined) and
    backtick spans."""
    out = [m.group(1).replace("\n", " ") for m in re.finditer(r"`([^`]+)`", text)]
    block = []
    for line in text.splitlines():
        if line.startswith("    ") and line.strip():
            block.append(line.strip().rstrip("\\").strip())
            if not line.rstrip().endswith("\\"):
                out.append(" ".join(block))
                block = []
        elif block:
            out.append(" ".join(block))
            block = []
    if block:
        out.append(" ".join(block))
    return out


def test_profile_commands_run_committed_files_with_known_options():
    from synth import CONFIGS
    opts = {a for act in bench_parser_actions() for a in act}
    n_python = n_ncu = 0
    for p in _files():
        text = open(p).read()
        assert "_work" not in text and "gpurun" not in text, p
        for cmd in _commands(text):
            for m in re.finditer(r"python (\S+)((?: --?[\w-]+(?: [\w.]+)?)*)", cmd):
                n_python += 1
                script = m.group(1)
                assert os.path.exists(os.path.join(ROOT, script)), (p, script)
                for flag in re.findall(r"(--?[\w-]+)", m.group(2)):
                    assert flag in opts, (p, flag)
                w = re.search(r"--workload (\w+)", m.group(2))
                if w:
                    assert w.group(1) in CONFIGS or w.group(1) == "batch64", (p, w.group(1))
            for m in re.finditer(r"(?:^|\s)ncu (?!-i\b)", cmd):
                n_ncu += 1
                stop = cmd.find(" python ", m.start())
                opts_text = cmd[m.start():stop if stop > 0 else len(cmd)]
                assert "--clock-control none" in opts_text, (p, opts_text)
    assert n_python >= 5 and n_ncu >= 5


def bench_parser_actions():
    import argparse
    import bench
    parser_holder = {}
    real = argparse.ArgumentParser.parse_args

    def grab(self, *a, **k):
        parser_holder["p"] = self
        raise SystemExit(0)

    argparse.ArgumentParser.parse_args = grab
    try:
        try:
            bench.parse()
        except SystemExit:
            pass
    finally:
        argparse.ArgumentParser.parse_args = real
    return [act.option_strings for act in parser_holder["p"]._actions]
