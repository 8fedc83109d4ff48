"""CPU checks of the sources against the rules the kernels are written to: no device traps or device asserts (a
failure is a status the host reads), every mbarrier poll inside a helper that gives up after a bounded number of
polls, host code that builds on both x86-64 and aarch64, and comments that stand on their own (no references to
documents outside the sources)."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1710_08830_gb300", "csrc")


def _sources(patterns):
    files = []
    for p in patterns:
        files += glob.glob(os.path.join(ROOT, p), recursive=True)
    return sorted(f for f in files if "/_work/" not in f and "/_build/" not in f and "/baseline/" not in f)


def _read(f):
    with open(f, encoding="utf-8") as fh:
        return fh.read()


def test_no_device_trap_or_assert():
    bad = []
    for f in _sources(["paper_1710_08830_gb300/csrc/*.cu", "paper_1710_08830_gb300/csrc/*.cuh", "include/*.h"]):
        for n, line in enumerate(_read(f).splitlines(), 1):
            code = line.split("//")[0]
            if "__trap" in code or re.search(r"\btrap\s*;", code) or re.search(r"(?<!static_)\bassert\s*\(", code):
                bad.append(f"{os.path.relpath(f, ROOT)}:{n}: {line.strip()}")
    assert not bad, "\n".join(bad)


def test_mbarrier_polls_are_bounded():
    """The only mbarrier poll is tc::mbar_try, and only the bounded helpers of the same header call it."""
    polls, callers = [], []
    for f in _sources(["paper_1710_08830_gb300/csrc/*.cu", "paper_1710_08830_gb300/csrc/*.cuh"]):
        src = _read(f)
        rel = os.path.relpath(f, ROOT)
        polls += [rel for _ in re.finditer(r"mbarrier\.(try|test)_wait", src)]
        callers += [(rel, m.start()) for m in re.finditer(r"\bmbar_try\s*\(", src)]
    assert polls == ["paper_1710_08830_gb300/csrc/tc_common.cuh"]
    hdr = _read(os.path.join(CSRC, "tc_common.cuh"))
    assert all(rel.endswith("tc_common.cuh") for rel, _ in callers)
    # every call sits in a loop bounded by WAIT_LIMIT
    for m in re.finditer(r"\bmbar_try\s*\(", hdr):
        head = hdr[:m.start()]
        if head.rstrip().endswith("bool"):
            continue   # the definition itself
        loop = head[head.rfind("for ("):]
        assert "WAIT_LIMIT" in loop.split(")")[0], "an mbar_try call outside a WAIT_LIMIT loop"


def test_host_code_is_portable():
    """Host code builds on aarch64 as well as x86-64: no x86 intrinsic headers and no -march=native."""
    bad = []
    for f in _sources(["paper_1710_08830_gb300/**/*.cu", "paper_1710_08830_gb300/**/*.cuh", "paper_1710_08830_gb300/**/*.py",
                       "oracle/**/*.c", "oracle/**/*.h", "oracle/**/*.py", "__graft_entry__.py", "bench.py"]):
        src = _read(f)
        if re.search(r"#include\s*<\w*intrin\.h>", src) or "-march=native" in src:
            bad.append(os.path.relpath(f, ROOT))
    assert not bad, bad


def test_comments_name_no_outside_documents():
    """Code and comments state facts themselves: no all-capitals document names (the one file the benchmark reads,
    the measured peaks, is the exception)."""
    bad = []
    for f in _sources(["paper_1710_08830_gb300/**/*.py", "paper_1710_08830_gb300/csrc/*.cu",
                       "paper_1710_08830_gb300/csrc/*.cuh", "include/*.h", "oracle/**/*.c", "oracle/**/*.py",
                       "tests/**/*.py", "bench.py", "__graft_entry__.py"]):
        for n, line in enumerate(_read(f).splitlines(), 1):
            for m in re.finditer(r"\b[A-Z][A-Z_]+\.(?:md|json)\b", line):
                if m.group(0) != "MEASURED_PEAKS.json":
                    bad.append(f"{os.path.relpath(f, ROOT)}:{n}: {m.group(0)}")
    assert not bad, "\n".join(bad)
