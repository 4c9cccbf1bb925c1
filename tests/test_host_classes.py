"""Host logic of the row schedule: the flops classes (eighths of an octave) and
the heavy-row threshold derived from them, compiled from the library's own
header with the host compiler (no GPU).  Rows of one class must differ by
less than 12.5 % in products, classes must be monotone in the product count,
and class_at_least(T) must split the rows exactly at the class boundary at or
above T (every row below T stays light, every row from that boundary on is
heavy).
"""
import os
import shutil
import subprocess
import textwrap

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2408_11988_gb300", "csrc")

PROGRAM = textwrap.dedent(r"""
    #include <cstdio>
    #include <cstdlib>
    #include "layout.h"
    using namespace ts;
    int main(int argc, char** argv) {
        // mode 0: class of each f read from stdin; mode 1: class_at_least of each T
        const int mode = atoi(argv[1]);
        long long f;
        while (scanf("%lld", &f) == 1)
            printf("%d\n", mode == 0 ? flops_class_host(f) : class_at_least(f));
        return 0;
    }
""")


@pytest.fixture(scope="module")
def classes(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("classes")
    src, exe = d / "classes.cpp", d / "classes"
    src.write_text(PROGRAM)
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)

    def run(mode, values):
        out = subprocess.run([str(exe), str(mode)], input="\n".join(str(int(v)) for v in values),
                             capture_output=True, text=True, check=True).stdout.split()
        return np.array([int(x) for x in out], dtype=np.int64)

    return run


def test_classes_monotone_and_narrow(classes):
    f = np.unique(np.concatenate([np.arange(0, 5000), (1.07 ** np.arange(0, 500)).astype(np.int64),
                                  (1 << np.arange(0, 46)).astype(np.int64)]))
    c = classes(0, f)
    assert c[f == 0][0] == 0 and np.all(c[f > 0] >= 1)
    assert np.all(np.diff(c) >= 0), "classes must not decrease with the product count"
    # within one class (8 <= f < 2^47; the last class holds everything above),
    # the largest count is below 1.125 x the smallest
    inner = (f >= 8) & (f < (1 << 47))
    for cls in np.unique(c[inner]):
        members = f[(c == cls) & inner]
        assert members.max() < 1.125 * members.min(), (cls, members.min(), members.max())


def test_heavy_threshold_at_class_boundary(classes):
    f = np.arange(1, 20000)
    c = classes(0, f)
    for t in (1, 2, 7, 64, 100, 1000, 4096, 5000, 16384):
        cta = int(classes(1, [t])[0])
        heavy = f[c >= cta]
        light = f[c < cta]
        assert light.size == 0 or light.max() < heavy.min()  # one split point
        f0 = heavy.min()
        assert f0 >= t                                         # no row below T is heavy
        # the split sits at the first class boundary at or above T: f0 starts
        # a class, and it is less than an eighth of an octave above T
        assert f0 == 1 or classes(0, [f0 - 1])[0] < classes(0, [f0])[0]
        assert t < 8 or f0 < 1.125 * t
