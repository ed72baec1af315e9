"""The FP64 oracle and the CUDA library share no code: neither imports,
includes or links the other, and importing the package does not load the
oracle (the product path never routes through it)."""
import glob
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _files(pattern):
    return glob.glob(os.path.join(ROOT, pattern), recursive=True)


def test_library_sources_do_not_reference_the_oracle():
    srcs = (_files("paper_1106_4198_gb300/**/*.py") + _files("paper_1106_4198_gb300/csrc/*")
            + _files("include/*.h"))
    assert srcs
    for p in srcs:
        text = open(p, errors="replace").read()
        assert not re.search(r"\boracle\b|\bor_[a-z_]+\(", text), p


def test_oracle_sources_do_not_reference_the_library():
    srcs = _files("oracle/*.py") + _files("oracle/*.c")
    assert srcs
    for p in srcs:
        text = open(p, errors="replace").read()
        assert "paper_1106_4198_gb300" not in text, p
        assert not re.search(r'#include\s+"', text), p  # system headers only
        assert "onmf.h" not in text and "csrc" not in text, p


def test_importing_the_package_does_not_load_the_oracle():
    code = ("import sys; sys.path.insert(0, %r); import paper_1106_4198_gb300 as m; "
            "m.lib(); print('oracle' in sys.modules, any('oracle' in k for k in sys.modules))"
            % ROOT)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                         check=True).stdout.split()
    assert out == ["False", "False"], out
