"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every function include/onmf.h declares, and rejects
invalid configurations before touching the device."""
import ctypes
import os
import re

import pytest

import paper_1106_4198_gb300 as onmf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "onmf.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b([A-Za-z_][A-Za-z0-9_]*)\s*\(", text)
    return sorted({n for n in names if n.startswith(("onmf_", "nmf_"))})


def test_header_and_binding_agree():
    decl = set(declared_functions())
    assert decl == set(onmf.EXPORTED), decl ^ set(onmf.EXPORTED)


def test_library_exports_every_declared_symbol():
    L = onmf.lib()
    for name in declared_functions():
        assert hasattr(L, name), name


def test_config_layout_and_defaults():
    assert ctypes.sizeof(onmf.onmf_config) == 96
    c = onmf.onmf_config_default(513, 100)
    assert (c.F, c.K, c.beta, c.n_inner) == (513, 100, 1000, 10)
    assert c.eps == 1e-12 and c.r == 1.0 and c.n_ref == 0
    assert c.h_exponent == 0.5 and c.normalize == 1 and c.rho_on_new == 0
    assert c.precision == onmf.ONMF_FP32 and c.hsolve == onmf.ONMF_HSOLVE_AUTO
    assert c.accumulate == onmf.ONMF_ACC_FP64 and c.stats_ranges == 0
    assert c.h_penalty == 0.0 and c.h_penalty_a == 1.0 and c.w_penalty == 0.0
    assert onmf.onmf_abi_version() == 6


def test_status_strings():
    for st in range(9):
        assert onmf.onmf_status_string(st).startswith("ONMF_")


@pytest.mark.parametrize("field,value", [
    ("F", 0), ("K", 0), ("K", 257), ("beta", 0), ("n_inner", -1),
    ("eps", -1.0), ("r", 1.5), ("h_exponent", 0.0), ("precision", 7),
    ("hsolve", 9), ("accumulate", 3), ("accumulate", -1), ("stats_ranges", -1), ("stats_ranges", 257),
    ("h_penalty", -0.1), ("h_penalty_a", 0.0), ("w_penalty", -1.0),
    ("h_penalty", float("nan")), ("w_penalty", float("inf")),
])
def test_invalid_config_rejected_on_host(field, value):
    import numpy as np
    c = onmf.onmf_config_default(16, 4)
    setattr(c, field, value)
    W0 = np.ones((4, 16), dtype=np.float32) / 16
    h = ctypes.c_void_p()
    st = onmf.lib().onmf_init(ctypes.byref(c), W0.ctypes.data, 0, None,
                              ctypes.byref(h))
    assert st == 1  # ONMF_EINVAL
    assert not h.value


def test_penalties_rejected_on_the_tcgen05_path():
    """The tcgen05 h-solve takes no penalties (the FP32, mma and cluster
    paths do); the host refuses the combination before any device work."""
    import numpy as np
    W0 = np.ones((8, 256), dtype=np.float32) / 256
    for hs in (onmf.ONMF_HSOLVE_TC,):
        for kw in (dict(h_penalty=0.5), dict(w_penalty=0.5)):
            c = onmf.onmf_config_default(256, 8, precision=onmf.ONMF_MIXED, hsolve=hs, **kw)
            h = ctypes.c_void_p()
            st = onmf.lib().onmf_init(ctypes.byref(c), W0.ctypes.data, 0, None,
                                      ctypes.byref(h))
            assert st == 1  # ONMF_EINVAL


def test_mixed_precision_shape_limits():
    """Mixed precision takes K <= 256 and F <= 1024; the host rejects the
    rest before any device work."""
    import numpy as np
    for F, K in ((16, 257), (1025, 8)):
        c = onmf.onmf_config_default(F, K, precision=onmf.ONMF_MIXED)
        W0 = np.ones((K, F), dtype=np.float32) / F
        h = ctypes.c_void_p()
        st = onmf.lib().onmf_init(ctypes.byref(c), W0.ctypes.data, 0, None,
                                  ctypes.byref(h))
        assert st == 1 and not h.value


@pytest.mark.parametrize("field,value", [
    ("F", 0), ("max_chunk", 4097), ("max_batch", 0), ("slots", 5), ("budget_bytes", 0),
    ("precision", 3), ("launch", 2),
])
def test_invalid_server_config_rejected_on_host(field, value):
    c = onmf.onmf_server_config(129, 512, 64, 2, 1 << 20, onmf.ONMF_MIXED,
                                onmf.ONMF_SERVE_GRAPH)
    setattr(c, field, value)
    h = ctypes.c_void_p()
    assert onmf.lib().onmf_server_create(ctypes.byref(c), ctypes.byref(h)) == 1  # ONMF_EINVAL
    assert ctypes.sizeof(onmf.onmf_server_config) == 32


def test_null_arguments_rejected():
    L = onmf.lib()
    assert L.onmf_push_frames(None, None, 0, 0, None, 0) == 1
    assert L.onmf_flush(None) == 1
    assert L.onmf_get_W(None, None, 0) == 1
    assert L.nmf_batch_step(None, 0, None, None, 1, 1, 1, 0.0, 0.5, 1, 1, 0,
                            None, None) == 1
    assert L.nmf_batch_plan_step(None, None, 0, None, None, 1, 0.0, 0.5, 1, 1,
                                 None, None) == 1
    h = ctypes.c_void_p()
    assert L.nmf_batch_plan_create(0, 4, 16, 0, ctypes.byref(h)) == 1  # F < 1
    assert L.nmf_batch_plan_create(16, 4, 0, 0, ctypes.byref(h)) == 1  # N_max < 1
    assert L.nmf_batch_plan_create(16, 4, 16, 7, ctypes.byref(h)) == 1  # precision
    assert not h.value
    L.nmf_batch_plan_destroy(None)  # a NULL plan is ignored
    # an unknown wait kind is refused before any device work
    assert L.onmf_selftest_wait(7, None, None) == 1
    assert L.onmf_selftest_wait(-1, None, None) == 1


def test_c_client_compiles_against_the_header():
    """The C ABI is plain C99: a C client builds against include/onmf.h
    with every warning an error (it runs in tests/test_gpu_c_client.py)."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no gcc")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-fsyntax-only",
                        "-I", os.path.join(root, "include"),
                        os.path.join(root, "tests", "c", "onmf_c_smoke.c")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_struct_layouts_match_the_header():
    """Every field of the C ABI's structs sits at the same offset in the
    ctypes binding as gcc places it from include/onmf.h."""
    import shutil
    import subprocess
    import tempfile
    if not shutil.which("gcc"):
        pytest.skip("no gcc")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    structs = [onmf.onmf_config, onmf.onmf_server_config, onmf.onmf_completion,
               onmf.onmf_server_stats]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "onmf.h"',
             'int main(void) {']
    for st in structs:
        name = st.__name__
        lines.append('printf("%s sizeof %%zu\\n", sizeof(%s));' % (name, name))
        for f, _ in st._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    lines.append("return 0; }")
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines))
        subprocess.run(["gcc", "-std=c99", "-I" + os.path.join(root, "include"), src, "-o", exe],
                       check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if line.strip():
            parts = line.split()
            got[(parts[0], parts[1])] = int(parts[2])
    for st in structs:
        name = st.__name__
        assert got[(name, "sizeof")] == ctypes.sizeof(st), name
        for f, _ in st._fields_:
            assert got[(name, f)] == getattr(st, f).offset, (name, f)


def declared_arity():
    """Parameter count of every function the header declares."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    arity = {}
    for m in re.finditer(r"\b((?:onmf|nmf)_[A-Za-z0-9_]*)\s*\(([^;{]*?)\)\s*;", text):
        params = m.group(2).strip()
        arity[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return arity


def test_binding_argument_counts_match_the_header():
    arity = declared_arity()
    assert set(arity) == set(declared_functions())
    L = onmf.lib()
    checked = 0
    for name, n in arity.items():
        at = getattr(L, name).argtypes
        if at is not None:
            assert len(at) == n, (name, len(at), n)
            checked += 1
    assert checked >= 20
