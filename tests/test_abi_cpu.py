"""Host-side checks of the C ABI (no GPU): the library builds and loads, it
exports every function that include/lrcc.h declares, and argument validation
rejects bad inputs before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2503_23144_gb300 import build, lrcc
    if not os.path.exists(lrcc._LIB_PATH):
        build.build()
    return lrcc


def _declared():
    src = open(os.path.join(ROOT, "include", "lrcc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lrcc_[a-z_]+)\s*\(", src)))


def test_header_symbols_exported(lib):
    names = _declared()
    assert "lrcc_setup" in names and "lrcc_solve" in names
    so = ctypes.CDLL(lib._LIB_PATH)
    for n in names:
        assert hasattr(so, n), n
    bound = {s[0] for s in lib.SIGNATURES}
    assert set(names) <= bound


def test_default_options(lib):
    o = lib.lrcc_default_options()
    assert o.max_iter == 200 and o.diis_size == 8 and o.prec == lib.LRCC_FP64
    assert 0 < o.r_tol < 1e-6 and 0 < o.x_tol < 1e-6


def _system(O=3, V=5, L=4, seed=0):
    return synth.make_system(O, V, L, seed)


def test_setup_rejects_non_hermitian(lib):
    s = _system()
    B = s["B"].copy()
    B[0, 0, 1] += 0.1
    with pytest.raises(lib.LrccError) as e:
        lib.lrcc_setup(s["eps"], B, s["mu"], s["O"], s["V"])
    assert e.value.status == lib.LRCC_EINVAL
    mu = s["mu"].copy()
    mu[1, 2, 3] += 0.1j
    with pytest.raises(lib.LrccError) as e:
        lib.lrcc_setup(s["eps"], s["B"], mu, s["O"], s["V"])
    assert e.value.status == lib.LRCC_EINVAL


def test_setup_rejects_bad_ordering_and_sizes(lib):
    s = _system()
    eps = s["eps"].copy()
    eps[0] = 10.0                       # occupied above the virtuals
    with pytest.raises(lib.LrccError) as e:
        lib.lrcc_setup(eps, s["B"], s["mu"], s["O"], s["V"])
    assert e.value.status == lib.LRCC_EINVAL
    eps = s["eps"].copy()
    eps[4] = np.nan
    with pytest.raises(lib.LrccError) as e:
        lib.lrcc_setup(eps, s["B"], s["mu"], s["O"], s["V"])
    assert e.value.status == lib.LRCC_EINVAL
    s1 = _system(O=1, V=5)
    with pytest.raises(lib.LrccError) as e:
        lib.lrcc_setup(s1["eps"], s1["B"], s1["mu"], 1, 5)
    assert e.value.status == lib.LRCC_EINVAL


def test_setup_rejects_bad_options(lib):
    """Option validation happens before any device call."""
    s = _system()
    for fields in ({"fns_density": 2}, {"prec": 7}, {"diis_size": 1}, {"solver": 2}, {"subspace_max": -1}, {"embed_budget_mb": -1}, {"ladder_hermitian": 2},
                   {"solver": 1, "prec": lib.LRCC_MIXED_BF16X3}):
        o = lib.lrcc_default_options()
        for field, bad in fields.items():
            setattr(o, field, bad)
        with pytest.raises(lib.LrccError) as e:
            lib.lrcc_setup(s["eps"], s["B"], s["mu"], s["O"], s["V"], o)
        assert e.value.status == lib.LRCC_EINVAL, fields
    o = lib.lrcc_default_options()
    assert o.fns_density == 0 and o.solver == 0 and o.subspace_max == 0 and o.embed_budget_mb == 0 and o.ladder_hermitian == 0


def test_pack_roundtrip(lib):
    rng = np.random.default_rng(0)
    t1 = rng.standard_normal((2, 3, 4)) + 0j
    t2 = rng.standard_normal((2, 3, 3, 4, 4)) + 1j
    flat = lib.pack_amplitudes(t1, t2)
    a, b = lib.unpack_amplitudes(flat, 3, 4)
    assert np.array_equal(a, t1) and np.array_equal(b, t2)


def test_missing_library_fails_loudly(tmp_path):
    """Without the built CUDA library every entry point raises ImportError:
    there is no CPU fallback behind the binding."""
    import subprocess
    import sys
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "from paper_2503_23144_gb300 import lrcc\n"
        "lrcc._LIB_PATH = %r\n"
        "lrcc._lib = None\n"
        "try:\n"
        "    lrcc.lrcc_default_options()\n"
        "except ImportError as e:\n"
        "    print('ImportError', e)\n"
        "    sys.exit(0)\n"
        "sys.exit(3)\n" % (ROOT, str(tmp_path / "absent" / "_lrcc.so")))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "not built" in r.stdout


C_CLIENT = r"""
#include "lrcc.h"
#include <stdio.h>
int main(void) {
    lrcc_options o;
    int64_t np = 0, pw = 0, n;
    lrcc_status st;
    lrcc_default_options(&o);
    st = lrcc_embed_layout(LRCC_MIXED_BF16X3, 7140, 7140, 1, &np, &pw);
    n = lrcc_plan_slabs(120, 1 << 20, 0, 1024, NULL, 0);
    printf("%d %d %lld %lld %lld\n", o.max_iter, (int)st, (long long)np, (long long)pw, (long long)n);
    return (st == LRCC_OK && o.max_iter == 200 && n > 0) ? 0 : 1;
}
"""


def test_header_is_plain_c99_and_links(lib, tmp_path):
    """include/lrcc.h compiles as strict C99 (-pedantic -Werror) and a C
    client links against the library and calls its host-only entry points."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    libdir = os.path.dirname(lib._LIB_PATH)
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe), lib._LIB_PATH,
                        "-Wl,-rpath," + libdir], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.split()[:2] == ["200", "0"]


def test_query_hooks_reject_null(lib):
    """Host-only measurement hooks validate their arguments without a context
    or a device: a NULL context or output pointer gives LRCC_EINVAL."""
    so = lib.library()
    v = [ctypes.c_int64(7) for _ in range(3)]
    assert so.lrcc_memory_stats(None, *[ctypes.byref(x) for x in v]) == lib.LRCC_EINVAL
    assert [x.value for x in v] == [7, 7, 7]
    assert so.lrcc_kernel_launches(None) == 0
