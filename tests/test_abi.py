"""The C ABI without a GPU: the library loads, exports every declared entry point,
and rejects bad arguments before touching the device."""
import ctypes
import os
import re

import pytest

from paper_1109_0778_b300 import kmeans

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(kmeans_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_exports_every_declared_symbol():
    names = declared_functions()
    assert names, "no declarations found"
    lib = ctypes.CDLL(kmeans.LIB_PATH)
    for name in names:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    assert set(names) == set(kmeans.EXPORTS)


def test_version_and_defaults():
    assert kmeans.version() == 200
    o = kmeans.make_opts()
    assert o.precision == 0 and o.recheck == 1 and not o.stream


FAKE = 1 << 40  # never dereferenced: argument checks run before any CUDA call


def _call(n=100, d=4, k=3, iters=1, prec=0, X=FAKE, C=FAKE + (1 << 30), a=FAKE + (2 << 30),
          s=FAKE + (3 << 30), c=FAKE + (4 << 30)):
    lib = kmeans.lib()
    o = kmeans.make_opts()
    o.precision = prec
    st = kmeans.Stats()
    return lib.kmeans_run_ex(ctypes.byref(o), X, n, d, C, k, a, s, c, iters, 0.0, ctypes.byref(st))


@pytest.mark.parametrize("kw", [dict(n=0), dict(k=0), dict(k=101), dict(d=0), dict(d=257), dict(iters=0),
                                dict(X=0), dict(C=0), dict(a=0), dict(s=0), dict(c=0),
                                dict(C=FAKE + 8), dict(a=FAKE + 16), dict(prec=7), dict(n=1 << 31, k=3)])
def test_bad_arguments_rejected(kw):
    assert _call(**kw) == kmeans.KM_EINVAL
    assert kmeans.lib().kmeans_last_error()


def test_host_entry_validates_too():
    lib = kmeans.lib()
    st = kmeans.Stats()
    rc = lib.kmeans_run_host(None, FAKE, 10, 0, FAKE + 4096, 2, FAKE + 8192, FAKE + 12288, FAKE + 16384, 1, 0.0,
                             ctypes.byref(st))
    assert rc == kmeans.KM_EINVAL
