"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares (no compute calls: these run without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2102_05613_gb300 import build as gbuild
from paper_2102_05613_gb300 import sk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if not f.endswith(".h"):
            continue
        txt = open(os.path.join(inc, f)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:sk_status|const char\s*\*)\s*(\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    path = gbuild.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert declared, "no declarations parsed"
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(sk.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    for name in declared:
        assert re.search(rf"\sT\s{name}$", out, flags=re.M), name


def test_binding_loads_and_reports_errors_without_compute():
    L = sk.lib()
    assert L.sk_last_error() is not None
    # a NULL handle is rejected before any device work
    with pytest.raises(sk.SKError) as e:
        sk._check(L.mcmcmc_advance(None, 1))
    assert e.value.status == sk.SK_ERR_INVALID_ARG


def test_peak_probes_reject_bad_arguments_without_compute():
    # the memory-ceiling probes (sk_peaks.h) check their arguments before any device work
    for call in (lambda: sk.peak_l2_read(1 << 20), lambda: sk.peak_l2_read(48 << 20, passes=0),
                 lambda: sk.peak_smem(7), lambda: sk.peak_smem(sk.SK_PEAK_SMEM_VEC16, iters=0),
                 lambda: sk.peak_tensor(2), lambda: sk.peak_tensor(0, tiles=0),
                 lambda: sk.peak_tensor(1, tiles=5000), lambda: sk.peak_tensor(0, reps=0)):
        with pytest.raises(sk.SKError) as e:
            call()
        assert e.value.status == sk.SK_ERR_INVALID_ARG
