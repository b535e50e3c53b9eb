"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function include/hesp.h declares; host-only entry points (platform models,
DAG queries) agree with the closed forms (no device work is launched)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1602_05510_b300 import build, hesp
from paper_1602_05510_b300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return hesp.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hesp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hesp_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert len(names) >= 15
    for nm in names:
        assert hasattr(L, nm), nm
    assert sorted(hesp.EXPORTS) == sorted(names)


def test_status_strings(L):
    assert L.hesp_status_string(0) == b"HESP_OK"
    assert L.hesp_status_string(-2) == b"HESP_ERR_CAPACITY"


def test_platform_models_match_oracle_values(L):
    import json
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "worked_examples.json")))
    p = hesp.Platform(W.PLATFORMS["cfg0"])
    assert [p.exec_ns(o, 0, 1024) for o in range(4)] == g["exec_ns"]["cpu_1024"]
    assert [p.exec_ns(o, 1, 512) for o in range(4)] == g["exec_ns"]["gpu_512"]
    assert [p.xfer_ns(s * s) for s in g["xfer_ns"]["bs"]] == g["xfer_ns"]["ns"]


def test_platform_argument_errors(L):
    bad = W.PlatformSpec("bad", 2, (W.CPU_TYPE,), ((0, 0), (2, 0)))
    with pytest.raises(hesp.HespError):
        hesp.Platform(bad)
    big = W.PlatformSpec("big", 5, (W.CPU_TYPE,), ((0, 0),))
    with pytest.raises(hesp.HespError):
        hesp.Platform(big)


def test_dag_counts(L):
    for n in (1, 3, 8, 16, 32):
        d = hesp.Dag(n, 2048, 3)
        assert d.n_base == n * (n + 1) * (n + 2) // 6
        op, k, i, j = d.base_tasks()
        assert (op == 0).sum() == n and (op == 3).sum() == n * (n - 1) * (n - 2) // 6
        rng = np.random.default_rng(n)
        for _ in range(5):
            lv = rng.integers(0, 4, d.n_base).astype(np.int8)
            t, f3 = d.count_tasks(lv)
            assert f3 == (n * 2048) ** 3
        for lvl in range(4):
            s = n << lvl
            assert d.count_tasks(np.full(d.n_base, lvl, np.int8))[0] == s * (s + 1) * (s + 2) // 6


def test_no_unresolved_internal_symbols():
    """Every internal (namespace hesp) symbol the library uses is defined in
    it: a shared-library link does not catch a function left in an anonymous
    namespace of another file, only loading does."""
    import shutil
    import subprocess
    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("nm not available")
    from paper_1602_05510_b300 import build
    lib = build.build()
    out = subprocess.run([nm, "-D", "--undefined-only", lib], capture_output=True, text=True, check=True).stdout
    assert not [l for l in out.splitlines() if "_ZN4hesp" in l]
