"""The C-ABI library on the CPU: it loads, exports every declared symbol, and
its host-only planner (parameter derivation, z tables) agrees with the
oracle's independent derivation. No GPU call is made here."""
import math
import os
import re
import subprocess

import numpy as np
import pytest

from oracle import chebyshev as ocheb, params as oparams, solver as osolver
from paper_2101_07088_b300 import build, dpslab

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dpslab.h")).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\*?\s+\*?(dpslab_[a-z_]+)\s*\(", src, re.M)))


def test_every_declared_symbol_is_exported():
    names = declared_functions()
    assert len(names) >= 10
    out = subprocess.run(["nm", "-D", "--defined-only", dpslab.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    L = dpslab.lib()
    for n in names:
        assert hasattr(L, n)


CASES = [
    # paper rule (Sec. 5.1): Tables ewnoparam / ewfreeslab, Sec. 6.3
    dict(Lx=2.0, Ly=2.0, H=0.75, gw=0.025, tol=5e-4, nx=40, ny=40),
    dict(Lx=28.0, Ly=28.0, H=2.0, gw=0.01, tol=1e-4, nx=236, ny=236),
    dict(Lx=2.0, Ly=2.0, H=1.0, gw=0.01, tol=1e-4, nx=38, ny=38),
    # grid resolving g_w, cutoff given (benchmark workloads)
    dict(Lx=128.0, Ly=128.0, H=64.0, gw=1.0, tol=1e-4, nx=256, ny=256, nz=128, r_cut=4.0),
    dict(Lx=32.0, Ly=24.0, H=20.0, gw=1.0, tol=5e-4, nx=64, ny=48, r_cut=4.0),
    # overrides
    dict(Lx=24.0, Ly=24.0, H=24.0, gw=1.0, tol=1e-4, nx=48, ny=48, xi=math.inf, n_sigma=7.0),
    dict(Lx=24.0, Ly=24.0, H=24.0, gw=1.0, tol=1e-4, nx=48, ny=48, xi=1.2, r_cut=10.0, n_sigma=7.0),
]


def _oracle(c):
    return oparams.derive(c["Lx"], c["Ly"], c["H"], c["gw"], c["tol"], c["nx"], c["ny"], nz=c.get("nz", 0),
                          xi=c.get("xi", 0.0), r_cut=c.get("r_cut", 0.0), n_sigma=c.get("n_sigma", 0.0))


@pytest.mark.parametrize("c", CASES)
def test_planner_matches_oracle_derivation(c):
    d = dpslab.derive(c)
    P = _oracle(c)
    assert d["nz"] == P["nz"]
    for k in ("xi", "gt", "HE", "a", "b", "Hbar"):
        if math.isinf(P[k]):
            assert math.isinf(d[k])
        else:
            assert d[k] == pytest.approx(P[k], rel=1e-10), k
    assert d["r_cut"] == pytest.approx(P["r_cut"], rel=1e-9, abs=0.0)
    assert d["kmax"] == pytest.approx(math.pi / P["h"])


@pytest.mark.parametrize("c", CASES)
def test_tables_match_oracle(c):
    P = _oracle(c)
    zn = dpslab.table(c, 0)
    assert np.allclose(zn, ocheb.nodes(P["nz"], P["a"], P["b"]), rtol=0, atol=1e-13 * P["Hbar"])
    wz = dpslab.table(c, 1)
    assert np.allclose(wz, ocheb.quadrature_weights(P["nz"], P["a"], P["b"]), rtol=1e-12, atol=1e-14 * P["Hbar"])
    wg = dpslab.table(c, 2)
    assert np.allclose(wg, osolver.gauge_weights(P), rtol=1e-11, atol=1e-12)


def test_error_codes():
    base = dict(Lx=32.0, Ly=32.0, H=32.0, gw=1.0, tol=1e-4, nx=64, ny=64, nz=64, r_cut=4.0)
    with pytest.raises(dpslab.DpslabError) as e:
        dpslab.derive(dict(base, tol=1e-3))
    assert e.value.code == -1
    with pytest.raises(dpslab.DpslabError) as e:
        dpslab.derive(dict(base, r_cut=16.0))
    assert e.value.code == -4
    with pytest.raises(dpslab.DpslabError) as e:
        dpslab.derive(dict(base, Lx=8.0, Ly=8.0, nx=8, ny=8))   # support of 9 points > 8
    assert e.value.code == -9
    with pytest.raises(dpslab.DpslabError) as e:
        dpslab.derive(dict(base, nx=2 * 67, ny=64))    # prime factor 67 > largest radix
    assert e.value.code == -9
    with pytest.raises(dpslab.DpslabError) as e:
        dpslab.derive(dict(base, H=6.0, strict=1))     # 2 H_E > H
    assert e.value.code == -5
    d = dpslab.derive(dict(base, H=6.0))
    assert d["violations"] & 1
    with pytest.raises(dpslab.DpslabError) as e:
        dpslab.derive(dict(base, gw=-1.0))
    assert e.value.code == -1
    with pytest.raises(dpslab.DpslabError) as e:
        dpslab.derive(dict(base, precision=dpslab.MIXED + 5))
    assert e.value.code == -10
    assert dpslab.lib().dpslab_strerror(-3).decode().startswith("a charge")


def test_plan_create_without_gpu_reports_no_device():
    """On a machine without a GPU, plan creation fails with an error code
    instead of crashing (on a GPU machine this test is skipped)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(dpslab.DpslabError) as e:
        dpslab.Plan(dict(Lx=32.0, Ly=32.0, H=32.0, gw=1.0, tol=1e-4, nx=64, ny=64, nz=64, r_cut=4.0), 128)
    assert e.value.code in (-8, -7)


def test_build_watches_every_source_and_header(monkeypatch):
    # the library is rebuilt when any CUDA/C++ source or header under csrc/
    # (including the .cuh kernel headers) is newer than it
    import glob
    import os

    from paper_2101_07088_b300 import build
    csrc = os.path.join(os.path.dirname(build.__file__), "csrc")
    files = {os.path.abspath(f) for f in glob.glob(os.path.join(csrc, "*"))
             if f.endswith((".cu", ".cpp", ".h", ".cuh"))}
    assert any(f.endswith(".cuh") for f in files)
    seen = set()
    real = os.path.getmtime

    def mtime(f):
        f = os.path.abspath(f)
        if f == os.path.abspath(build.LIB):
            return float("inf")          # library newest: every dependency is examined
        seen.add(f)
        return real(f)
    monkeypatch.setattr(os.path, "exists", lambda f: True)
    monkeypatch.setattr(os.path, "getmtime", mtime)
    assert build.needs_build() is False
    assert files <= seen
