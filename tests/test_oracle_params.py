"""Oracle parameter derivation pinned to the paper's printed tables (CPU)."""
import json
import math
import os

import pytest

from oracle import params


@pytest.fixture(scope="module")
def tables(golden_dir):
    with open(os.path.join(golden_dir, "paper_tables.json")) as f:
        return json.load(f)


def test_ewnoparam_rows(tables):
    t = tables["ewnoparam"]
    for row in t["rows"]:
        P = params.derive(t["L"], t["L"], t["H"], t["gw"], t["tol"], row["N"], row["N"])
        assert P["xi"] == pytest.approx(row["xi"], abs=0.1)   # printed 4.3, 9.2, 12.2, 26.0
        assert P["nz"] == row["nz"]
        assert P["HE"] == pytest.approx(row["HE"], abs=0.005)
        assert P["r_nf"] == pytest.approx(row["rnf"], abs=0.0101)   # printed to 2 digits


def test_ewfreeslab_setup(tables):
    t = tables["ewfreeslab"]
    for g in t["grids"]:
        P = params.derive(g["L"], g["L"], t["H"], t["gw"], t["tol"], g["N"], g["N"])
        assert P["nz"] == g["nz"]
        assert P["gt"] == pytest.approx(t["gt"], abs=5e-4)
        assert P["HE"] == pytest.approx(t["HE"], abs=5e-3)
        assert P["r_nf"] == pytest.approx(t["rnf"], abs=5e-3)
        assert P["xi"] == pytest.approx(t["xi"], abs=0.05)


def test_energy_test_setup(tables):
    t = tables["energslabEw"]
    P = params.derive(t["L"], t["L"], t["H"], 1e-2, t["tol"], t["N"], t["N"])
    assert P["nz"] == t["nz"]
    assert P["xi"] == pytest.approx(t["xi"], abs=0.06)
    assert P["gt"] == pytest.approx(t["gt"], abs=5e-3)
    assert P["HE"] == pytest.approx(t["HE"], abs=5e-3)
    assert P["r_nf"] == pytest.approx(t["rnf"], abs=5e-3)


def test_alpha(tables):
    assert params.alpha_estimate(1e-4) == pytest.approx(tables["alpha"]["1e-4"], abs=0.01)
    assert params.alpha_estimate(5e-4) == pytest.approx(tables["alpha"]["5e-4"], abs=0.01)


def test_tolerance_table():
    assert params.tolerance_constants(1e-4) == (1.4, 12, 12 / 2.8)
    assert params.tolerance_constants(5e-4) == (1.2, 10, 10 / 2.4)
    with pytest.raises(ValueError):
        params.tolerance_constants(1e-3)


def test_resolved_grid_rule():
    """Grid resolving g_w (h = g_w/2): xi from the averaged-kernel cutoff rule.
    At the chosen xi the ratio equals delta; just below xi it is above."""
    from oracle.kernels import near_kernel_dr
    for tol in (1e-4, 5e-4):
        P = params.derive(32.0, 32.0, 32.0, 1.0, tol, 64, 64, nz=64, r_cut=4.0)
        ref = near_kernel_dr(4.0, 1.0, 0.0)
        ratio = abs(near_kernel_dr(4.0, 1.0, P["xi"]) / ref)
        assert ratio == pytest.approx(tol, rel=1e-9)
        assert abs(near_kernel_dr(4.0, 1.0, 0.99 * P["xi"]) / ref) > tol
        assert P["HE"] == pytest.approx(P["n_sigma"] * math.sqrt(0.25 / P["xi"] ** 2 + 1.0))
    P = params.derive(32.0, 32.0, 32.0, 1.0, 1e-4, 64, 64, nz=64, r_cut=4.0)
    assert P["xi"] == pytest.approx(20.82, abs=0.01)


def test_paper_rule_infeasible_without_cutoff():
    with pytest.raises(ValueError):
        params.derive(32.0, 32.0, 32.0, 1.0, 1e-4, 64, 64, nz=64)
