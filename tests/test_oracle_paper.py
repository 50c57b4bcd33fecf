"""The paper's own numerical tests, run on the oracle (CPU).

* Sec. 6.1, Table (ewfreeslab): four charges near the walls of a slab that
  is unbounded in x, y; the periodic solves at L = 28 and L = 32 are
  extrapolated in 1/L and compared with the free-space image series.
* Sec. 6.2, Table (ewnoparam): the answer does not depend on the splitting
  parameter xi (grids and xi as printed, against a xi = inf solve).
* Sec. 6.3, Table (energslabEw): F = -grad U by the rate of work, Eq. (w1),
  (w2), with the self potential removed (no wall charge here).
"""
import json
import os

import numpy as np
import pytest
from scipy.special import erf

from oracle import brute, params, solver
from oracle.kernels import self_potential


@pytest.fixture(scope="module")
def tables(golden_dir):
    with open(os.path.join(golden_dir, "paper_tables.json")) as f:
        return json.load(f)


def _free_space_field(pos, q, H, gw, eps, eb, et):
    """Ebar of Gaussian charges in free space (no periodicity) with the full
    image series: the averaged Coulomb kernel erf(r/(2 g_w))/(4 pi eps r)."""
    Gb, Gt = (eb - eps) / (eb + eps), (et - eps) / (et + eps)
    E = np.zeros((len(q), 3))
    a = 2.0 * gw
    for s in range(len(q)):
        zi, si = brute.image_series(pos[s, 2], H, Gb, Gt, tol=1e-20)
        src = np.stack([np.full_like(zi, pos[s, 0]), np.full_like(zi, pos[s, 1]), zi], 1)
        for t in range(len(q)):
            rv = pos[t] - src
            r = np.linalg.norm(rv, axis=1)
            m = r > 0
            r, rv, st = r[m], rv[m], si[m] * q[s]
            dG = (-erf(r / a) / r ** 2 + 2.0 / (np.sqrt(np.pi) * a) * np.exp(-(r / a) ** 2) / r) / (4 * np.pi * eps)
            E[t] += np.sum((-st * dG / r)[:, None] * rv, axis=0)
    return E


@pytest.mark.slow
def test_free_space_four_charges(tables):
    t = tables["ewfreeslab"]
    pos = np.array([c["pos"] for c in t["charges"]])
    q = np.array([c["q"] for c in t["charges"]])
    EF = _free_space_field(pos, q, t["H"], t["gw"], t["eps"], t["eps_b"], t["eps_t"])
    Es = []
    for g in t["grids"]:
        P = params.derive(g["L"], g["L"], t["H"], t["gw"], t["tol"], g["N"], g["N"],
                          eps=t["eps"], eps_b=t["eps_b"], eps_t=t["eps_t"])
        assert P["nz"] == g["nz"]
        Es.append(solver.solve(pos, q, P)["force"] / q[:, None])
    L1, L2 = t["grids"][0]["L"], t["grids"][1]["L"]
    Einf = (L2 * Es[1] - L1 * Es[0]) / (L2 - L1)
    scale = np.mean(np.linalg.norm(EF, axis=1))
    rel = (Einf - EF) / scale
    # the paper reports |rel| <= 1e-5 per component (Table (ewfreeslab))
    assert np.max(np.abs(rel)) < 3e-5, rel
    # Table (ewfreeslab) prints these errors per component; the magnitudes
    # agree to ~10% (the printed signs are all opposite: the table lists the
    # difference the other way round)
    printed = np.array([c["rel_err"] for c in t["charges"]])
    assert np.allclose(np.abs(rel), np.abs(printed), rtol=0.15), (rel, printed)
    assert np.all(np.sign(rel) == -np.sign(printed))


@pytest.mark.slow
def test_independent_of_splitting_parameter(tables):
    t = tables["ewnoparam"]
    rng = np.random.default_rng(21)
    n = 100
    pos = np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n),
                    rng.uniform(4.5 * t["gw"], t["H"] - 4.5 * t["gw"], n)], 1)
    q = np.array([1.0, -1.0] * (n // 2))
    kw = dict(eps=t["eps"], eps_b=t["eps_b"], eps_t=t["eps_t"])
    # reference without splitting (xi = inf), Sec. 3.1, on a fine grid
    Pref = params.derive(t["L"], t["L"], t["H"], t["gw"], 1e-4, 128, 128, xi=np.inf, **kw)
    ref = solver.solve(pos, q, Pref)["force"] / q[:, None]
    scale = np.mean(np.linalg.norm(ref, axis=1))
    stds = []
    for row in t["rows"]:
        P = params.derive(t["L"], t["L"], t["H"], t["gw"], t["tol"], row["N"], row["N"], **kw)
        E = solver.solve(pos, q, P)["force"] / q[:, None]
        stds.append(np.std((E - ref) / scale))
    # paper: error std 2.7e-5 ... 7.9e-5 at delta = 5e-4
    print("E2 error std per xi", stds)
    assert max(stds) < 2e-4, stds


@pytest.mark.slow
@pytest.mark.parametrize("gw", [1e-2, 1e-4])
def test_rate_of_work(tables, gw):
    t = tables["energslabEw"]
    rng = np.random.default_rng(33)
    n = 10
    pos = np.stack([rng.uniform(-t["L"], t["L"], n), rng.uniform(-t["L"], t["L"], n),
                    rng.uniform(4.5 * gw, t["H"] - 4.5 * gw, n)], 1)
    q = np.array([1.0, -1.0] * (n // 2))
    P = params.derive(t["L"], t["L"], t["H"], gw, t["tol"], t["N"], t["N"],
                      eps=t["eps"], eps_b=t["eps_b"], eps_t=t["eps_t"])
    dX = rng.standard_normal(pos.shape)
    dX /= np.linalg.norm(dX, axis=1, keepdims=True)
    d0 = t["delta0"]
    self_u = 0.5 * np.sum(q * q) * self_potential(gw, t["eps"])

    def U(p):
        return solver.solve(p, q, P)["U"] - self_u
    W1 = -(U(pos + 0.5 * d0 * dX) - U(pos - 0.5 * d0 * dX)) / d0
    W2 = float(np.sum(solver.solve(pos, q, P)["force"] * dX))
    # paper: |W1 - W2|/W1 = 2.1e-4 ... 5e-4 (with wall charge)
    print("E3 |W1-W2|/W1", gw, abs(W1 - W2) / abs(W1))
    assert abs(W1 - W2) / abs(W1) < 1e-3
