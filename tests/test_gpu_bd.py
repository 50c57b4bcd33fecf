"""Brownian dynamics on the device (dpslab_bd_*) against the oracle's
Sec. 7.1 step: the same Philox noise, steric forces on the solve's cell list,
proposals and retries as kernels in stream order. FP64 trajectories agree
with the oracle's to 1e-9 over several steps (the forces to 1e-10); the mixed
path follows the FP64 one within its force bar; a step whose proposals all
leave the slab changes nothing and is reported; counterions between charged
walls (Sec. 7.3's setting) step like the oracle."""
import numpy as np
import pytest

from gpu_helpers import oracle_params, plan_for
from oracle import bd as obd
from paper_2101_07088_b300 import build, dpslab, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gpu_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


BP = dict(dt=0.01, mu=1.0, kT=1.0, a=0.8, U0=1.0, p=6, r_m=1.6, max_disp=0.0, max_retries=8, seed=2024)


def _dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def _gpu_bp(bp):
    return dpslab.bd_params(bp["dt"], bp["mu"], bp["kT"], bp["a"], bp["U0"], bp["r_m"], bp["p"],
                            bp["max_retries"], bp["max_disp"], bp["seed"])


def _setup():
    P = oracle_params(24.0, 20.0, 20.0, 1.0, 1e-4, 48, 40, nz=37, eps_b=1 / 80, eps_t=0.5, r_cut=4.0)
    pos, q = synth.electrolyte(102, 24.0, 20.0, 1.0, 19.0, seed=3)
    return P, pos, q


def test_noise_matches_oracle():
    W = torch.empty((5000, 3), dtype=torch.float64, device="cuda")
    dpslab.bd_init_noise(77, W)
    ref = obd.normals(5000, 0, 0, 77)
    assert np.max(np.abs(W.cpu().numpy() - ref)) < 1e-13


@pytest.mark.parametrize("max_disp", [0.0, 0.05])
def test_fp64_trajectory_matches_oracle(max_disp):
    P, pos, q = _setup()
    bp = dict(BP, max_disp=max_disp)
    # steric contacts are present
    d = pos[:, None] - pos[None]
    d[..., 0] -= 24.0 * np.round(d[..., 0] / 24.0)
    d[..., 1] -= 20.0 * np.round(d[..., 1] / 20.0)
    r = np.sqrt((d ** 2).sum(-1)) + np.eye(len(q)) * 1e9
    assert (r < 2 ** (1 / 6) * 1.6).sum() > 0
    plan = plan_for(P, len(q))
    pt, qt = _dev(pos), _dev(q)
    W = torch.empty((len(q), 3), dtype=torch.float64, device="cuda")
    dpslab.bd_init_noise(bp["seed"], W)
    opos, oW = pos.copy(), obd.normals(len(q), 0, 0, bp["seed"])
    for k in range(4):
        code, r_gpu = plan.bd_step(_gpu_bp(bp), pt, qt, W, k)
        opos, oW, r_or, ok = obd.step(opos, q, oW, k, P, bp)
        assert ok and code == dpslab.OK and r_gpu == r_or
        err = np.max(np.abs(pt.cpu().numpy() - opos))
        print(f"step {k}: max position difference {err:.2e}")
        assert err < 1e-9
        assert np.max(np.abs(W.cpu().numpy() - oW)) < 1e-13


def test_mixed_follows_fp64():
    P, pos, q = _setup()
    out = {}
    for prec in (dpslab.FP64, dpslab.MIXED):
        plan = plan_for(P, len(q), precision=prec)
        pt, qt = _dev(pos), _dev(q)
        W = torch.empty((len(q), 3), dtype=torch.float64, device="cuda")
        dpslab.bd_init_noise(BP["seed"], W)
        for k in range(3):
            plan.bd_step(_gpu_bp(BP), pt, qt, W, k)
        out[prec] = pt.cpu().numpy()
    disp = np.linalg.norm(out[dpslab.FP64] - pos)
    assert np.linalg.norm(out[dpslab.MIXED] - out[dpslab.FP64]) < 1e-5 * disp


def test_rejected_step_changes_nothing():
    P, pos, q = _setup()
    plan = plan_for(P, len(q))
    pt, qt = _dev(pos), _dev(q)
    W = torch.empty((len(q), 3), dtype=torch.float64, device="cuda")
    dpslab.bd_init_noise(1, W)
    W0 = W.clone()
    bp = dict(BP, dt=50.0, max_retries=3)
    code, r = plan.bd_step(_gpu_bp(bp), pt, qt, W, 0, check=False)
    assert code == dpslab.ERR_BD_REJECTED and r == 3
    assert np.array_equal(pt.cpu().numpy(), pos) and torch.equal(W, W0)
    # the plan stays usable
    code, r = plan.bd_step(_gpu_bp(BP), pt, qt, W, 1)
    assert code == dpslab.OK


def test_counterions_between_charged_walls():
    # Sec. 7.3: only cations, walls at sigma = -N e / (2 L^2) each
    P = oracle_params(16.0, 16.0, 12.0, 1.0, 1e-4, 32, 32, nz=0, eps_b=0.2, eps_t=0.2, r_cut=4.0)
    rng = np.random.default_rng(9)
    n = 40
    pos = np.stack([rng.uniform(0, 16, n), rng.uniform(0, 16, n), rng.uniform(1.0, 11.0, n)], 1)
    q = np.ones(n)
    s = -n / (2 * 16.0 * 16.0)
    sb = np.full((32, 32), s)
    plan = plan_for(P, n)
    plan.set_wall_charge(sb, sb)
    pt, qt = _dev(pos), _dev(q)
    W = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    bp = dict(BP, a=0.5, r_m=1.0)
    dpslab.bd_init_noise(bp["seed"], W)
    opos, oW = pos.copy(), obd.normals(n, 0, 0, bp["seed"])
    for k in range(3):
        code, r_gpu = plan.bd_step(_gpu_bp(bp), pt, qt, W, k)
        opos, oW, r_or, ok = obd.step(opos, q, oW, k, P, bp, sigma_b=sb, sigma_t=sb)
        assert ok and code == dpslab.OK and r_gpu == r_or
        assert np.max(np.abs(pt.cpu().numpy() - opos)) < 1e-9
