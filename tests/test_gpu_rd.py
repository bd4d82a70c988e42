"""Parity of the GPU forward model (Section 2.1, Eq. 1-2) with the oracle.

The GPU computes in binary32, the oracle in binary64.  Tolerance, from the
arithmetic of one GPU step (u, the face coefficients h, a = dt D_w and
b = dt rho rounded to binary32; u in [0, 1]; a sum_j h_j <= cfl <= 1):
the six differences, products and sums of the flux cost at most 8 units of
2^-24 relative to a sum_j h_j |u_j - u| <= 1, the coefficient, a and b
roundings 3 more, the logistic term 1 (b u (1 - u) <= 1/4) and the final
additions 2 (|u| <= 1), so one step adds at most delta = 14 * 2^-24 to the
error.  The diffusion part of a step is a convex combination (it never
grows an error) and the logistic part multiplies it by at most 1 + b, so
after n steps

    |u_gpu - u_oracle| <= delta ((1 + b)^n - 1) / b      (delta n for b = 0).

Beyond that bound: the support must agree (u_gpu > 0 wherever the oracle
holds a value above 1e-20 -- binary32 represents it -- and the oracle is
positive wherever u_gpu is), and u_gpu is exactly 0 outside the domain; these
catch a tile skipped by mistake, whose values would be far below the bound.
"""
import numpy as np
import pytest

import oracle
from paper_2205_04550_gb300 import (DBQ_STORE_BITS, Database, DbqError, ForwardModel, _dbq,
                                    synth)
from tests._gpu_helpers import assert_hits_equal

pytestmark = pytest.mark.gpu

DELTA = 14 * 2.0 ** -24


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    from paper_2205_04550_gb300 import build
    build.build()
    return _t


def _bound(theta, steps):
    if steps == 0:
        return 0.0
    b = theta[5] / steps * theta[4]
    return DELTA * steps if b == 0 else DELTA * ((1.0 + b) ** steps - 1.0) / b


def _check(u_gpu, tissue, theta, steps, u0, cfl):
    # u0 is a binary32 argument of the C call: the oracle starts from that value
    ref, n = oracle.rd_simulate(tissue, theta, u0=float(np.float32(u0)), cfl=cfl)
    assert steps == n
    err = np.abs(u_gpu.astype(np.float64) - ref)
    assert err.max() <= _bound(theta, n), (err.max(), _bound(theta, n))
    assert np.all(u_gpu[ref > 1e-20] > 0)
    assert np.all(ref[u_gpu > 0] > 0)
    assert np.all(u_gpu[tissue == 0] == 0)
    return err.max()


def _params(shape, count, seed=5, t_cap=None):
    th = synth.rd_params(shape, seed, np.arange(count))
    if t_cap is not None:
        th[:, 5] = np.minimum(th[:, 5], t_cap)
    return th


@pytest.mark.parametrize("shape,batch", [((33, 29, 25), 3), ((64, 40, 17), 16)])
def test_forward_model_matches_oracle(torch, shape, batch):
    nx, ny, nz = shape
    tissue = synth.brain_tissue(shape)
    th = _params(shape, 5, t_cap=60.0)
    th[1, 5] = 0.0                               # T_end = 0: the initial condition
    th[2, 4] = 0.0                               # pure diffusion
    with ForwardModel(tissue, batch=batch) as fm:
        u, steps = fm.simulate(th, u0=0.8, cfl=0.9)
        st = fm.stats()
    assert st["slots"] == min(batch, 5)
    assert st["step_launches"] >= max(steps) and st["step_launches"] <= sum(steps)
    for j in range(5):
        _check(u[j], tissue, th[j], int(steps[j]), 0.8, 0.9)
    assert steps[1] == 0 and u[1].sum() == np.float32(0.8)


def test_forward_model_device_output_and_cfl(torch):
    shape = (48, 48, 32)
    nx, ny, nz = shape
    tissue = synth.brain_tissue(shape)
    th = _params(shape, 4, seed=9, t_cap=40.0)
    out = torch.zeros((4, nz, ny, nx), dtype=torch.float32, device="cuda")
    with ForwardModel(torch.from_numpy(tissue).cuda(), batch=2) as fm:
        _, steps = fm.simulate(th, out=out, u0=1.0, cfl=0.5)
    u = out.cpu().numpy()
    for j in range(4):
        _check(u[j], tissue, th[j], int(steps[j]), 1.0, 0.5)
        assert u[j].max() <= 1.0 and u[j].min() >= 0.0


def test_forward_model_full_size_128(torch):
    """The bench's grid and batch size; one simulation checked in full."""
    shape = (128, 128, 128)
    tissue = synth.brain_tissue(shape)
    th = _params(shape, 16, seed=3)
    with ForwardModel(tissue, batch=16) as fm:
        u, steps = fm.simulate(th, u0=1.0, cfl=0.9)
    j = int(np.argmin(steps))                   # the cheapest one for the oracle
    _check(u[j], tissue, th[j], int(steps[j]), 1.0, 0.9)
    # every simulation: bounded and exactly 0 outside the domain
    assert np.all(u >= 0) and np.all(u <= 1)
    assert np.all(u[:, tissue == 0] == 0)


def test_simulated_database_query(torch):
    """Simulations feed the query: their masks, queried with one of them,
    give the oracle's hits (and the planted entry itself at score 1)."""
    shape = (64, 64, 48)
    nx, ny, nz = shape
    tissue = synth.brain_tissue(shape)
    th = _params(shape, 24, seed=21)
    with ForwardModel(tissue, batch=8) as fm:
        u, _ = fm.simulate(th)
    with Database(shape, 24, DBQ_STORE_BITS, 0.6, 0.25, n_params=6) as db:
        db.load(0, u, params=th)
        db.build()
        hits, params = db.query(u[7], 5)
    ref = oracle.query(u, u[7], np.float32(0.6), np.float32(0.25), 5)
    assert_hits_equal(hits, ref, 5)
    assert hits["index"][0] == 7 and hits["score"][0] == 1.0
    np.testing.assert_array_equal(params[0], th[7])


def test_forward_model_errors(torch):
    shape = (33, 29, 25)
    tissue = synth.brain_tissue(shape)
    bad = tissue.copy()
    bad[3, 3, 3] = -1.0
    with pytest.raises(DbqError, match="EINVAL"):
        ForwardModel(bad)
    bad[3, 3, 3] = np.nan
    with pytest.raises(DbqError, match="EINVAL"):
        ForwardModel(bad)
    with ForwardModel(tissue, batch=2) as fm:
        with pytest.raises(DbqError, match="EINVAL"):
            fm.simulate([[16, 14, 12, 0.5, 0.1, 10.0]])       # seed in the ventricle
        with pytest.raises(DbqError, match="EINVAL"):
            fm.simulate([[20, 14, 12, 0.5, 0.1, 10.0]], cfl=1.5)
        with pytest.raises(DbqError, match="EINVAL"):
            fm.simulate([[20, 14, 12, -0.5, 0.1, 10.0]])
        with pytest.raises(DbqError, match="EINVAL"):
            fm.simulate([[200, 14, 12, 0.5, 0.1, 10.0]])
        u, steps = fm.simulate(np.zeros((0, 6)))
        assert u.shape[0] == 0
