"""Pins of the oracle's forward model (Section 2.1, Eq. 1-2) to facts that do
not come from the oracle itself:

* conservation: with rho = 0 the no-flux scheme keeps sum(u) = u0 exactly
  (up to rounding), and no mass enters voxels outside the domain (Eq. 2);
* the exact second moment of the explicit scheme in free space: for a
  lattice random walk each step adds 2 D_w dt to the variance along every
  axis, so after n steps of dt = T/n the variance is 2 D_w T per axis and
  the mean stays at the seed (also on a grid whose three sizes differ);
* pure reaction: with D_w = 0 every voxel follows the logistic equation,
  whose solution is u0 e^{rho t} / (1 - u0 + u0 e^{rho t}); explicit Euler
  converges to it at first order;
* reflection symmetry of the solution on a symmetric atlas with a central
  seed (catches transposed strides);
* the Fisher-KPP front: in one dimension the front travels at
  2 sqrt(D_w rho) (Fisher 1937; Kolmogorov, Petrovsky & Piskunov 1937),
  less a logarithmic delay (Bramson 1983) and the explicit-Euler slowdown;
* the steady state of pure diffusion with no-flux boundaries: uniform
  u0 / |Omega| on the connected domain;
* the maximum principle 0 <= u <= 1 for cfl <= 1.
"""
import numpy as np
import pytest

import oracle
from paper_2205_04550_gb300 import synth


def _moments(u):
    nz, ny, nx = u.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    mass = u.sum()
    mean = [float((u * c).sum() / mass) for c in (x, y, z)]
    var = [float((u * (c - m) ** 2).sum() / mass) for c, m in zip((x, y, z), mean)]
    return mass, mean, var


def test_mass_conserved_and_no_flux_into_csf():
    tissue = synth.brain_tissue((33, 29, 25))
    theta = (20.0, 14.0, 12.0, 0.8, 0.0, 30.0)
    assert tissue[12, 14, 20] > 0
    u, n = oracle.rd_simulate(tissue, theta, u0=0.7, cfl=0.9)
    assert n == int(np.ceil(30.0 * (6.0 * 0.8 * 1.0 + 0.0) / 0.9))
    assert abs(u.sum() - 0.7) <= 1e-13
    assert np.all(u[tissue == 0] == 0.0)
    assert u.min() >= 0.0
    # it did spread into grey matter
    assert np.count_nonzero(u[tissue == np.float32(0.1)]) > 0


@pytest.mark.parametrize("shape,seed", [((41, 41, 41), (20, 20, 20)),
                                        ((43, 39, 45), (21, 19, 22))])
def test_free_space_second_moment_is_exact(shape, seed):
    nx, ny, nz = shape
    tissue = np.ones((nz, ny, nx), np.float32)
    d_w, t_end = 0.5, 5.0
    u, n = oracle.rd_simulate(tissue, (*seed, d_w, 0.0, t_end), u0=1.0, cfl=0.9)
    assert n == 17 and n < min(shape) // 2    # the walk never reaches an edge
    mass, mean, var = _moments(u)
    assert abs(mass - 1.0) <= 1e-13
    np.testing.assert_allclose(mean, seed, rtol=0, atol=1e-12)
    np.testing.assert_allclose(var, [2.0 * d_w * t_end] * 3, rtol=1e-12)


def test_pure_reaction_converges_to_logistic_solution():
    tissue = np.ones((3, 3, 3), np.float32)
    rho, t_end, u0 = 0.3, 12.0, 0.05
    exact = u0 * np.exp(rho * t_end) / (1.0 - u0 + u0 * np.exp(rho * t_end))
    errs = []
    for cfl in (0.1, 0.05, 0.025):
        u, n = oracle.rd_simulate(tissue, (1, 1, 1, 0.0, rho, t_end), u0=u0, cfl=cfl)
        assert n == int(np.ceil(t_end * rho / cfl))
        assert np.count_nonzero(u) == 1
        errs.append(abs(u[1, 1, 1] - exact))
    assert errs[-1] < 5e-3
    for a, b in zip(errs, errs[1:]):
        assert 1.8 < a / b < 2.2       # first order in dt


def test_reflection_symmetry_on_symmetric_atlas():
    shape = (33, 29, 25)
    tissue = synth.brain_tissue(shape).copy()
    # fill the central ventricle with white matter (a box symmetric about the
    # centre voxel, inside the white-matter ellipsoid) to seed at the centre
    box = tissue[12 - 2:12 + 3, 14 - 5:14 + 6, 16 - 3:16 + 4]
    box[box == 0] = np.float32(1.0)
    u, _ = oracle.rd_simulate(tissue, (16.0, 14.0, 12.0, 0.6, 0.15, 25.0), u0=1.0, cfl=0.9)
    np.testing.assert_allclose(u, u[::-1, :, :], rtol=0, atol=1e-14)
    np.testing.assert_allclose(u, u[:, ::-1, :], rtol=0, atol=1e-14)
    np.testing.assert_allclose(u, u[:, :, ::-1], rtol=0, atol=1e-14)
    assert np.count_nonzero(u > 1e-3) > 500
    assert np.count_nonzero(u[tissue == np.float32(0.1)]) > 0


def test_fisher_kpp_front_speed():
    tissue = np.ones((1, 1, 300), np.float32)
    d_w, rho = 1.0, 0.25

    def front(t):
        u, _ = oracle.rd_simulate(tissue, (0, 0, 0, d_w, rho, t), u0=1.0, cfl=0.9)
        r = u.reshape(-1)
        i = int(np.argmax(r < 0.5))
        return i - 1 + (r[i - 1] - 0.5) / (r[i - 1] - r[i])

    speed = (front(140.0) - front(80.0)) / 60.0
    # 2 sqrt(D rho) = 1; Bramson's delay (3 / (2 lambda*)) d(ln t)/dt ~ 0.03
    # and the explicit-Euler slowdown ~ 0.03 at cfl 0.9 lower it slightly
    assert 0.90 <= speed <= 1.0, speed


def test_steady_state_is_uniform_on_domain():
    shape = (13, 11, 9)
    tissue = synth.brain_tissue(shape)
    omega = tissue > 0
    z, y, x = np.argwhere(omega)[0]
    u, _ = oracle.rd_simulate(tissue, (x, y, z, 1.0, 0.0, 2500.0), u0=1.0, cfl=0.9)
    np.testing.assert_allclose(u[omega], 1.0 / omega.sum(), rtol=1e-6)
    assert np.all(u[~omega] == 0.0)


def test_maximum_principle_and_saturation():
    shape = (24, 20, 16)
    tissue = synth.brain_tissue(shape)
    theta = synth.rd_params(shape, 11, np.arange(4))
    for th in theta:
        th = th.copy()
        th[5] = min(th[5], 60.0)
        u, n = oracle.rd_simulate(tissue, th, u0=1.0, cfl=1.0)
        assert n >= 1
        assert u.min() >= 0.0 and u.max() <= 1.0
    # the step count follows the largest diffusivity: a map with m up to 3
    x, y, z = theta[0, :3]
    u, n = oracle.rd_simulate(tissue * np.float32(3.0), (x, y, z, 0.4, 0.1, 40.0), cfl=1.0)
    assert n == int(np.ceil(40.0 * (6.0 * 0.4 * 3.0 + 0.1) / 1.0))
    assert u.min() >= 0.0 and u.max() <= 1.0
    # long proliferation saturates the whole connected domain at 1
    u, _ = oracle.rd_simulate(np.ones((5, 5, 5), np.float32), (2, 2, 2, 0.5, 0.5, 400.0))
    np.testing.assert_allclose(u, 1.0, rtol=0, atol=1e-9)


def test_rejects_seed_outside_domain_and_bad_cfl():
    tissue = synth.brain_tissue((33, 29, 25))
    with pytest.raises(ValueError):
        oracle.rd_simulate(tissue, (0, 0, 0, 0.5, 0.1, 10.0))       # outside the brain
    with pytest.raises(ValueError):
        oracle.rd_simulate(tissue, (16, 14, 12, 0.5, 0.1, 10.0))    # in the ventricle
    with pytest.raises(ValueError):
        oracle.rd_simulate(tissue, (20, 14, 12, 0.5, 0.1, 10.0), cfl=1.5)
    u, n = oracle.rd_simulate(tissue, (20, 14, 12, 0.5, 0.1, 0.0), u0=0.3)
    assert n == 0 and u.sum() == 0.3
