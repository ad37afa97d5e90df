"""CPU pins for the FP64 oracle: every check here is independent of the oracle's own code.

Pins used (none re-types the oracle's formula):
  * closed-form pair values at special distances (r = sigma, the LJ minimum, the cutoff);
  * a two-atom system across the periodic boundary (minimum image and force sign);
  * O(N^2) brute force against the cell-list evaluation on small random boxes;
  * lattice sums: perfect fcc WCA has U = F = 0, perfect fcc LJ has the shell sum computed here
    by enumerating lattice vectors;
  * invariants: zero net force, sum u_i = 2U, momentum conservation, bounded energy drift,
    time reversibility, second-order convergence against a tight ODE integration;
  * neighbour sets against the brute-force distance definition;
  * the paper's printed neighbour statistics (tests/golden/paper_statistics.json);
  * finite differences for the Jacobian, the parameter derivatives and the adjoint.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2003_14061_gb300 import inputs

RC_WCA = 2.0 ** (1.0 / 6.0)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def wca():
    return oracle.pot(eps=1.0, sigma=1.0, rc=RC_WCA, shift=True)


def lj(rc=2.5):
    return oracle.pot(eps=1.0, sigma=1.0, rc=rc, shift=True)


# ---------------------------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------------------------
def test_pair_closed_forms():
    # WCA at r = sigma: 4(1 - 1) + 1 = 1, force magnitude 24 (2 - 1) = 24.
    u, g = oracle.pair(wca(), 1.0)
    assert u == pytest.approx(1.0, abs=1e-15)
    assert g * 1.0 == pytest.approx(24.0, abs=1e-13)
    # continuity at the WCA cutoff (the LJ minimum): u and f vanish
    r2 = RC_WCA ** 2 * (1 - 1e-12)
    u, g = oracle.pair(wca(), r2)
    assert abs(u) < 1e-9 and abs(g) < 1e-9
    assert oracle.pair(wca(), RC_WCA ** 2) == (0.0, 0.0)
    assert oracle.pair(wca(), 4.0) == (0.0, 0.0)
    # shifted LJ at r = sigma: u_LJ(1) = 0, so u = -u_LJ(2.5) = -4 (2.5^-12 - 2.5^-6)
    # = -4 (1.6777216e-5 - 4.096e-3) = 0.016316891136 (exact decimals)
    u, g = oracle.pair(lj(), 1.0)
    assert u == pytest.approx(0.016316891136, abs=1e-14)
    assert g == pytest.approx(24.0, abs=1e-13)
    # LJ minimum at r = 2^(1/6): u_LJ = -1, zero force
    u, g = oracle.pair(lj(), RC_WCA ** 2)
    assert u == pytest.approx(-1.0 + 0.016316891136, abs=1e-13)
    assert abs(g) < 1e-13
    u, g = oracle.pair(oracle.pot(rc=2.5, shift=False), RC_WCA ** 2)
    assert u == pytest.approx(-1.0, abs=1e-14)
    # scaling: u(r; eps, sigma) = eps u(r/sigma; 1, 1)
    p = oracle.pot(eps=2.0, sigma=1.5, rc=1.5 * 2.5, shift=True)
    u1, g1 = oracle.pair(p, (1.5 * 1.1) ** 2)
    u0, g0 = oracle.pair(lj(), 1.1 ** 2)
    assert u1 == pytest.approx(2.0 * u0, rel=1e-13)
    assert g1 * 1.5 * 1.1 == pytest.approx(2.0 * g0 * 1.1 / 1.5, rel=1e-13)


def test_two_atoms_across_boundary():
    L = 5.0
    box = np.array([L, L, L])
    x = np.array([[0.05, 2.0, 2.0], [L - 0.95, 2.0, 2.0]])   # separation 1.0 through x = 0
    for method in ("brute", "cells"):
        f, ua, U, W = oracle.forces(x, box, wca(), method)
        assert f[0] == pytest.approx([24.0, 0.0, 0.0], abs=1e-12)   # pushed towards +x
        assert f[1] == pytest.approx([-24.0, 0.0, 0.0], abs=1e-12)
        assert U == pytest.approx(1.0, abs=1e-14)
        assert ua == pytest.approx([1.0, 1.0], abs=1e-14)
        assert W == pytest.approx(24.0, abs=1e-12)                  # r . f = 1 * 24


# ---------------------------------------------------------------------------------------------
# brute force vs cell list
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("ncell,rho,amp,pot_name", [(2, 0.8, 0.15, "wca"), (3, 0.8, 0.2, "wca"),
                                                   (3, 0.85, 0.1, "lj"), (4, 0.5, 0.3, "lj")])
def test_brute_matches_cells(ncell, rho, amp, pot_name):
    x, box = inputs.fcc_lattice(ncell, rho)
    x = inputs.perturb(x, box, amp, seed=11 + ncell)
    p = wca() if pot_name == "wca" else lj()
    fb, ub, Ub, Wb = oracle.forces(x, box, p, "brute")
    fc, uc, Uc, Wc = oracle.forces(x, box, p, "cells")
    scale = np.abs(fb).max() + 1.0
    assert np.abs(fb - fc).max() <= 1e-12 * scale
    assert np.abs(ub - uc).max() <= 1e-12 * (np.abs(ub).max() + 1)
    assert Uc == pytest.approx(Ub, rel=1e-12, abs=1e-12)
    assert Wc == pytest.approx(Wb, rel=1e-12, abs=1e-12)


def test_brute_matches_cells_orthorhombic():
    rng = np.random.default_rng(5)
    box = np.array([6.0, 4.5, 7.5])
    # jittered simple-cubic points, far from overlap
    g = np.stack(np.meshgrid(np.arange(5), np.arange(4), np.arange(6), indexing="ij"), -1).reshape(-1, 3)
    x = (g + 0.5 + rng.uniform(-0.2, 0.2, g.shape)) * (box / np.array([5, 4, 6]))
    x = np.mod(x, box)
    fb, _, Ub, Wb = oracle.forces(x, box, lj(1.4), "brute")
    fc, _, Uc, Wc = oracle.forces(x, box, lj(1.4), "cells")
    assert np.abs(fb - fc).max() <= 1e-12 * (np.abs(fb).max() + 1)
    assert Uc == pytest.approx(Ub, rel=1e-12)


# ---------------------------------------------------------------------------------------------
# lattice sums
# ---------------------------------------------------------------------------------------------
def test_fcc_wca_lattice_is_force_free():
    # nearest-neighbour distance a/sqrt(2) = 1.2091 > 2^(1/6): no pair interacts
    x, box = inputs.fcc_lattice(6, 0.8)
    f, ua, U, W = oracle.forces(x, box, wca())
    assert U == 0.0 and W == 0.0 and np.all(f == 0.0)


def _fcc_shell_sum(rho, rc):
    a = (4.0 / rho) ** (1.0 / 3.0)
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    k = int(math.ceil(rc / a)) + 1
    r = np.arange(-k, k + 1)
    cells = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    pts = (cells[:, None, :] + basis[None]).reshape(-1, 3) * a
    d = np.sqrt((pts ** 2).sum(1))
    d = d[(d > 0) & (d < rc)]
    u = 4 * (d ** -12 - d ** -6) - 4 * (rc ** -12 - rc ** -6)
    return 0.5 * u.sum(), len(d)


def test_fcc_lj_lattice_sum():
    expect, nshell = _fcc_shell_sum(0.8442, 2.5)
    assert nshell == 12 + 6 + 24 + 12                  # four shells inside r_c = 2.5
    assert expect == pytest.approx(-6.33281, abs=5e-6)
    x, box = inputs.fcc_lattice(8, 0.8442)
    f, ua, U, W = oracle.forces(x, box, lj())
    assert U / x.shape[0] == pytest.approx(expect, rel=1e-12)
    assert np.abs(f).max() < 1e-10


# ---------------------------------------------------------------------------------------------
# invariants of forces and props
# ---------------------------------------------------------------------------------------------
def test_force_invariants():
    x, box = inputs.fcc_lattice(5, 0.8442)
    x = inputs.perturb(x, box, 0.12, seed=3)
    f, ua, U, W = oracle.forces(x, box, lj())
    assert np.abs(f.sum(0)).max() <= 1e-12 * np.abs(f).sum()       # Newton's third law
    assert ua.sum() == pytest.approx(2.0 * U, rel=1e-12)            # sum u_i = 2U


def test_props_ideal_lattice():
    x, box = inputs.fcc_lattice(5, 0.8)      # no interacting pairs under WCA
    n = x.shape[0]
    v = inputs.maxwell(n, 1.3, seed=9)
    pr = oracle.props(x, v, box, wca())
    U, K, W, P, px, py, pz, vmax = pr
    assert U == 0.0 and W == 0.0
    assert K == pytest.approx(1.5 * (n - 1) * 1.3, rel=1e-12)       # generator fixes T exactly
    V = box.prod()
    assert P == pytest.approx(2.0 * K / (3.0 * V), rel=1e-12)       # ideal gas: P V = (2/3) K
    assert abs(px) + abs(py) + abs(pz) < 1e-10
    assert vmax == pytest.approx(np.sqrt((v ** 2).sum(1)).max(), rel=1e-15)


# ---------------------------------------------------------------------------------------------
# integrator
# ---------------------------------------------------------------------------------------------
def _min_image(d, box):
    return d - box * np.round(d / box)


def test_kdk_conserves_momentum_and_energy():
    # Leapfrog does not conserve E exactly; its error is bounded and O(dt^2).  From a melting
    # lattice the largest excursion at dt = 0.005 is ~7e-4 of E, and it shrinks 4x per halving.
    x, box = inputs.fcc_lattice(8, 0.8)
    v = inputs.maxwell(x.shape[0], 1.0, seed=1)
    errs = []
    for dt, nsteps in ((0.005, 1000), (0.0025, 2000)):
        x1, v1, pr, _ = oracle.run(x, v, box, wca(), dt=dt, nsteps=nsteps)
        E = pr[:, 0] + pr[:, 1]
        assert np.abs(pr[:, 4:7]).max() < 1e-10                      # momentum conserved
        errs.append(np.abs(E - E[0]).max() / abs(E[0]))
        if dt == 0.005:
            assert np.std(E[len(E) // 2:]) / abs(E[0]) < 5e-5        # bounded fluctuation
            assert pr[-1, 0] > 0.01 * x.shape[0]                      # the lattice has melted
    assert errs[0] < 1e-3
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_kdk_time_reversible():
    x, box = inputs.fcc_lattice(4, 0.8442)
    x = inputs.perturb(x, box, 0.05, seed=4)
    v = inputs.maxwell(x.shape[0], 0.72, seed=5)
    x1, v1, _, _ = oracle.run(x, v, box, lj(), dt=0.005, nsteps=100, with_props=False)
    x2, v2, _, _ = oracle.run(x1, -v1, box, lj(), dt=0.005, nsteps=100, with_props=False)
    assert np.abs(_min_image(x2 - x, box)).max() < 1e-9
    assert np.abs(v2 + v).max() < 1e-9


def test_kdk_second_order_against_ode():
    scipy_integrate = pytest.importorskip("scipy.integrate")
    # head-on two-atom collision along x in a large box (cells 8 per axis)
    L = 10.0
    box = np.array([L, L, L])
    x0 = np.array([[4.0, 5.0, 5.0], [5.05, 5.0, 5.0]])
    v0 = np.array([[1.0, 0.0, 0.0], [-1.0, 0.0, 0.0]])
    T = 0.4

    def rhs(t, y):
        r = y[1] - y[0]
        rr = abs(r)
        if rr < RC_WCA:
            g = 24.0 * (2 * rr ** -14 - rr ** -8)
            f0 = -g * r
        else:
            f0 = 0.0
        return [y[2], y[3], f0, -f0]

    sol = scipy_integrate.solve_ivp(rhs, (0, T), [4.0, 5.05, 1.0, -1.0], rtol=1e-12, atol=1e-12,
                                    method="DOP853")
    exact = sol.y[:2, -1]
    errs = []
    for dt in (0.004, 0.002):
        nsteps = int(round(T / dt))
        x1, v1, _, _ = oracle.run(x0, v0, box, wca(), dt=dt, nsteps=nsteps, with_props=False)
        errs.append(np.abs(x1[:, 0] - exact).max())
    assert errs[0] < 1e-3
    assert 3.0 < errs[0] / errs[1] < 5.0        # second order: halving dt quarters the error


# ---------------------------------------------------------------------------------------------
# cells and neighbour sets
# ---------------------------------------------------------------------------------------------
def test_cells_and_order():
    rng = np.random.default_rng(2)
    box = np.array([9.0, 7.0, 8.0])
    x = rng.uniform(0, 1, (3000, 3)) * box
    nc, cell = oracle.cells(x, box, 1.5)
    assert list(nc) == [6, 4, 5]
    w = box / nc
    c = np.stack([cell % nc[0], (cell // nc[0]) % nc[1], cell // (nc[0] * nc[1])], 1)
    assert np.all(c * w <= x + 1e-12) and np.all(x < (c + 1) * w + 1e-12)
    ncells = int(np.prod(nc))
    start, order = oracle.cell_order(cell, ncells)
    assert np.array_equal(order, np.argsort(cell, kind="stable"))
    assert np.array_equal(np.diff(start), np.bincount(cell, minlength=ncells))


def _definition_pairs(x, box, rl):
    d = _min_image(x[None, :, :] - x[:, None, :], box)
    r = np.sqrt((d ** 2).sum(-1))
    np.fill_diagonal(r, np.inf)
    return r


@pytest.mark.parametrize("fp32", [False, True])
def test_neighbour_sets_match_definition(fp32):
    x, box = inputs.fcc_lattice(5, 0.8)
    x = inputs.perturb(x, box, 0.25, seed=21)
    rc, skin = RC_WCA, 0.4
    nc, counts, off, nb = oracle.neighbours(x, box, rc, skin, fp32=fp32)
    r = _definition_pairs(x, box, rc + skin)
    n = x.shape[0]
    got = np.zeros((n, n), dtype=bool)
    for i in range(n):
        got[i, nb[off[i]:off[i + 1]]] = True
        assert np.all(np.diff(nb[off[i]:off[i + 1]]) > 0)
    want = r < rc + skin
    diff = got != want
    band = 1e-5 if fp32 else 1e-9
    assert np.all(np.abs(r[diff] - (rc + skin)) < band)
    assert np.array_equal(got, got.T)                 # the criterion is symmetric in i, j
    assert np.array_equal(counts, got.sum(1))


def test_neighbour_count_perfect_fcc():
    # rho = 0.8: first shell 12 at 1.2091, second 6 at 1.7100 > r_c + 0.4 = 1.5225
    x, box = inputs.fcc_lattice(6, 0.8)
    for fp32 in (True, False):
        nc, counts, off, nb = oracle.neighbours(x, box, RC_WCA, 0.4, fp32=fp32)
        assert np.all(counts == 12)


# ---------------------------------------------------------------------------------------------
# the paper's neighbour statistics (Sec. 4.1 item 5)
# ---------------------------------------------------------------------------------------------
def _equilibrate(x, v, box, p, T, nsteps, chunk=100):
    for _ in range(nsteps // chunk):
        x, v, _, _ = oracle.run(x, v, box, p, dt=0.005, nsteps=chunk, with_props=False)
        v = v - v.mean(0)
        v *= math.sqrt(T * 3 * (len(v) - 1) / (v ** 2).sum())
    return x, v


@pytest.mark.parametrize("name", ["SP", "LJ"])
def test_paper_mean_neighbour_counts(name):
    ref = json.load(open(os.path.join(GOLDEN, "paper_statistics.json")))[name]
    x, box = inputs.fcc_lattice(7, ref["rho"])
    v = inputs.maxwell(x.shape[0], ref["T"], seed=7)
    p = oracle.pot(rc=ref["rc"], shift=True)
    x, v = _equilibrate(x, v, box, p, ref["T"], 1500)
    nc, counts, off, nb = oracle.neighbours(x, box, ref["rc"], ref["skin"], fp32=False)
    assert counts.mean() == pytest.approx(ref["mean_neighbours"], rel=0.10)


# ---------------------------------------------------------------------------------------------
# derivatives
# ---------------------------------------------------------------------------------------------
def _snapshot(seed=31, ncell=3, rho=0.8, amp=0.15):
    x, box = inputs.fcc_lattice(ncell, rho)
    return inputs.perturb(x, box, amp, seed=seed), box


@pytest.mark.parametrize("pot_name", ["wca", "lj"])
def test_force_jvp_matches_finite_difference(pot_name):
    p = wca() if pot_name == "wca" else lj(1.8)
    x, box = _snapshot(rho=0.9 if pot_name == "lj" else 0.8)
    lam = np.random.default_rng(1).standard_normal(x.shape)
    h = 1e-6
    fp, _, _, _ = oracle.forces(x + h * lam, box, p)
    fm, _, _, _ = oracle.forces(x - h * lam, box, p)
    fd = (fp - fm) / (2 * h)
    jv = oracle.force_jvp(x, box, p, lam)
    assert np.linalg.norm(jv - fd) <= 1e-6 * np.linalg.norm(fd)
    b = np.random.default_rng(2).standard_normal(x.shape)
    jb = oracle.force_jvp(x, box, p, b)
    assert np.vdot(lam, jb) == pytest.approx(np.vdot(jv, b), rel=1e-12)   # J is symmetric


def test_param_grads_match_finite_difference():
    x, box = _snapshot(amp=0.2)
    h = 1e-6
    fe, fs, ue, us = oracle.param_grads(x, box, wca())
    # eps
    fp, _, Up, _ = oracle.forces(x, box, oracle.pot(eps=1 + h, rc=RC_WCA))
    fm, _, Um, _ = oracle.forces(x, box, oracle.pot(eps=1 - h, rc=RC_WCA))
    assert ue == pytest.approx((Up - Um) / (2 * h), rel=1e-7)
    assert np.abs(fe - (fp - fm) / (2 * h)).max() <= 1e-6 * np.abs(fe).max()
    # sigma, with the WCA cutoff moving as 2^(1/6) sigma
    ps = oracle.pot(sigma=1 + h, rc=RC_WCA * (1 + h))
    pm = oracle.pot(sigma=1 - h, rc=RC_WCA * (1 - h))
    fp, _, Up, _ = oracle.forces(x, box, ps)
    fm, _, Um, _ = oracle.forces(x, box, pm)
    assert us == pytest.approx((Up - Um) / (2 * h), rel=1e-6)
    assert np.abs(fs - (fp - fm) / (2 * h)).max() <= 1e-5 * np.abs(fs).max()


def test_adjoint_matches_finite_difference():
    # The WCA force has a kink in its derivative at r_c, so over tens of steps the loss is only
    # piecewise smooth in the parameters: central differences converge to the adjoint as h
    # shrinks (1e-7 here) and sit 1e-3 (eps) to 1e-2 (sigma) away at h = 1e-4.
    x, box = _snapshot(seed=41, ncell=3, amp=0.1)
    n = x.shape[0]
    v = inputs.maxwell(n, 1.0, seed=42)
    S, dt = 30, 0.005
    loss, ge, gs, gv, _, _ = oracle.adjoint(x, v, box, wca(), dt=dt, nsteps=S)
    assert loss == pytest.approx(oracle.loss(x, v, box, wca(), dt=dt, nsteps=S), rel=1e-14)

    def L(eps=1.0, sig=1.0, vv=v):
        return oracle.loss(x, vv, box, oracle.pot(eps=eps, sigma=sig, rc=RC_WCA * sig), dt=dt, nsteps=S)

    # sigma also moves the cutoff, so it needs the smaller step to leave the kinks behind
    h = 1e-7
    assert ge == pytest.approx((L(eps=1 + h) - L(eps=1 - h)) / (2 * h), rel=1e-6)
    assert gs == pytest.approx((L(sig=1 + h) - L(sig=1 - h)) / (2 * h), rel=1e-6)
    h = 1e-4
    assert ge == pytest.approx((L(eps=1 + h) - L(eps=1 - h)) / (2 * h), rel=2e-3)
    assert gs == pytest.approx((L(sig=1 + h) - L(sig=1 - h)) / (2 * h), rel=2e-2)
    rng = np.random.default_rng(3)
    h = 1e-5
    for _ in range(4):
        i, a = int(rng.integers(n)), int(rng.integers(3))
        vp = v.copy(); vp[i, a] += h
        vm = v.copy(); vm[i, a] -= h
        fd = (L(vv=vp) - L(vv=vm)) / (2 * h)
        assert gv[i, a] == pytest.approx(fd, rel=1e-5, abs=1e-7)


def test_adjoint_single_step_closed_form():
    # One step: L = U(x_1) + |v_1|^2 with x_1 = x_0 + dt (v_0 + c F_0), v_1 = v_0 + c (F_0 + F_1).
    # dL/dv_0 = -dt F_1 + 2 v_1 + 2 c dt J(x_1) v_1, written out with the oracle's force and
    # Jacobian evaluations (each pinned above) and no reverse sweep.
    x, box = _snapshot(seed=5, ncell=3, amp=0.1)
    v = inputs.maxwell(x.shape[0], 1.0, seed=6)
    dt = 0.005
    c = dt / 2
    f0, _, _, _ = oracle.forces(x, box, wca())
    x1 = np.mod(x + dt * (v + c * f0), box)
    f1, _, _, _ = oracle.forces(x1, box, wca())
    v1 = v + c * (f0 + f1)
    want = -dt * f1 + 2 * v1 + 2 * c * dt * oracle.force_jvp(x1, box, wca(), v1)
    _, _, _, gv, _, _ = oracle.adjoint(x, v, box, wca(), dt=dt, nsteps=1)
    assert np.abs(gv - want).max() <= 1e-12 * np.abs(want).max()
