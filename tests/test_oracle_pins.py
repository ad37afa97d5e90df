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
  * the paper's printed neighbour statistics and refresh intervals
    (tests/golden/paper_statistics.json);
  * hand-computed rebuild steps of both refresh rules for atoms at constant velocity;
  * the sampled checkers used at full size (forces on listed atoms, neighbour sets of listed
    atoms) against the whole-system evaluations pinned above;
  * the pressure with a non-zero virial and the trajectory loss, written out from pinned pieces;
  * finite differences for the Jacobian, the parameter derivatives and the adjoint;
  * the VACF / MSD: free flight in closed form, origin counts, caging at density 1.0;
  * the polymer chain terms: F = -grad U by finite differences per term, closed forms (FENE bond,
    straight / right / reversed bends, cis / 90 degree / trans dihedrals), zero net force and
    torque, the virial as sum r . F, chain boundaries by id, O(dt^2) energy error in a run.
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


@pytest.mark.parametrize("pot_name,r", [("wca", 1.0), ("lj", 1.5), ("lj", 1.05)])
def test_pressure_with_virial(pot_name, r):
    # one interacting pair at distance r across the periodic boundary: W = r . f(r) =
    # 24 (2 r^-12 - r^-6) (repulsive: W > 0; LJ at r = 1.5 attractive: W < 0), U = u(r), and the
    # pressure is (2K + W) / (3V) with K from the given velocities
    L = 7.0
    box = np.array([L, L, L])
    x = np.array([[0.5 * r, 3.0, 3.5], [L - 0.5 * r, 3.0, 3.5]])
    v = np.array([[0.3, -0.2, 0.7], [-0.1, 0.4, -0.5]])
    p = wca() if pot_name == "wca" else lj()
    W_want = 24.0 * (2.0 * r ** -12 - r ** -6)
    u_lj = 4.0 * (r ** -12 - r ** -6)
    U_want = u_lj + 1.0 if pot_name == "wca" else u_lj - 4.0 * (2.5 ** -12 - 2.5 ** -6)
    K = 0.5 * float((v ** 2).sum())
    U, Kp, W, P, px, py, pz, vmax = oracle.props(x, v, box, p)
    assert W == pytest.approx(W_want, rel=1e-13)
    assert U == pytest.approx(U_want, rel=1e-13, abs=1e-15)
    assert Kp == pytest.approx(K, rel=1e-15)
    assert P == pytest.approx((2.0 * K + W_want) / (3.0 * L ** 3), rel=1e-13)
    assert [px, py, pz] == pytest.approx([0.2, 0.2, 0.2], abs=1e-15)
    assert W != 0.0


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


@pytest.mark.parametrize("rule", [1, 2])
@pytest.mark.parametrize("start", [2.0, 19.5])
def test_refresh_rules_hand_count(rule, start):
    # Three atoms that never come within r_c of each other; only atom 0 moves, at constant
    # speed u along x (from x = 19.5 it crosses the periodic boundary at x = 20).  After n steps
    # it has moved n dt u, and both rules fire at the first step with n dt u > skin/2:
    # 0.3 / (0.005 * 1.7) = 35.29, so at steps 36, 72, 108, 144 and 180 -- five rebuilds in 200
    # steps, four in 179, one in 71, none in 35.
    L = 20.0
    box = np.array([L, L, L])
    x = np.array([[start, 5.0, 5.0], [10.0, 12.0, 10.0], [15.0, 2.0, 14.0]])
    v = np.array([[1.7, 0.0, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    for nsteps, want in ((35, 0), (36, 1), (71, 1), (179, 4), (200, 5)):
        x1, v1, _, rb = oracle.run(x, v, box, wca(), dt=0.005, nsteps=nsteps, rule=rule, skin=0.6,
                                   with_props=False)
        assert rb == want, (nsteps, rb)
        assert np.array_equal(v1, v)                                   # no force acted
        assert x1[0, 0] == pytest.approx((start + nsteps * 0.005 * 1.7) % L, abs=1e-12)
    # rule 0 counts nothing
    assert oracle.run(x, v, box, wca(), dt=0.005, nsteps=200, rule=0, skin=0.6, with_props=False)[3] == 0


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


@pytest.mark.parametrize("fp32", [True, False])
def test_neighbours_sample_matches_full_sets(fp32):
    # the sampled neighbour checker (used on the full-size workloads) returns, for each listed
    # atom, the full count and the same ascending set as the whole-system evaluation pinned
    # above; with a capacity below the count it keeps `cap` members of that set, ascending
    x, box = inputs.fcc_lattice(5, 0.8)
    x = inputs.perturb(x, box, 0.25, seed=21)
    rc, skin = RC_WCA, 0.4
    _, counts, off, nb = oracle.neighbours(x, box, rc, skin, fp32=fp32)
    n = x.shape[0]
    sample = np.unique(np.concatenate([[0, n - 1], np.random.default_rng(3).choice(n, 80, replace=False)]))
    cap = int(counts.max())
    sc, snb = oracle.neighbours_sample(x, box, rc, skin, sample, cap, fp32=fp32)
    assert np.array_equal(sc, counts[sample])
    for k, i in enumerate(sample):
        assert np.array_equal(snb[k, : sc[k]], nb[off[i]: off[i + 1]])
        assert np.all(snb[k, sc[k]:] == -1)
    capt = int(np.median(counts)) - 2
    assert (counts[sample] > capt).any()
    tc, tnb = oracle.neighbours_sample(x, box, rc, skin, sample, capt, fp32=fp32)
    assert np.array_equal(tc, counts[sample])                      # the full count is reported
    for k, i in enumerate(sample):
        row = tnb[k, : min(capt, tc[k])]
        assert np.all(np.diff(row) > 0)
        assert np.isin(row, nb[off[i]: off[i + 1]]).all()
        if tc[k] <= capt:
            assert np.array_equal(row, nb[off[i]: off[i + 1]])


@pytest.mark.parametrize("pot_name", ["wca", "lj"])
def test_force_on_atoms_matches_whole_system(pot_name):
    # the sampled force checker (used on the full-size workloads) equals the whole-system
    # evaluation, itself pinned to brute force above, on every listed atom
    rho = 0.8 if pot_name == "wca" else 0.8442
    x, box = inputs.fcc_lattice(5, rho)
    x = inputs.perturb(x, box, 0.12, seed=13)
    p = wca() if pot_name == "wca" else lj()
    f, ua, _, _ = oracle.forces(x, box, p)
    n = x.shape[0]
    sample = np.unique(np.concatenate([[0, n - 1], np.random.default_rng(4).choice(n, 60, replace=False)]))
    fs, us = oracle.force_on_atoms(x, box, p, sample)
    assert np.abs(f[sample]).max() > 1.0
    assert np.abs(fs - f[sample]).max() <= 1e-14 * np.abs(f).max()
    assert np.abs(us - ua[sample]).max() <= 1e-14 * (np.abs(ua).max() + 1.0)


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


_EQUILIBRATED = {}


def _paper_state(name):
    """The paper's SP or LJ state (Sec. 3.1), 1372 atoms equilibrated at its temperature."""
    if name not in _EQUILIBRATED:
        ref = json.load(open(os.path.join(GOLDEN, "paper_statistics.json")))[name]
        x, box = inputs.fcc_lattice(7, ref["rho"])
        v = inputs.maxwell(x.shape[0], ref["T"], seed=7)
        p = oracle.pot(rc=ref["rc"], shift=True)
        x, v = _equilibrate(x, v, box, p, ref["T"], 1500)
        _EQUILIBRATED[name] = (ref, x, v, box, p)
    return _EQUILIBRATED[name]


@pytest.mark.parametrize("name", ["SP", "LJ"])
def test_paper_mean_neighbour_counts(name):
    ref, x, v, box, p = _paper_state(name)
    nc, counts, off, nb = oracle.neighbours(x, box, ref["rc"], ref["skin"], fp32=False)
    assert counts.mean() == pytest.approx(ref["mean_neighbours"], rel=0.10)


@pytest.mark.parametrize("name,tiles,nsteps", [("SP", 6, 60), ("LJ", 5, 60)])
def test_paper_refresh_interval(name, tiles, nsteps):
    # Sec. 4.1 item 5: the largest systems refresh every 10.2 (SP) and 9.8 (LJ) steps at
    # delta = 0.6 under the maximum-velocity rule.  That interval is about (delta/2) / (dt vmax),
    # and vmax, the largest speed among N atoms, grows with N (the extreme of N Maxwell draws),
    # so a 1372-atom state refreshes every ~14 steps.  The state here has the size the interval
    # needs: the equilibrated 1372-atom configuration repeated tiles^3 times (a periodic
    # configuration of the larger box; 296k and 171k atoms) with fresh Maxwell velocities at the
    # state's temperature -- in equilibrium positions and momenta are independent, so this is an
    # equilibrium state of the larger system.  vmax is still below that of the paper's 16.8M
    # (SP) and 7.1M (LJ) atoms, which biases the interval up by a few per cent.  The rule counts
    # whole steps, so the count c over nsteps admits any interval in (nsteps/(c+1), nsteps/c];
    # that range must meet the paper's figure +-15%.
    ref, x, _, box, p = _paper_state(name)
    sh = np.stack(np.meshgrid(*[np.arange(tiles)] * 3, indexing="ij"), -1).reshape(-1, 3)
    X = np.ascontiguousarray((x[None, :, :] + sh[:, None, :] * box[None, None, :]).reshape(-1, 3))
    B = box * tiles
    V = inputs.maxwell(X.shape[0], ref["T"], seed=8)
    _, _, _, c = oracle.run(X, V, B, p, dt=0.005, nsteps=nsteps, rule=1, skin=ref["skin"], with_props=False)
    lo, hi = nsteps / (c + 1), nsteps / max(c, 1e-9)
    want = ref["refresh_steps"]
    assert c > 0 and lo < 1.15 * want and hi >= 0.85 * want, (c, lo, hi, want)


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


def test_loss_closed_form():
    # L = (1/S) sum_{n=1..S} U(x_n) + |v_S|^2, written out for S = 1 and 2 from the pinned force
    # evaluation and the leapfrog steps: x_{n+1} = x_n + dt (v_n + c F_n), v_{n+1} = v_n + c (F_n
    # + F_{n+1}), c = dt / 2m
    x, box = _snapshot(seed=7, ncell=3, amp=0.12)
    v = inputs.maxwell(x.shape[0], 1.0, seed=8)
    dt = 0.005
    c = dt / 2
    f0, _, _, _ = oracle.forces(x, box, wca())
    x1 = np.mod(x + dt * (v + c * f0), box)
    f1, _, U1, _ = oracle.forces(x1, box, wca())
    v1 = v + c * (f0 + f1)
    x2 = np.mod(x1 + dt * (v1 + c * f1), box)
    f2, _, U2, _ = oracle.forces(x2, box, wca())
    v2 = v1 + c * (f1 + f2)
    assert U1 > 1.0 and U2 > 1.0
    assert oracle.loss(x, v, box, wca(), dt=dt, nsteps=1) == pytest.approx(U1 + (v1 ** 2).sum(), rel=1e-13)
    assert oracle.loss(x, v, box, wca(), dt=dt, nsteps=2) == pytest.approx(0.5 * (U1 + U2) + (v2 ** 2).sum(),
                                                                          rel=1e-13)


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


# ---------------------------------------------------------------------------------------------
# velocity autocorrelation and mean-square displacement (Sec. 4.1 items 1 and 7)
# ---------------------------------------------------------------------------------------------
def test_dynamics_free_flight_closed_form():
    # atoms on a grid of spacing 3 moving at most 0.3 in the run stay farther apart than r_c: no
    # force acts, so v_i(t) = v_i(0) and r_i(t) - r_i(0) = v_i t: VACF(k) = <v^2> and MSD(k) =
    # <v^2> (k T)^2, T = every dt, for every lag, however the atoms wrap through the box
    g = np.stack(np.meshgrid(*[np.arange(6)] * 3, indexing="ij"), -1).reshape(-1, 3)
    box = np.array([18.0, 18.0, 18.0])
    x = (g + 0.5) * 3.0
    v = np.random.default_rng(8).uniform(-0.5, 0.5, x.shape)
    x[0] = [17.95, 1.5, 1.5]                        # crosses x = L at once
    v[0] = [0.5, 0.0, 0.0]
    every, nlag, origin_every, nsamples = 4, 12, 3, 30
    vacf, msd, cnt = oracle.dynamics(x, v, box, wca(), dt=0.005, nsamples=nsamples, every=every, nlag=nlag,
                                     origin_every=origin_every)
    v2 = float((v ** 2).sum(1).mean())
    T = every * 0.005
    assert np.allclose(vacf, v2, rtol=1e-13)
    assert np.allclose(msd, v2 * (np.arange(nlag) * T) ** 2, rtol=1e-11, atol=1e-16)
    # origins at samples 0, 3, ..., 27; lag k is reached by the origins with start + k < nsamples
    starts = np.arange(0, nsamples, origin_every)
    assert np.array_equal(cnt, [(starts + k < nsamples).sum() for k in range(nlag)])


def test_dynamics_caged_vacf_goes_negative():
    # Sec. 4.1 item 7: in the SP fluid at rho = 1.0 the VACF oscillates -- each atom bounces off
    # the cage of its neighbours -- so it turns negative within a fraction of a time unit; at
    # lag 0 it is <v^2> = 3T at the state's temperature
    x, box = inputs.fcc_lattice(5, 1.0)
    v = inputs.maxwell(x.shape[0], 1.0, seed=9)
    x, v = _equilibrate(x, v, box, wca(), 1.0, 400)
    vacf, msd, cnt = oracle.dynamics(x, v, box, wca(), dt=0.005, nsamples=121, every=1, nlag=100, origin_every=5)
    t_vmin = int(np.argmin(vacf))
    assert vacf[0] == pytest.approx(3.0, rel=0.15)
    assert vacf[t_vmin] < -0.05 * vacf[0] and 0.05 < t_vmin * 0.005 < 0.4
    assert np.all(np.diff(msd[:20]) > 0)             # displacements grow at first ...
    assert msd[1] == pytest.approx(vacf[0] * 0.005 ** 2, rel=0.05)   # ... ballistically


# ---------------------------------------------------------------------------------------------
# polymer chains (Sec. 4.3 item 2): FENE bonds, bending and dihedral terms
# ---------------------------------------------------------------------------------------------
def _bent_chain(m=7, seed=3):
    # a random walk of bond length ~1 with bond angles away from 0 and 180 degrees, mid-box
    rng = np.random.default_rng(seed)
    x = [np.array([10.0, 10.0, 10.0])]
    d = np.array([1.0, 0.0, 0.0])
    for _ in range(m - 1):
        while True:
            e = rng.normal(size=3)
            e /= np.linalg.norm(e)
            if 0.2 < np.dot(e, d) < 0.85:
                break
        d = e
        x.append(x[-1] + (0.95 + 0.1 * rng.random()) * d)
    return np.array(x), np.array([20.0, 20.0, 20.0])


@pytest.mark.parametrize("terms", [dict(ka=0.0, kd=0.0), dict(ka=5.0, kd=0.0), dict(ka=0.0, kd=2.0),
                                   dict(ka=5.0, kd=2.0)])
def test_chain_forces_are_minus_the_energy_gradient(terms):
    x, box = _bent_chain()
    ch = oracle.chains(x.shape[0], **terms)
    f, U, W = oracle.chain_forces(x, box, ch)
    h = 1e-6
    fd = np.zeros_like(x)
    for i in range(x.shape[0]):
        for a in range(3):
            xp = x.copy(); xp[i, a] += h
            xm = x.copy(); xm[i, a] -= h
            fd[i, a] = -(oracle.chain_forces(xp, box, ch)[1] - oracle.chain_forces(xm, box, ch)[1]) / (2 * h)
    assert np.abs(f - fd).max() <= 1e-6 * np.abs(f).max()
    # an isolated chain: no net force, no net torque, and the virial is sum_a r_a . F_a
    assert np.abs(f.sum(0)).max() <= 1e-10 * np.abs(f).max()
    assert np.abs(np.cross(x, f).sum(0)).max() <= 1e-9 * np.abs(f).max() * 20
    assert W == pytest.approx(float((x * f).sum()), rel=1e-10, abs=1e-10)


def test_chain_closed_forms():
    box = np.array([20.0, 20.0, 20.0])
    # one FENE bond of length 1 across the boundary: U = -(1/2) 30 1.5^2 ln(1 - 1/2.25),
    # tension 30 / (1 - 1/2.25) = 54 pulling the atoms together, W = -54
    x = np.array([[0.4, 5.0, 5.0], [19.4, 5.0, 5.0]])
    f, U, W = oracle.chain_forces(x, box, oracle.chains(2))
    assert U == pytest.approx(-0.5 * 30 * 2.25 * math.log(1 - 1 / 2.25), rel=1e-14)
    assert f[0] == pytest.approx([-54.0, 0, 0], rel=1e-13) and f[1] == pytest.approx([54.0, 0, 0], rel=1e-13)
    assert W == pytest.approx(-54.0, rel=1e-13)
    # bending: straight U = 0 and no force; a right angle U = ka; antiparallel bonds U = 2 ka
    ch = oracle.chains(3, kb=0.0, ka=4.0)
    for pts, u in (([[5, 5, 5], [6, 5, 5], [7, 5, 5]], 0.0), ([[5, 5, 5], [6, 5, 5], [6, 6, 5]], 4.0)):
        f, U, _ = oracle.chain_forces(np.array(pts, float), box, ch)
        assert U == pytest.approx(u, abs=1e-14)
    f, _, _ = oracle.chain_forces(np.array([[5, 5, 5], [6, 5, 5], [7, 5, 5]], float), box, ch)
    assert np.abs(f).max() == 0.0
    # dihedral: cis (p = 0) U = 0, p = 90 degrees U = kd, trans (p = 180) U = 2 kd
    ch = oracle.chains(4, kb=0.0, kd=3.0)
    for last, u in (([5, 6, 5], 0.0), ([6, 5, 6], 3.0), ([7, 4, 5], 6.0)):
        pts = np.array([[5, 6, 5], [5, 5, 5], [6, 5, 5], last], float)
        _, U, _ = oracle.chain_forces(pts, box, ch)
        assert U == pytest.approx(u, abs=1e-13)


def test_chains_split_by_length_and_run_conserves_energy():
    # chains are consecutive ids: 3 chains of 5 have 12 bonds, not 14
    x, box = _bent_chain(m=15, seed=8)
    ch = oracle.chains(5)
    _, U, _ = oracle.chain_forces(x, box, ch)
    U_sep = sum(oracle.chain_forces(x[k:k + 5], box, ch)[1] for k in (0, 5, 10))
    assert U == pytest.approx(U_sep, rel=1e-14)
    # chains of 4 (the 4 basis sites of each fcc cell, bonds of 1.26) packed at density 0.7 with
    # bending and dihedral terms: momentum conserved, energy error bounded and O(dt^2)
    xs, bx = inputs.fcc_lattice(4, 0.7)
    xs = inputs.perturb(xs, bx, 0.02, seed=3)
    n = xs.shape[0]
    v = inputs.maxwell(n, 1.0, seed=4)
    ch = oracle.chains(4, ka=2.0, kd=0.5)
    _, Ub, _ = oracle.chain_forces(xs, bx, ch)
    assert np.isfinite(Ub)
    errs = []
    for dt, ns in ((0.002, 500), (0.001, 1000)):
        _, _, pr = oracle.run_chains(xs, v, bx, wca(), ch, dt=dt, nsteps=ns)
        E = pr[:, 0] + pr[:, 1]
        assert np.abs(pr[:, 4:7]).max() < 1e-9
        errs.append(np.abs(E - E[0]).max() / abs(E[0]))
    # (the stiff FENE bonds, k = 30, make the error larger than the fluid's at the same dt)
    assert errs[0] < 5e-3 and 3.0 < errs[0] / errs[1] < 5.0
