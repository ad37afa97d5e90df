"""Degenerate and boundary cases of the GPU path, each against the oracle or an exact result."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2003_14061_gb300 import binding as B
from paper_2003_14061_gb300 import inputs
from paper_2003_14061_gb300.system import WCA_RC, MDSystem

pytestmark = pytest.mark.gpu


def min_image(d, box):
    return d - box * np.round(d / box)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
def test_single_atom_moves_ballistically(prec):
    box = np.array([5.0, 5.0, 5.0])                 # 3 cells of side >= r_c + skin per axis
    x = np.array([[4.9, 0.05, 2.5]])
    v = np.array([[1.3, -0.7, 0.2]])
    s = MDSystem(x, v, box, rc=WCA_RC, skin=0.4, precision=prec)
    s.integrate(100)
    x1, v1, f = s.state(f=True)
    want = np.mod(x + 100 * 0.005 * v, box)
    tol = 1e-12 if prec != "fp32" else 1e-5
    assert np.abs(min_image(x1 - want, box)).max() <= tol
    assert np.abs(v1 - v).max() <= (0 if prec != "fp32" else 1e-7) + 1e-15
    assert np.all(f == 0)
    p = s.props()[0]
    assert p["U"] == 0 and p["max_nbrs"] == 0


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
def test_two_atom_collision_matches_oracle(prec):
    box = np.array([6.0, 6.0, 6.0])
    x = np.array([[2.0, 3.0, 3.0], [3.05, 3.0, 3.0]])
    v = np.array([[1.0, 0.0, 0.0], [-1.0, 0.0, 0.0]])
    s = MDSystem(x, v, box, rc=WCA_RC, skin=0.3, precision=prec)
    s.integrate(200)
    xg, vg, _ = s.state()
    xo, vo, _, _ = oracle.run(x, v, box, oracle.pot(), dt=0.005, nsteps=200, with_props=False)
    tol = 1e-10 if prec == "fp64" else 1e-5
    assert np.abs(min_image(xg - xo, box)).max() <= tol
    assert np.abs(vg - vo).max() <= tol * 10
    assert abs(vg.sum(0)).max() <= 1e-5                 # momentum stays ~0


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_three_cells_per_axis(prec):
    rl = WCA_RC + 0.4
    L = 3.0 * rl * 1.0001                               # the smallest grid the method allows
    box = np.array([L, L, L])
    rng = np.random.default_rng(12)
    g = np.stack(np.meshgrid(*[np.arange(4)] * 3, indexing="ij"), -1).reshape(-1, 3)
    x = np.mod((g + 0.5 + rng.uniform(-0.25, 0.25, g.shape)) * (L / 4), L)
    v = inputs.maxwell(x.shape[0], 1.0, 3)
    s = MDSystem(x, v, box, rc=WCA_RC, skin=0.4, precision=prec)
    assert list(s.cells_per_axis()) == [3, 3, 3]
    counts, nb = s.neighbours()
    _, oc, off, onb = oracle.neighbours(x, box, WCA_RC, 0.4, fp32=(prec != "fp64"))
    assert np.array_equal(counts, oc)
    for i in range(x.shape[0]):
        assert np.array_equal(np.sort(nb[i, : counts[i]]), onb[off[i]:off[i + 1]])
    _, _, f = s.state(x=False, v=False, f=True)
    of, _, _, _ = oracle.forces(x, box, oracle.pot())
    assert np.linalg.norm(f - of) <= 1e-5 * np.linalg.norm(of)


def test_dense_fluid_near_overlap():
    # density 1.1 with perturbations: strong repulsion, many neighbours
    x, box = inputs.fcc_lattice(6, 1.1)
    x = inputs.perturb(x, box, 0.07, 4)
    v = inputs.maxwell(x.shape[0], 1.0, 5)
    s = MDSystem(x, v, box, rc=WCA_RC, skin=0.4)
    _, _, f = s.state(x=False, v=False, f=True)
    of, _, _, _ = oracle.forces(x, box, oracle.pot())
    assert np.linalg.norm(f - of) <= 1e-5 * np.linalg.norm(of)
    s.integrate(50)
    xg, vg, _ = s.state()
    xo, vo, _, _ = oracle.run(x, v, box, oracle.pot(), dt=0.005, nsteps=50, with_props=False)
    assert np.abs(min_image(xg - xo, box)).max() <= 1e-4


def test_batch_with_one_atom_replica_and_ragged_tails():
    reps = [(1, 0.2), (129, 0.7), (300, 0.8)]
    sts = []
    for k, (n, rho) in enumerate(reps):
        xb, bb = inputs.fcc_subset(n, rho, seed=k)
        if n < 10:
            bb = np.array([5.0, 5.0, 5.0])
        xb = inputs.perturb(xb, bb, 0.05, 10 + k)
        sts.append((xb, inputs.maxwell(n, 1.0, 20 + k) if n > 1 else np.array([[0.4, 0.1, -0.2]]), bb))
    x = np.concatenate([a for a, _, _ in sts])
    v = np.concatenate([b for _, b, _ in sts])
    s = MDSystem(x, v, n_rep=[n for n, _ in reps], boxes=np.stack([c for _, _, c in sts]), rc=WCA_RC, skin=0.4)
    s.integrate(40)
    xg, vg, _ = s.state()
    off = 0
    for xb, vb, bb in sts:
        n = xb.shape[0]
        xo, vo, _, _ = oracle.run(xb, vb, bb, oracle.pot(), dt=0.005, nsteps=40, with_props=False)
        assert np.abs(min_image(xg[off:off + n] - xo, bb)).max() <= 1e-4
        off += n


def test_positions_several_box_lengths_away():
    # md_create wraps any number of periods: cells, forces and the returned positions are those
    # of the in-box positions
    x, box = inputs.fcc_lattice(6, 0.8)
    x = inputs.perturb(x, box, 0.15, 31)
    k = np.random.default_rng(32).integers(-4, 5, x.shape)
    assert (np.abs(k) >= 2).any()
    v = inputs.maxwell(x.shape[0], 1.0, 33)
    s = MDSystem(x + k * box, v, box, rc=WCA_RC, skin=0.4)
    xg, _, f = s.state(f=True)
    assert np.abs(min_image(xg - x, box)).max() <= 1e-12
    _, cell = oracle.cells(x, box, WCA_RC + 0.4)
    assert np.array_equal(s.cells(), cell)
    of, _, _, _ = oracle.forces(x, box, oracle.pot())
    assert np.linalg.norm(f - of) <= 1e-5 * np.linalg.norm(of)


@pytest.mark.parametrize("what,bad", [("x", np.nan), ("v", np.nan), ("x", np.inf), ("v", -np.inf)])
def test_nonfinite_state_is_reported(what, bad):
    x, box = inputs.fcc_lattice(5, 0.8)
    x = inputs.perturb(x, box, 0.1, 34)
    v = inputs.maxwell(x.shape[0], 1.0, 35)
    xb, vb = x.copy(), v.copy()
    (xb if what == "x" else vb)[17, 1] = bad
    with pytest.raises(B.MDError) as e:
        MDSystem(xb, vb, box, rc=WCA_RC, skin=0.4)
    assert e.value.status == "MD_ERR_NONFINITE"
    s = MDSystem(x, v, box, rc=WCA_RC, skin=0.4)
    with pytest.raises(B.MDError) as e:
        s.set_state(xb, vb)
    assert e.value.status == "MD_ERR_NONFINITE"
    s.set_state(x, v)                                   # a good state makes the system usable again
    s.integrate(20)
    xg, _, _ = s.state()
    xo, _, _, _ = oracle.run(x, v, box, oracle.pot(), dt=0.005, nsteps=20, with_props=False)
    assert np.abs(min_image(xg - xo, box)).max() <= 1e-4


@pytest.mark.parametrize("status", ["MD_ERR_TIMEOUT", "MD_ERR_NONFINITE", "MD_ERR_NBR_OVERFLOW"])
def test_latched_device_errors_are_reported_once(status):
    # the device error word set from the host, as a kernel meeting the condition would: the next
    # call that waits returns the status and clears it (no kernel is made to fail)
    x, box = inputs.fcc_lattice(4, 0.8)
    v = inputs.maxwell(x.shape[0], 1.0, 36)
    s = MDSystem(x, v, box, rc=WCA_RC, skin=0.4)
    s.integrate(5)
    s.debug_set_error(status)
    with pytest.raises(B.MDError) as e:
        s.check()
    assert e.value.status == status
    s.check()                                           # reported once
    s.debug_set_error(status)
    with pytest.raises(B.MDError) as e:
        s.props()
    assert e.value.status == status
    s.integrate(5)
    assert s.props()[0]["step"] == 10
