"""GPU adjoint (md_adjoint and MDTrajectoryFn) against the FP64 oracle adjoint.

The oracle adjoint is itself pinned by finite differences and a closed-form single step
(tests/test_oracle_pins.py).  The GPU forward runs FP32 pair forces, so its trajectory and its
gradients differ from the FP64 ones at the level that rounding, amplified by the chaotic
dynamics, allows: 1e-4 relative on short horizons.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2003_14061_gb300 import inputs
from paper_2003_14061_gb300.autograd import MDTrajectoryFn
from paper_2003_14061_gb300.system import WCA_RC, MDSystem

pytestmark = pytest.mark.gpu


def rel(a, b):
    return abs(a - b) / abs(b)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def small_case(seed=1):
    x, box = inputs.fcc_lattice(5, 0.8)                   # 500 atoms: 3 full tiles + a ragged tail
    x = inputs.perturb(x, box, 0.1, seed)
    v = inputs.maxwell(x.shape[0], 1.0, seed + 1)
    return x, v, box


@pytest.mark.parametrize("nsteps,ckpt", [(1, 1), (30, 10), (30, 7)])
def test_adjoint_matches_oracle_short(nsteps, ckpt):
    x, v, box = small_case()
    s = MDSystem(x, v, box, rc=WCA_RC, skin=0.4, precision="mixed")
    loss, ge, gs, gv = s.adjoint(nsteps, ckpt)
    ol, oge, ogs, ogv, _, _ = oracle.adjoint(x, v, box, oracle.pot(), dt=0.005, nsteps=nsteps)
    assert rel(loss, ol) <= 1e-6
    assert rel(ge, oge) <= 1e-4
    assert rel(gs, ogs) <= 1e-4
    assert rel_l2(gv, ogv) <= 1e-4
    # the system is left at its initial state
    x1, v1, _ = s.state()
    d = x1 - x
    d -= box * np.round(d / box)
    assert np.abs(d).max() < 1e-12 and np.abs(v1 - v).max() < 1e-12


def test_checkpoint_interval_does_not_change_gradients():
    x, v, box = small_case(3)
    s = MDSystem(x, v, box, rc=WCA_RC, skin=0.4)
    res = [s.adjoint(40, k) for k in (40, 20, 8, 5)]
    for r in res[1:]:
        assert rel(r[0], res[0][0]) <= 1e-7
        assert rel(r[1], res[0][1]) <= 1e-5 and rel(r[2], res[0][2]) <= 1e-5
        assert rel_l2(r[3], res[0][3]) <= 1e-5


def test_adjoint_graphs_follow_tuning_and_horizon():
    # segments replay cached graphs; a new launch shape or horizon captures new ones, and the
    # results do not depend on which graphs ran
    x, v, box = small_case(11)
    s = MDSystem(x, v, box, rc=WCA_RC, skin=0.4)
    a = s.adjoint(30, 7)
    s.set_tuning(ctas_per_sm=4, nbr_batch=8, build_batch=32)
    b = s.adjoint(30, 7)
    c = s.adjoint(30, 10)
    s.set_tuning(ctas_per_sm=12, nbr_batch=2, build_batch=2)
    d = s.adjoint(30, 7)
    assert a[0] == b[0] == d[0] and a[1] == b[1] == d[1] and a[2] == b[2] == d[2]
    assert np.array_equal(a[3], b[3]) and np.array_equal(a[3], d[3])
    assert rel(c[0], a[0]) <= 1e-7 and rel(c[1], a[1]) <= 1e-5 and rel(c[2], a[2]) <= 1e-5


def test_adjoint_is_deterministic():
    x, v, box = small_case(5)
    s = MDSystem(x, v, box, rc=WCA_RC, skin=0.4)
    a = s.adjoint(20, 10)
    b = s.adjoint(20, 10)
    assert a[0] == b[0] and a[1] == b[1] and a[2] == b[2] and np.array_equal(a[3], b[3])


def test_autograd_function():
    x, v, box = small_case(7)
    eps = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    sig = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    v0 = torch.from_numpy(v).clone().requires_grad_(True)
    loss = MDTrajectoryFn.apply(eps, sig, v0, x, box, 20, 5, {})
    (2.5 * loss).backward()
    s = MDSystem(x, v, box, rc=WCA_RC, skin=0.4)
    l2, ge, gs, gv = s.adjoint(20, 5)
    assert float(loss.detach()) == pytest.approx(l2, rel=1e-12)
    assert float(eps.grad) == pytest.approx(2.5 * ge, rel=1e-12)
    assert float(sig.grad) == pytest.approx(2.5 * gs, rel=1e-12)
    assert np.allclose(v0.grad.numpy(), 2.5 * gv, rtol=1e-12, atol=0)


def test_gpu_loss_finite_difference_in_eps():
    # sanity of the GPU forward loss: FP32 forces limit the usable step to h ~ 1e-3
    x, v, box = small_case(9)
    h = 1e-3

    def L(e):
        s = MDSystem(x, v, box, eps=e, rc=WCA_RC, skin=0.4)
        return s.adjoint(20, 10)[0]

    s = MDSystem(x, v, box, rc=WCA_RC, skin=0.4)
    ge = s.adjoint(20, 10)[1]
    fd = (L(1 + h) - L(1 - h)) / (2 * h)
    assert rel(ge, fd) <= 2e-2


@pytest.fixture(scope="module")
def workload():
    # the adjoint workload: 32,000 atoms at density 0.8 on a random fcc subset, T = 1
    x, box = inputs.fcc_subset(32000, 0.8, seed=5)
    v = inputs.maxwell(32000, 1.0, seed=6)
    oracle.set_threads(0)
    return x, v, box


def test_adjoint_workload_size_100_steps(workload):
    x, v, box = workload
    s = MDSystem(x, v, box, rc=WCA_RC, skin=0.4)
    loss, ge, gs, gv = s.adjoint(100, 20)
    ol, oge, ogs, ogv, _, _ = oracle.adjoint(x, v, box, oracle.pot(), dt=0.005, nsteps=100)
    assert rel(loss, ol) <= 1e-6
    assert rel(ge, oge) <= 1e-3 and rel(gs, ogs) <= 1e-3
    assert rel_l2(gv, ogv) <= 1e-3


def test_adjoint_workload_size_400_steps(workload):
    # Over 400 steps (t = 2) the gradient is ill-conditioned: displacing the initial positions by
    # 1e-7 moves the FP64 oracle's own gradients by ~2e-2 (eps, sigma) and ~5e-3 (v0).  The FP32
    # forward perturbs the trajectory at that level every step, so the bar is the oracle's own
    # sensitivity, measured here, with a factor 2 of room.
    x, v, box = workload
    s = MDSystem(x, v, box, rc=WCA_RC, skin=0.4)
    loss, ge, gs, gv = s.adjoint(400, 20)
    o = oracle.adjoint(x, v, box, oracle.pot(), dt=0.005, nsteps=400)
    xp = np.mod(x + np.random.default_rng(0).uniform(-1e-7, 1e-7, x.shape), box)
    op = oracle.adjoint(xp, v, box, oracle.pot(), dt=0.005, nsteps=400)
    assert rel(loss, o[0]) <= 1e-5
    assert abs(ge - o[1]) <= 2.0 * abs(op[1] - o[1]) + 1e-6 * abs(o[1])
    assert abs(gs - o[2]) <= 2.0 * abs(op[2] - o[2]) + 1e-6 * abs(o[2])
    assert np.linalg.norm(gv - o[3]) <= 2.0 * np.linalg.norm(op[3] - o[3]) + 1e-6 * np.linalg.norm(o[3])
