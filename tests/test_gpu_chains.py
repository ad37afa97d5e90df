"""GPU parity of the polymer chain terms (md_set_chains, Sec. 4.3 item 2) against the FP64 oracle.

Inputs: the 4 basis sites of every fcc cell as chains of 4 (bent bonds of 1.26, density 0.7) with
bending and dihedral terms, and chains of 25 along a serpentine path through a simple cubic
lattice at density 0.85 (bonds of 1.06, straight runs and right-angle turns) with bending.  The
bars are those of the pair forces: step-0 forces within 1e-5 relative L2, 100-step positions
within 1e-4 and velocities within 1e-4 relative L2, energy per atom within 1e-6 (1e-5 with the
stiff bonds' larger energies).
"""
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


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def fcc_chains():
    x, box = inputs.fcc_lattice(5, 0.7)
    return inputs.perturb(x, box, 0.02, seed=3), box, dict(length=4, bend_k=2.0, dihedral_k=0.5)


def serpentine_chains():
    x, box = inputs.cubic_lattice(10, 0.85, serpentine=True)
    return inputs.perturb(x, box, 0.02, seed=4), box, dict(length=25, bend_k=3.0, dihedral_k=0.0)


CASES = {"fcc4": fcc_chains, "serpentine25": serpentine_chains}


def _oracle_chains(c):
    return oracle.chains(c["length"], ka=c["bend_k"], kd=c["dihedral_k"])


@pytest.mark.parametrize("kernel", [1, 4, 5])
@pytest.mark.parametrize("prec", ["mixed", "fp32"])
@pytest.mark.parametrize("name", list(CASES))
def test_chain_forces_and_trajectory(name, prec, kernel):
    x, box, c = CASES[name]()
    n = x.shape[0]
    v = inputs.maxwell(n, 1.0, seed=5)
    s = MDSystem(x, v, box, rc=WCA_RC, skin=0.4, precision=prec)
    s.set_chains(**c)
    if kernel != 1:
        s.set_tuning(step_kernel=kernel)
    _, _, f = s.state(x=False, v=False, f=True)
    p = oracle.pot()
    ch = _oracle_chains(c)
    fp, _, Up, Wp = oracle.forces(x, box, p)
    fc, Uc, Wc = oracle.chain_forces(x, box, ch)
    assert rel_l2(f, fp + fc) <= 1e-5
    pr = s.props()[0]
    assert abs(pr["U"] - (Up + Uc)) / n <= 1e-5
    assert abs(pr["virial"] - (Wp + Wc)) / n <= 1e-4
    s.integrate(100)
    xg, vg, _ = s.state()
    pr = s.props()[0]
    xo, vo, po = oracle.run_chains(x, v, box, p, ch, dt=0.005, nsteps=100)
    assert np.abs(min_image(xg - xo, box)).max() <= 1e-4
    assert rel_l2(vg, vo) <= 1e-4
    assert abs(pr["E_per_atom"] - (po[-1, 0] + po[-1, 1]) / n) <= 1e-5
    s.close()


def test_chains_in_batched_replicas():
    # replicas of different sizes, each split into chains by its own local ids
    states = []
    for k, ncell in enumerate((3, 4, 5)):
        x, box = inputs.fcc_lattice(ncell, 0.7)
        states.append((inputs.perturb(x, box, 0.02, 10 + k), inputs.maxwell(x.shape[0], 1.0, 20 + k), box))
    n_rep = [st[0].shape[0] for st in states]
    s = MDSystem(np.concatenate([st[0] for st in states]), np.concatenate([st[1] for st in states]), n_rep=n_rep,
                 boxes=np.stack([st[2] for st in states]), rc=WCA_RC, skin=0.4, precision="mixed")
    c = dict(length=4, bend_k=2.0, dihedral_k=0.5)
    s.set_chains(**c)
    s.integrate(60)
    xg, vg, _ = s.state()
    props = s.props()
    off = 0
    for r, (xr, vr, br) in enumerate(states):
        m = xr.shape[0]
        xo, vo, po = oracle.run_chains(xr, vr, br, oracle.pot(), _oracle_chains(c), dt=0.005, nsteps=60)
        assert np.abs(min_image(xg[off:off + m] - xo, br)).max() <= 1e-4
        assert rel_l2(vg[off:off + m], vo) <= 1e-4
        assert abs(props[r]["E_per_atom"] - (po[-1, 0] + po[-1, 1]) / m) <= 1e-5
        off += m


def test_chain_arguments():
    x, box, c = fcc_chains()
    v = inputs.maxwell(x.shape[0], 1.0, seed=5)
    s = MDSystem(x, v, box, rc=WCA_RC, skin=0.4, precision="fp64")
    with pytest.raises(B.MDError):
        s.set_chains(**c)                               # FP32 chain arithmetic: MIXED / FP32 only
    s = MDSystem(x, v, box, rc=WCA_RC, skin=0.4, precision="mixed")
    s.set_chains(**c)
    with pytest.raises(B.MDError):
        s.adjoint(10, 5)                                # the adjoint covers the pair forces only
    s.set_chains(0)                                     # chains removed: the pair forces alone
    _, _, f = s.state(x=False, v=False, f=True)
    fp, _, _, _ = oracle.forces(x, box, oracle.pot())
    # (this lattice has no pair within r_c: both are zero)
    assert np.abs(f - fp).max() <= 1e-5 * max(1.0, np.abs(fp).max())
