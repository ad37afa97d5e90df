"""GPU parity of the VACF / MSD measurement (md_dyn_*) against the FP64 oracle.

Atoms are followed by their permanent ids through reorders (a reorder every 30 steps inside
the measured stretch), so a mix-up of ids would break the per-atom products.  Tolerances follow
from the trajectory bars (positions within 1e-4, velocities within 1e-4 relative): the VACF
within 2e-4 of its lag-0 value, the MSD within 2e-4 sqrt(MSD) + 1e-8; FP64 to rounding.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2003_14061_gb300 import inputs
from paper_2003_14061_gb300.system import WCA_RC, MDSystem

pytestmark = pytest.mark.gpu

EVERY, NLAG, ORIGIN_EVERY, NSAMPLES = 5, 8, 3, 20            # 95 steps, 7 origins


def _run_gpu(s):
    s.dyn_begin(NLAG, ORIGIN_EVERY)
    for k in range(NSAMPLES):
        if k:
            s.integrate(EVERY)
        s.dyn_sample()
    return s.dyn_result()


def _check(vg, mg, vo, mo, prec):
    if prec == "fp64":
        assert np.abs(vg - vo).max() <= 1e-10 * vo[0]
        assert np.abs(mg - mo).max() <= 1e-10 * mo.max()
    else:
        assert np.abs(vg - vo).max() <= 2e-4 * vo[0]
        assert np.all(np.abs(mg - mo) <= 2e-4 * np.sqrt(mo) + 1e-8)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
def test_vacf_msd_match_oracle(prec):
    x, box = inputs.fcc_lattice(8, 0.8)
    x = inputs.perturb(x, box, 0.15, 1)
    v = inputs.maxwell(x.shape[0], 1.0, seed=5)
    s = MDSystem(x, v, box, rc=WCA_RC, skin=0.4, precision=prec, reorder_every=30)
    vg, mg, cg = _run_gpu(s)
    assert s.props()[0]["reorders"] >= 3
    s.close()
    vo, mo, co = oracle.dynamics(x, v, box, oracle.pot(), dt=0.005, nsamples=NSAMPLES, every=EVERY, nlag=NLAG,
                                 origin_every=ORIGIN_EVERY)
    assert np.array_equal(cg, co)
    assert mo[1] > 0 and vo[0] > 1.0
    _check(vg, mg, vo, mo, prec)


def test_vacf_msd_batched_replicas():
    # sums run over the atoms of all replicas, each unwrapped in its own box: the result is the
    # atom-weighted mean of the replicas' own measurements
    specs = inputs.replica_specs(4, 300, 1500, 0.6, 0.9, seed=21)
    states = [(inputs.perturb(xr, br, 0.08, 70 + r), vr, br)
              for r, (xr, vr, br) in enumerate(inputs.replica_states(specs, 1.0, seed=21))]
    n_rep = [sp[0] for sp in specs]
    x = np.concatenate([st[0] for st in states])
    v = np.concatenate([st[1] for st in states])
    s = MDSystem(x, v, n_rep=n_rep, boxes=np.stack([st[2] for st in states]), rc=WCA_RC, skin=0.4,
                 precision="mixed", reorder_every=30)
    vg, mg, cg = _run_gpu(s)
    s.close()
    vo = np.zeros(NLAG)
    mo = np.zeros(NLAG)
    for (xr, vr, br), n in zip(states, n_rep):
        a, b, c = oracle.dynamics(xr, vr, br, oracle.pot(), dt=0.005, nsamples=NSAMPLES, every=EVERY, nlag=NLAG,
                                  origin_every=ORIGIN_EVERY)
        vo += n * a
        mo += n * b
        co = c
    vo /= sum(n_rep)
    mo /= sum(n_rep)
    assert np.array_equal(cg, co)
    _check(vg, mg, vo, mo, "mixed")


def test_dynamics_arguments_are_checked():
    from paper_2003_14061_gb300 import binding as B
    x, box = inputs.fcc_lattice(4, 0.8)
    s = MDSystem(x, inputs.maxwell(x.shape[0], 1.0, 2), box, rc=WCA_RC, skin=0.4)
    with pytest.raises(B.MDError):
        s.dyn_sample()                                  # no measurement begun
    with pytest.raises(B.MDError):
        s.dyn_begin(100, 10)                            # 10 origins at once: above the limit of 8
    s.dyn_begin(80, 10)
    s.dyn_sample()
    vacf, msd, cnt = s.dyn_result()
    assert cnt[0] == 1 and cnt[1] == 0 and msd[0] == 0.0
    assert vacf[0] == pytest.approx(float((inputs.maxwell(x.shape[0], 1.0, 2) ** 2).sum(1).mean()), rel=1e-12)
