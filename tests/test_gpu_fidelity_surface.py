"""Fidelity surface (Sec. VI: the fidelity per site of the states at pairs of
points J1, J2 of a coupling line, from mixed-network CTMs, Sec. III) on the
batch engine: every plain and mixed network of a small line advanced together
by the batch's graph launches, then ipeps_batch_fidelity, against the
oracle's kappa and fidelity of the same networks after the same sweeps."""
import itertools

import numpy as np
import pytest

import oracle as O
import synth
from gpu_common import DEFAULTS, oracle_options

pytestmark = pytest.mark.gpu

TOL = 1e-10


def test_fidelity_surface_matches_oracle():
    from paper_1711_04798_gb300 import Batch
    n, D, chi, sweeps = 3, 2, 8, 4
    line = synth.fidelity_line(seed=3, n=n, D=D)
    pat = [[0, 1], [2, 3]]
    insts = [{"tensors": ts, "pattern": pat, "chi": chi} for ts in line]  # plain networks 0..n-1
    pairs, mixed = [], {}
    for a, b in itertools.combinations_with_replacement(range(n), 2):
        mixed[(a, b)] = len(insts)
        insts.append({"tensors": line[a], "bra": line[b], "pattern": pat, "chi": chi})
        pairs.append((mixed[(a, b)], a, b))
    bt = Batch(insts, tune=False, prec="fp64", **DEFAULTS)
    bt.sweep(sweeps)
    d_block, d_spin = bt.fidelity(pairs)
    bt.close()
    kap = {}
    for i, inst in enumerate(insts):
        st = O.make_state(inst["tensors"], pat, D, chi, mixed_with=inst.get("bra"))
        opt = oracle_options(chi, D)
        for _ in range(sweeps):
            st = O.sweep(st, opt)
        kap[i] = O.kappa(st)
    surface = np.zeros((n, n))
    for p, (i12, i11, i22) in enumerate(pairs):
        db_ref, ds_ref = O.fidelity(kap[i12], kap[i11], kap[i22])
        assert abs(d_block[p] - db_ref) < TOL and abs(d_spin[p] - ds_ref) < TOL, (p, d_block[p], db_ref)
        a, b = i11, i22
        surface[a, b] = surface[b, a] = d_block[p]
    print("fidelity surface (per block site):\n", np.array2string(surface, precision=12))
    # d(psi, psi) = 1: the mixed network of a state with itself is its plain network
    assert np.allclose(np.diag(surface), 1.0, atol=1e-12)
    # off the diagonal the overlap per site is below one and falls with the distance on the line
    assert surface[0, 1] < 1.0 and surface[0, 2] < surface[0, 1]


def test_fidelity_surface_argument_errors():
    from paper_1711_04798_gb300 import Batch, CTMError
    line = synth.fidelity_line(seed=1, n=2, D=2)
    pat = [[0, 1], [2, 3]]
    bt = Batch([{"tensors": ts, "pattern": pat, "chi": 8} for ts in line], tune=False, prec="fp64", **DEFAULTS)
    with pytest.raises(CTMError) as e:
        bt.fidelity([(0, 1, 2)])
    assert e.value.status == 1 and "instance 2" in str(e.value)
    bt.close()
