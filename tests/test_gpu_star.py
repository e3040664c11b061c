"""Star lattice on the same engine (App. B): triangle block sites on the 2x2
cell with their empty edges as trivial bonds of dimension 1 (handed to the
library with their true leg sizes, ipeps_cell.leg_dims, and embedded there),
and the star-lattice Heisenberg operator table (ipeps_energy_star), against
the oracle on the same tensors zero-padded to D on the trivial legs."""
import numpy as np
import pytest

import oracle as O
import synth
from gpu_common import gpu_ctm, oracle_options, rel_err, spectra_err

pytestmark = pytest.mark.gpu

TOL = 1e-10
J = (1.0, 0.6)


def _padded(ts, D):
    out = []
    for t in ts:
        p = np.zeros((t.shape[0], D, D, D, D), dtype=t.dtype)
        p[:, :t.shape[1], :t.shape[2], :t.shape[3], :t.shape[4]] = t
        out.append(p)
    return out


def test_star_lattice_energy_matches_oracle():
    D, chi, sweeps = 2, 8, 3
    ts = synth.star_tensors(seed=5, D=D)
    pat = [[0, 1], [2, 3]]
    g = gpu_ctm(ts, pat, chi)  # trivial legs passed with their size 1
    g.sweep(sweeps)
    e = g.energy_star(J)
    full = _padded(ts, D)
    st = O.make_state(full, pat, D, chi)
    opt = oracle_options(chi, D)
    for _ in range(sweeps):
        st = O.sweep(st, opt)
    rd = O.bond_rdms(st, full, pat)
    e_ref = O.energy_per_spin(rd, J, 2, 2, model="star")
    print(f"star lattice D={D} chi={chi}: E gpu {e:.15f} oracle {e_ref:.15f}")
    assert abs(e - e_ref) < TOL * abs(e_ref)
    r = g.rdms()
    assert rel_err(r["h"], rd["h"]) < TOL and rel_err(r["v"], rd["v"]) < TOL
    assert spectra_err(g.spectra(), O.corner_spectra(st)) < TOL
    # the same tensors padded by the caller give the same network
    g2 = gpu_ctm(full, pat, chi)
    g2.sweep(sweeps)
    assert abs(g2.energy_star(J) - e) < 1e-13 * abs(e)
    g.close()
    g2.close()


def test_star_lattice_product_state_closed_form():
    """D = 1: the all-up product gives J_t + J_e / 2 per spin."""
    up = np.zeros((8, 1, 1, 1, 1))
    up[0] = 1.0
    g = gpu_ctm([up] * 4, [[0, 1], [2, 3]], 1)
    g.sweep(1)
    assert abs(g.energy_star(J) - (J[0] + J[1] / 2)) < 1e-13
    g.close()


def test_leg_sizes_other_than_one_or_D_are_refused():
    from paper_1711_04798_gb300 import CTMError
    ts = synth.star_tensors(seed=1, D=3)
    ts[0] = ts[0][:, :, :2]  # a leg of size 2 with D = 3
    with pytest.raises(CTMError) as e:
        gpu_ctm(ts, [[0, 1], [2, 3]], 9)
    assert e.value.status == 1 and "leg_dims" in str(e.value)
