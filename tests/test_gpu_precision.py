"""The precision form (tensor-core contractions, FP64 projectors and
normalisation) against the FP64 oracle: the energy error is reported and
bounded per precision."""
import numpy as np
import pytest

import oracle as O
import synth
from gpu_common import gpu_ctm, oracle_options

pytestmark = pytest.mark.gpu

# measured: BF16x3 ~1e-6 after six sweeps (not yet the converged-energy target
# of 1e-6 at every point; see the precision notes), TF32 ~1e-4
BOUND = {"bf16x3": 3e-6, "tf32": 1e-3}


@pytest.mark.parametrize("prec", ["bf16x3", "tf32"])
def test_precision_form_energy_error(prec):
    w = synth.workload("product_noise", seed=2, D=3, chi=18)
    g = gpu_ctm(w["tensors"], w["pattern"], 18, prec=prec)
    g.sweep(6)
    st = O.make_state(w["tensors"], w["pattern"], w["D"], 18)
    opt = oracle_options(18, w["D"])
    for _ in range(6):
        st = O.sweep(st, opt)
    e_ref = O.energy_per_spin(O.bond_rdms(st, w["tensors"], w["pattern"]), w["J"], 2, 2)
    e = g.energy(w["J"])
    print(f"{prec}: E = {e:.12f}, oracle {e_ref:.12f}, |dE| = {abs(e - e_ref):.3e}")
    assert abs(e - e_ref) < BOUND[prec]
    # one-site RDMs: entries of size <= 1, errors of the energy's order
    err = np.max(np.abs(g.site_rdms() - O.site_rdms(st, w["tensors"], w["pattern"])))
    print(f"{prec}: site RDM max |d rho| = {err:.3e}")
    assert err < 10 * BOUND[prec]
