"""Failure paths on the GPU that fault nothing: each ends in a status code
the host reads, and the library stays usable afterwards.

* a NaN in the input tensors: the normalisation of the initial environment
  meets a non-finite norm -> ENUMERIC at create;
* a Jacobi budget of one sweep: the projector SVD stops unconverged and
  reports it -> ETIMEOUT from the move (no wait is unbounded);
* a handle too large for the device: the allocation fails -> ENOMEM, and the
  failure leaves no error behind for the next handle."""
import numpy as np
import pytest

import oracle as O
import synth
from gpu_common import gpu_ctm, oracle_options

pytestmark = pytest.mark.gpu


def _healthy_sweep_matches_oracle():
    w = synth.workload("real", seed=4, chi=8)
    g = gpu_ctm(w["tensors"], w["pattern"], 8)
    g.sweep(1)
    st = O.sweep(O.make_state(w["tensors"], w["pattern"], 2, 8), oracle_options(8, 2))
    e_ref = O.energy_per_spin(O.bond_rdms(st, w["tensors"], w["pattern"]), w["J"], 2, 2)
    assert abs(g.energy(w["J"]) - e_ref) < 1e-10 * abs(e_ref)


def test_nan_input_reports_enumeric():
    from paper_1711_04798_gb300 import CTMError
    w = synth.workload("product_noise", seed=3, D=2, chi=8)
    ts = [t.copy() for t in w["tensors"]]
    ts[1][0, 1, 0, 1, 0] = np.nan
    with pytest.raises(CTMError) as e:
        gpu_ctm(ts, w["pattern"], 8)
    assert e.value.status == 6, str(e.value)
    _healthy_sweep_matches_oracle()


def test_jacobi_budget_reports_etimeout():
    from paper_1711_04798_gb300 import CTMError
    w = synth.workload("product_noise", seed=3, D=2, chi=8)
    g = gpu_ctm(w["tensors"], w["pattern"], 8, jacobi_max_sweeps=1)
    with pytest.raises(CTMError) as e:
        g.move("L", 1)
    assert e.value.status == 5 and "Jacobi" in str(e.value), str(e.value)
    g.reset_env()  # the handle is still usable
    g.close()
    _healthy_sweep_matches_oracle()


def test_failed_allocation_reports_enomem_and_leaves_no_error():
    from paper_1711_04798_gb300 import CTMError
    rng = np.random.default_rng(1)
    A = rng.standard_normal((2, 12, 12, 12, 12))
    with pytest.raises(CTMError) as e:
        gpu_ctm([A], [[0]], 1008)  # D = 12, chi = 1008: terabytes of enlarged corners
    assert e.value.status == 2 and "cudaMalloc" in str(e.value), str(e.value)
    _healthy_sweep_matches_oracle()


def test_grid_barrier_wait_limit_reports_etimeout():
    """The small-row Jacobi (rows of at most 256 complex numbers, fewer than 32
    rows: the projector of D = 2, chi = 8 with k = 24 rows of length 32) runs
    as one cooperative launch whose CTAs meet at a grid barrier between
    rounds.  With a wait limit of one clock cycle the waiting CTAs give up at
    the first barrier, count it and return: ETIMEOUT from the move, and the
    library stays usable."""
    from paper_1711_04798_gb300 import CTMError
    w = synth.workload("product_noise", seed=3, D=2, chi=8)
    g = gpu_ctm(w["tensors"], w["pattern"], 8, wait_cycles=1)
    with pytest.raises(CTMError) as e:
        g.move("L", 1)
    assert e.value.status == 5 and "grid-barrier" in str(e.value), str(e.value)
    g.reset_env()
    g.close()
    _healthy_sweep_matches_oracle()
