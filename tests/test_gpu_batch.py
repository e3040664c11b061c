"""Batched scan (independent instances advanced by one CUDA graph launch per
move, autotuned tensor-core tiles) against the FP64 oracle and against the
same instances run one by one through the single-instance API."""
import numpy as np
import pytest

import oracle as O
import synth
from gpu_common import DEFAULTS, oracle_options, spectra_err

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _instances(n=4, seed=5):
    # uneven D and chi, as in the scan recipe, at sizes the oracle runs in seconds
    return synth.scan(seed=seed, n=n, Ds=(2, 3), chis=(9, 12, 16))


def _oracle_energy(inst, sweeps):
    st = O.make_state(inst["tensors"], inst["pattern"], inst["D"], inst["chi"])
    opt = oracle_options(inst["chi"], inst["D"])
    for _ in range(sweeps):
        st = O.sweep(st, opt)
    rd = O.bond_rdms(st, inst["tensors"], inst["pattern"])
    return O.energy_per_spin(rd, inst["J"], 2, 2), O.corner_spectra(st)


def test_batch_fp64_matches_oracle():
    from paper_1711_04798_gb300 import Batch
    insts = _instances()
    b = Batch(insts, tune=False, prec="fp64", **DEFAULTS)
    b.sweep(1)
    b.sweep(1)  # second call replays the captured graph
    e = b.energies([i["J"] for i in insts])
    for i, inst in enumerate(insts):
        e_ref, s_ref = _oracle_energy(inst, 2)
        assert abs(e[i] - e_ref) < TOL * abs(e_ref), (i, e[i], e_ref)
        assert spectra_err(b.instance(i).spectra(), s_ref) < TOL, i
    assert b.launch_count() > 0
    b.close()


def test_batch_single_direction_graphs():
    from paper_1711_04798_gb300 import Batch
    insts = _instances(n=3, seed=2)
    b = Batch(insts, tune=False, prec="fp64", **DEFAULTS)
    for d in ("L", "U", "R", "D"):
        b.move(d, 1)
    e = b.energies([i["J"] for i in insts])
    for i, inst in enumerate(insts):
        st = O.make_state(inst["tensors"], inst["pattern"], inst["D"], inst["chi"])
        opt = oracle_options(inst["chi"], inst["D"])
        for d in ("L", "U", "R", "D"):
            st = O.move(st, d, opt)
        e_ref = O.energy_per_spin(O.bond_rdms(st, inst["tensors"], inst["pattern"]), inst["J"], 2, 2)
        assert abs(e[i] - e_ref) < TOL * abs(e_ref), i
    b.close()


def test_batch_precision_matches_single_handles_and_oracle():
    from paper_1711_04798_gb300 import Batch, CTM
    insts = _instances(n=4, seed=7)
    kw = dict(DEFAULTS, cutoff=1e-6)  # above the BF16x3 noise floor (oracle uses the same)
    b = Batch(insts, tune=False, prec="bf16x3", **kw)
    b.sweep(2)
    e_b = b.energies([i["J"] for i in insts])
    for i, inst in enumerate(insts):
        g = CTM(inst["tensors"], inst["pattern"], inst["chi"], prec="bf16x3", **kw)
        g.sweep(2)
        e_s = g.energy(inst["J"])
        g.close()
        # same kernels, same tile choices, same order within the instance
        assert abs(e_b[i] - e_s) < 1e-12 * max(abs(e_s), 1.0), (i, e_b[i], e_s)
        st = O.make_state(inst["tensors"], inst["pattern"], inst["D"], inst["chi"])
        opt = oracle_options(inst["chi"], inst["D"], cutoff=1e-6)
        for _ in range(2):
            st = O.sweep(st, opt)
        e_ref = O.energy_per_spin(O.bond_rdms(st, inst["tensors"], inst["pattern"]), inst["J"], 2, 2)
        print(f"instance {i}: batch {e_b[i]:.12f} single {e_s:.12f} oracle {e_ref:.12f}")
        assert abs(e_b[i] - e_ref) < 1e-5, (i, e_b[i], e_ref)
    b.close()


def test_batch_autotuner_choices_and_results():
    """Tuned tiles change only rounding: a tuned and an untuned batch agree
    with the oracle to the precision form's energy target (1e-6, BF16x6), with
    a truncation cutoff (1e-6) above the contraction noise on both sides."""
    from paper_1711_04798_gb300 import Batch
    insts = _instances(n=3, seed=11)
    kw = dict(DEFAULTS, cutoff=1e-6)
    b = Batch(insts, tune=True, prec="bf16x6", **kw)
    table = b.tuning()
    assert len(table) > 0
    for t in table:
        assert t["bn"] in (128, 256) and t["splits"] >= 1
        assert t["us"] <= t["default_us"] * 1.0000001
    b.sweep(2)
    e = b.energies([i["J"] for i in insts])
    b.close()
    p = Batch(insts, tune=False, prec="bf16x6", **kw)
    p.sweep(2)
    e_plain = p.energies([i["J"] for i in insts])
    p.close()
    for i, inst in enumerate(insts):
        st = O.make_state(inst["tensors"], inst["pattern"], inst["D"], inst["chi"])
        opt = oracle_options(inst["chi"], inst["D"], cutoff=1e-6)
        for _ in range(2):
            st = O.sweep(st, opt)
        e_ref = O.energy_per_spin(O.bond_rdms(st, inst["tensors"], inst["pattern"]), inst["J"], 2, 2)
        print(f"instance {i}: |dE| tuned {abs(e[i] - e_ref):.2e}, default {abs(e_plain[i] - e_ref):.2e}")
        assert abs(e[i] - e_ref) < 1e-6 and abs(e_plain[i] - e_ref) < 1e-6, (i, e[i], e_plain[i], e_ref)


def test_batch_create_error_names_instance():
    from paper_1711_04798_gb300 import Batch, CTMError
    insts = _instances(n=3, seed=1)
    insts[1] = dict(insts[1], chi=2)  # chi < D^2
    with pytest.raises(CTMError) as ei:
        Batch(insts, tune=False, prec="fp64", **DEFAULTS)
    assert "instance 1" in str(ei.value) and ei.value.status == 1


def test_single_handle_autotune_keeps_environment():
    """ipeps_ctm_autotune restores the environment; tuned tiles change results only by rounding."""
    from paper_1711_04798_gb300 import CTM
    w = synth.workload("product_noise", seed=4, D=3, chi=16)
    kw = dict(DEFAULTS, cutoff=1e-6, prec="bf16x3")
    a = CTM(w["tensors"], w["pattern"], 16, **kw)
    b = CTM(w["tensors"], w["pattern"], 16, **kw)
    a.sweep(1)
    b.sweep(1)
    env_before = b.env(4, 0, 0)
    n = b.autotune()
    assert n > 0
    assert np.array_equal(b.env(4, 0, 0), env_before)
    a.sweep(2)
    b.sweep(2)
    assert abs(a.energy(w["J"]) - b.energy(w["J"])) < 1e-6
    assert a.autotune() > 0 and CTM(w["tensors"], w["pattern"], 16, **dict(kw, prec="fp64")).autotune() == 0
    a.close()
    b.close()
