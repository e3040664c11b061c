"""User-supplied environments, checkpoint and resume (ipeps_ctm_env_set,
ipeps_ctm_save, ipeps_ctm_load) on the GPU.

An environment taken from the oracle after a few of its own sweeps, set into
a GPU handle, must give the oracle's invariants after one more move: parity of
a single move from an identical state, independent of the moves before it."""
import numpy as np
import pytest

import oracle as O
import synth
from gpu_common import DEFAULTS, gpu_ctm, oracle_options, rel_err, spectra_err

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _set_state(g, st):
    for role in range(8):
        for y in range(st.Ly):
            for x in range(st.Lx):
                g.set_env(role, x, y, st.C[role][y][x] if role < 4 else st.T[role - 4][y][x])


def _all_env(g):
    return [g.env(role, x, y) for role in range(8) for y in range(2) for x in range(2)]


@pytest.mark.parametrize("direction", ["L", "U", "sweep"])
def test_oracle_environment_then_one_move_matches(direction):
    w = synth.workload("product_noise", seed=12, D=2, chi=10)
    opt = oracle_options(10, 2)
    st = O.make_state(w["tensors"], w["pattern"], 2, 10)
    for _ in range(2):
        st = O.sweep(st, opt)
    g = gpu_ctm(w["tensors"], w["pattern"], 10)
    _set_state(g, st)
    for role in (0, 5):  # round trip of the layout
        ref = st.C[role][1][0] if role < 4 else st.T[role - 4][1][0]
        assert np.array_equal(g.env(role, 0, 1), ref)
    g.move(direction, 1)
    st = O.sweep(st, opt) if direction == "sweep" else O.move(st, direction, opt)
    r_gpu, r_ref = g.rdms(), O.bond_rdms(st, w["tensors"], w["pattern"])
    for key in ("h", "v"):
        assert rel_err(r_gpu[key], r_ref[key]) < TOL, key
    assert spectra_err(g.spectra(), O.corner_spectra(st)) < TOL
    e_gpu = g.energy(w["J"])
    e_ref = O.energy_per_spin(r_ref, w["J"], 2, 2)
    assert abs(e_gpu - e_ref) < TOL * abs(e_ref)


def test_save_then_load_resumes(tmp_path):
    from paper_1711_04798_gb300 import env_file_info
    w = synth.workload("product_noise", seed=13, D=3, chi=12)
    g1 = gpu_ctm(w["tensors"], w["pattern"], 12)
    g1.sweep(3)
    path = tmp_path / "env.ipeps"
    g1.save(path)
    assert not (tmp_path / "env.ipeps.part").exists()
    info = env_file_info(path)
    assert (info["Lx"], info["Ly"], info["d"], info["D"], info["chi"]) == (2, 2, 8, 3, 12)
    saved = _all_env(g1)
    g1.sweep(2)
    g2 = gpu_ctm(w["tensors"], w["pattern"], 12)
    g2.load(path)
    for a, b in zip(_all_env(g2), saved):
        assert np.array_equal(a, b)
    g2.sweep(2)
    assert rel_err(g2.spectra(), g1.spectra()) < 1e-12
    e1, e2 = g1.energy(w["J"]), g2.energy(w["J"])
    assert abs(e1 - e2) < 1e-12 * abs(e1)


def test_refused_load_leaves_environment(tmp_path):
    from paper_1711_04798_gb300 import CTMError
    w = synth.workload("product_noise", seed=14, D=2, chi=8)
    g = gpu_ctm(w["tensors"], w["pattern"], 8)
    g.sweep(1)
    path = tmp_path / "chi8.ipeps"
    g.save(path)
    other = gpu_ctm(w["tensors"], w["pattern"], 9)
    before = _all_env(other)
    with pytest.raises(CTMError) as e:
        other.load(path)  # chi 8 into a chi 9 handle
    assert e.value.status == 1 and "chi 8" in str(e.value)
    raw = bytearray(path.read_bytes())
    raw[-20] ^= 0x01
    damaged = tmp_path / "damaged.ipeps"
    damaged.write_bytes(bytes(raw))
    with pytest.raises(CTMError) as e:
        g.load(damaged)
    assert e.value.status == 8
    for a, b in zip(_all_env(other), before):
        assert np.array_equal(a, b)
    with pytest.raises(CTMError) as e:
        g.save(tmp_path / "no_such_dir" / "x.ipeps")
    assert e.value.status == 8


def test_environment_set_into_a_batch_instance():
    """The captured graphs of a batch keep their buffers: an environment set
    between replays is what the next replay starts from."""
    from paper_1711_04798_gb300 import Batch
    insts = synth.scan(seed=3, n=2, Ds=(2,), chis=(9,))
    b = Batch(insts, tune=False, prec="fp64", **DEFAULTS)
    b.sweep(1)  # captures and replays the sweep graph
    inst = insts[0]
    opt = oracle_options(9, 2)
    st = O.make_state(inst["tensors"], inst["pattern"], 2, 9)
    for _ in range(3):
        st = O.sweep(st, opt)
    _set_state(b.instance(0), st)
    b.sweep(1)
    st = O.sweep(st, opt)
    e = b.energies([i["J"] for i in insts])
    e_ref = O.energy_per_spin(O.bond_rdms(st, inst["tensors"], inst["pattern"]), inst["J"], 2, 2)
    assert abs(e[0] - e_ref) < TOL * abs(e_ref)
    b.close()
