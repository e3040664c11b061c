"""Unit cells and sizes beyond the 2x2 four-tensor workloads: the paper's own
A/B checkerboard of two tensors (Sec. II.B), rectangular 2x1 / 1x2 cells (the
frame rotations with Lx != Ly), D = 1 product states against their closed
forms, and the full D = 5, chi = 100 size against the oracle."""
import numpy as np
import pytest

import oracle as O
import synth
from gpu_common import gpu_ctm, oracle_options, rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _sweeps(ts, pat, D, chi, n, **kw):
    st = O.make_state(ts, pat, D, chi)
    opt = oracle_options(chi, D, **kw)
    for _ in range(n):
        st = O.sweep(st, opt)
    return st


def test_checkerboard_two_tensor_cell():
    w = synth.workload("product_noise", seed=8, D=2, chi=10)
    ts, pat = w["tensors"][:2], [[0, 1], [1, 0]]
    g = gpu_ctm(ts, pat, 10)
    g.sweep(3)
    st = _sweeps(ts, pat, 2, 10, 3)
    rd = O.bond_rdms(st, ts, pat)
    e_ref = O.energy_per_spin(rd, w["J"], 2, 2)
    assert abs(g.energy(w["J"]) - e_ref) < TOL * abs(e_ref)
    r = g.rdms()
    assert rel_err(r["h"], rd["h"]) < TOL and rel_err(r["v"], rd["v"]) < TOL
    g.close()


@pytest.mark.parametrize("pat", [[[0, 1]], [[0], [1]]])
def test_rectangular_cells(pat):
    w = synth.workload("product_noise", seed=9, D=2, chi=8)
    ts = w["tensors"][:2]
    g = gpu_ctm(ts, pat, 8)
    g.sweep(2)
    st = _sweeps(ts, pat, 2, 8, 2)
    rd = O.bond_rdms(st, ts, pat)
    r = g.rdms()
    assert rel_err(r["h"], rd["h"]) < TOL and rel_err(r["v"], rd["v"]) < TOL
    s_ref = O.corner_spectra(st)
    mask = s_ref > 1e-8
    assert np.max(np.abs(g.spectra() - s_ref)[mask]) < 1e-8
    g.close()


def test_product_states_D1_closed_forms():
    """D = 1: the environment is exact; every bond RDM is rho_i (x) rho_j with
    rho = phi phi^H / |phi|^2, and the all-up state has energy -Jz per spin."""
    d = 8
    A = np.zeros((d, 1, 1, 1, 1))
    A[0] = 1.0
    g = gpu_ctm([A] * 4, [[0, 1], [2, 3]], 1)
    g.sweep(1)
    assert abs(g.energy((1.0, 1.0, 0.37)) + 0.37) < 1e-13
    g.close()
    rng = np.random.default_rng(21)
    phis = [rng.standard_normal(d) + 1j * rng.standard_normal(d) for _ in range(4)]
    ts = [p.reshape(d, 1, 1, 1, 1) for p in phis]
    pat = [[0, 1], [2, 3]]
    g = gpu_ctm(ts, pat, 1)
    g.sweep(2)
    r = g.rdms()
    rho = [np.outer(p, p.conj()) / np.vdot(p, p).real for p in phis]
    for y in range(2):
        for x in range(2):
            a, b, c = pat[y][x], pat[y][(x + 1) % 2], pat[(y + 1) % 2][x]
            assert np.max(np.abs(r["h"][y, x] - np.kron(rho[a], rho[b]))) < 1e-13
            assert np.max(np.abs(r["v"][y, x] - np.kron(rho[a], rho[c]))) < 1e-13
    g.close()


def test_full_size_D5_chi100_one_sweep():
    """D = 5, chi = 100 (the bench's workload): one sweep from the trace
    initialisation, FP64 GPU path vs the oracle at 1e-10, and the BF16x3
    precision form within the 1e-6 energy target."""
    w = synth.workload("product_noise", seed=0, D=5, chi=100)
    st = _sweeps(w["tensors"], w["pattern"], 5, 100, 1)
    rd = O.bond_rdms(st, w["tensors"], w["pattern"])
    e_ref = O.energy_per_spin(rd, w["J"], 2, 2)
    g = gpu_ctm(w["tensors"], w["pattern"], 100)
    g.sweep(1)
    assert abs(g.energy(w["J"]) - e_ref) < TOL * abs(e_ref)
    r = g.rdms()
    assert rel_err(r["h"], rd["h"]) < TOL and rel_err(r["v"], rd["v"]) < TOL
    s_ref = O.corner_spectra(st)
    mask = s_ref > 1e-8
    assert np.max(np.abs(g.spectra() - s_ref)[mask]) < 1e-8
    g.close()
    gp = gpu_ctm(w["tensors"], w["pattern"], 100, prec="bf16x3", cutoff=0.0)
    gp.sweep(1)
    e_p = gp.energy(w["J"])
    print(f"full size, one sweep: E fp64 oracle {e_ref:.12f}, bf16x3 {e_p:.12f}, |dE| {abs(e_p - e_ref):.2e}")
    assert abs(e_p - e_ref) < 1e-6
    gp.close()
