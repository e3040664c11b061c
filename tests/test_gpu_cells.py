"""Unit cells and sizes beyond the 2x2 four-tensor workloads: the paper's own
A/B checkerboard of two tensors (Sec. II.B), rectangular 2x1 / 1x2 cells (the
frame rotations with Lx != Ly), D = 1 product states against their closed
forms, and the full D = 5, chi = 100 size against the oracle."""
import numpy as np
import pytest

import oracle as O
import synth
from gpu_common import golden, gpu_ctm, oracle_options, rel_err, spectra_err

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
    assert spectra_err(g.spectra(), O.corner_spectra(st)) < TOL
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
    initialisation, FP64 GPU path against the stored exact-SVD oracle record
    (tests/golden/make_golden.py) at 1e-10."""
    w = synth.workload("product_noise", seed=0, D=5, chi=100)
    ref = golden("product_noise_D5_chi100_cut8")
    g = gpu_ctm(w["tensors"], w["pattern"], 100)
    g.sweep(1)
    e = g.energy(w["J"])
    e_ref = float(ref["E_sweep1"])
    print(f"full size, one sweep: E gpu {e:.15f} oracle {e_ref:.15f}")
    assert abs(e - e_ref) < TOL * abs(e_ref)
    r = g.rdms()
    assert rel_err(r["h"], ref["rho_h_sweep1"]) < TOL and rel_err(r["v"], ref["rho_v_sweep1"]) < TOL
    assert rel_err(g.site_rdms(), ref["rho_site_sweep1"]) < TOL
    assert spectra_err(g.spectra(), ref["spectra_sweep1"]) < TOL
    g.close()


def test_full_size_D4_chi64_converged_energy_and_fidelity():
    """D = 4, chi = 64, psi1 = product state + noise (seed 0), psi2 the same
    recipe with seed 1: each environment converged to 1e-10 in the corner
    spectra, energy at (Jx, Jy, Jz) = (1, 1, 0.5), RDMs, spectra, and the
    fidelity per site from the converged mixed network (Sec. III), all at
    1e-10 against the stored exact-SVD oracle record."""
    from paper_1711_04798_gb300 import CTM
    ref = golden("product_noise_D4_chi64_converged")
    w1 = synth.workload("product_noise", seed=0, D=4, chi=64)
    w2 = synth.workload("product_noise", seed=1, D=4, chi=64)
    t1, t2, pat = w1["tensors"], w2["tensors"], w1["pattern"]
    hs = {"11": gpu_ctm(t1, pat, 64), "22": gpu_ctm(t2, pat, 64), "12": gpu_ctm(t1, pat, 64, bra=t2)}
    for tag, g in hs.items():
        k_ref = complex(ref["kappa_" + tag])
        if tag == "12":
            # the mixed network's ring is not Hermitian; with the range finder
            # (k = chi + 16, q = 2) its corner spectra settle at a floor of
            # about 1e-4 in the convergence measure (the oracle's own range-finder
            # route does the same), while kappa is steady: it takes the exact-SVD
            # oracle's sweep count and is compared there
            n = int(ref["sweeps_12"])
            g.sweep(n)
            k = g.kappa()
            print(f"psi12: gpu {n} sweeps, kappa {k:.15f} vs oracle {k_ref:.15f} "
                  f"(rel {abs(k - k_ref) / abs(k_ref):.1e})")
            assert abs(k - k_ref) < TOL * abs(k_ref), (tag, k, k_ref)
            continue
        n, delta, ok = g.converge(1e-10, 120)
        print(f"psi{tag}: gpu {n} sweeps (delta {delta:.2e}), oracle {int(ref['sweeps_' + tag])} "
              f"({float(ref['delta_' + tag]):.2e})")
        assert ok and abs(n - int(ref["sweeps_" + tag])) <= 1
        k = g.kappa()
        assert abs(k - k_ref) < TOL * abs(k_ref), (tag, k, k_ref)
        assert spectra_err(g.spectra(), ref["spectra_" + tag]) < TOL
    for tag in ("11", "22"):
        g = hs[tag]
        e, e_ref = g.energy(w1["J"]), float(ref["E_" + tag])
        print(f"psi{tag}: E gpu {e:.15f} oracle {e_ref:.15f}")
        assert abs(e - e_ref) < TOL * abs(e_ref)
        r = g.rdms()
        assert rel_err(r["h"], ref["rho_h_" + tag]) < TOL and rel_err(r["v"], ref["rho_v_" + tag]) < TOL
        assert rel_err(g.site_rdms(), ref["rho_site_" + tag]) < TOL
    d_block, d_spin = CTM.fidelity(hs["12"], hs["11"], hs["22"])
    print(f"fidelity per block site {d_block:.15f} (oracle {float(ref['d_block']):.15f})")
    assert abs(d_block - float(ref["d_block"])) < TOL and abs(d_spin - float(ref["d_spin"])) < TOL
    for g in hs.values():
        g.close()
