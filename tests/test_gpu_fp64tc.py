"""The FP64-accurate tensor-core form (IPEPS_PREC_FP64TC): every contraction
product large enough for the tensor cores is computed by exact base-256 digit
splitting of both operands on tcgen05 (one rounding to FP64, the last); every
other step is the FP64 path's.  It is held to the FP64 path's tolerances
against the exact-SVD oracle: 1e-10 relative on energies, RDM elements and
fidelities, 1e-10 on the corner spectra s_i/s_0 (wherever s_i/s_0 >= 1e-8),
at small sizes, at the full D = 5, chi = 100 size and on the converged
D = 4, chi = 64 pair with its fidelity."""
import numpy as np
import pytest

import oracle as O
import synth
from gpu_common import golden, gpu_ctm, oracle_options, rel_err, spectra_err

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _oracle(w, chi, sweeps, **kw):
    st = O.make_state(w["tensors"], w["pattern"], w["D"], chi)
    opt = oracle_options(chi, w["D"], **kw)
    for _ in range(sweeps):
        st = O.sweep(st, opt)
    return st


@pytest.mark.parametrize("kind,seed,D,chi,sweeps", [("real", 0, 2, 16, 20), ("product_noise", 2, 3, 18, 3)])
def test_matches_oracle(kind, seed, D, chi, sweeps):
    w = synth.workload(kind, seed=seed, D=D, chi=chi)
    g = gpu_ctm(w["tensors"], w["pattern"], chi, prec="fp64tc")
    g.sweep(sweeps)
    st = _oracle(w, chi, sweeps)
    rd = O.bond_rdms(st, w["tensors"], w["pattern"])
    e_ref = O.energy_per_spin(rd, w["J"], 2, 2)
    e = g.energy(w["J"])
    r = g.rdms()
    s_err = spectra_err(g.spectra(), O.corner_spectra(st))
    print(f"{kind} D={D} chi={chi}: |dE|/|E| {abs(e - e_ref) / abs(e_ref):.1e}, "
          f"rho {max(rel_err(r['h'], rd['h']), rel_err(r['v'], rd['v'])):.1e}, spectra {s_err:.1e}")
    assert abs(e - e_ref) < TOL * abs(e_ref)
    assert rel_err(r["h"], rd["h"]) < TOL and rel_err(r["v"], rd["v"]) < TOL
    assert rel_err(g.site_rdms(), O.site_rdms(st, w["tensors"], w["pattern"])) < TOL
    assert s_err < TOL
    g.close()


def test_full_size_D5_chi100_one_sweep():
    """The bench's workload: one sweep from the trace initialisation against
    the stored exact-SVD oracle record (tests/golden/make_golden.py)."""
    w = synth.workload("product_noise", seed=0, D=5, chi=100)
    ref = golden("product_noise_D5_chi100_cut8")
    g = gpu_ctm(w["tensors"], w["pattern"], 100, prec="fp64tc")
    g.sweep(1)
    e, e_ref = g.energy(w["J"]), float(ref["E_sweep1"])
    r = g.rdms()
    s_err = spectra_err(g.spectra(), ref["spectra_sweep1"])
    print(f"full size, one sweep: E gpu {e:.15f} oracle {e_ref:.15f}; spectra {s_err:.1e}")
    assert abs(e - e_ref) < TOL * abs(e_ref)
    assert rel_err(r["h"], ref["rho_h_sweep1"]) < TOL and rel_err(r["v"], ref["rho_v_sweep1"]) < TOL
    assert rel_err(g.site_rdms(), ref["rho_site_sweep1"]) < TOL
    assert s_err < TOL
    g.close()


def test_D4_chi64_converged_energy_and_fidelity():
    """psi1 (seed 0) and psi2 (seed 1), D = 4, chi = 64: environments
    converged to 1e-10 in the corner spectra, energy at (1, 1, 0.5), RDMs,
    spectra, and the fidelity per site from the mixed network (Sec. III),
    against the stored converged exact-SVD oracle record.  The mixed network
    takes the oracle's sweep count (its range-finder spectra settle at a
    floor, kappa does not move)."""
    from paper_1711_04798_gb300 import CTM
    ref = golden("product_noise_D4_chi64_converged")
    w1 = synth.workload("product_noise", seed=0, D=4, chi=64)
    w2 = synth.workload("product_noise", seed=1, D=4, chi=64)
    t1, t2, pat = w1["tensors"], w2["tensors"], w1["pattern"]
    hs = {"11": gpu_ctm(t1, pat, 64, prec="fp64tc"), "22": gpu_ctm(t2, pat, 64, prec="fp64tc"),
          "12": gpu_ctm(t1, pat, 64, bra=t2, prec="fp64tc")}
    for tag, g in hs.items():
        k_ref = complex(ref["kappa_" + tag])
        if tag == "12":
            g.sweep(int(ref["sweeps_12"]))
        else:
            n, delta, ok = g.converge(1e-10, 120)
            print(f"psi{tag}: {n} sweeps (delta {delta:.2e}), oracle {int(ref['sweeps_' + tag])}")
            assert ok and abs(n - int(ref["sweeps_" + tag])) <= 1
            assert spectra_err(g.spectra(), ref["spectra_" + tag]) < TOL
        k = g.kappa()
        assert abs(k - k_ref) < TOL * abs(k_ref), (tag, k, k_ref)
    for tag in ("11", "22"):
        g = hs[tag]
        e, e_ref = g.energy(w1["J"]), float(ref["E_" + tag])
        print(f"psi{tag}: E gpu {e:.15f} oracle {e_ref:.15f}")
        assert abs(e - e_ref) < TOL * abs(e_ref)
        r = g.rdms()
        assert rel_err(r["h"], ref["rho_h_" + tag]) < TOL and rel_err(r["v"], ref["rho_v_" + tag]) < TOL
    d_block, d_spin = CTM.fidelity(hs["12"], hs["11"], hs["22"])
    print(f"fidelity per block site {d_block:.15f} (oracle {float(ref['d_block']):.15f})")
    assert abs(d_block - float(ref["d_block"])) < TOL and abs(d_spin - float(ref["d_spin"])) < TOL
    for g in hs.values():
        g.close()


@pytest.mark.parametrize("Nv", [2, 4])
def test_boundary_spectrum(Nv):
    """Dense boundary density operator (Sec. IV) against the oracle's, 1e-10."""
    w = synth.workload("product_noise", seed=6, D=2, chi=8)
    g = gpu_ctm(w["tensors"], w["pattern"], 8, prec="fp64tc")
    g.sweep(3)
    st = _oracle(w, 8, 3)
    lam, S = g.boundary_rho(0, Nv)
    lam_ref = O.boundary_spectrum(st, 0, Nv)
    assert np.max(np.abs(lam - lam_ref)) < TOL
    assert abs(S - O.entropy(lam_ref)) < TOL
    g.close()


def test_precision_form_polished_to_the_oracle_fixed_point():
    """A BF16x6 convergence (its spectra settle at a floor set by FP32
    accumulation) continued by FP64-accurate sweeps from its environment
    (ipeps_ctm_env_copy, device to device): converged to 1e-10, the result is
    the FP64 oracle's converged one at the same cutoff (1e-6), 1e-10."""
    w, chi, cut = synth.workload("product_noise", seed=2, D=3, chi=18), 18, 1e-6
    gm = gpu_ctm(w["tensors"], w["pattern"], chi, prec="bf16x6", cutoff=cut)
    n1, d1, _ = gm.converge(1e-8, 30)
    gp = gpu_ctm(w["tensors"], w["pattern"], chi, prec="fp64tc", cutoff=cut)
    gp.copy_env_from(gm)
    assert np.max(np.abs(gp.env(4, 1, 0) - gm.env(4, 1, 0))) == 0.0
    n2, d2, ok = gp.converge(1e-10, 40)
    st = O.make_state(w["tensors"], w["pattern"], w["D"], chi)
    st, n_ref, d_ref = O.ctm_converge(st, oracle_options(chi, w["D"], cutoff=cut), 1e-10, 100)
    rd = O.bond_rdms(st, w["tensors"], w["pattern"])
    e_ref = O.energy_per_spin(rd, w["J"], 2, 2)
    e = gp.energy(w["J"])
    r = gp.rdms()
    s_err = spectra_err(gp.spectra(), O.corner_spectra(st))
    print(f"bf16x6 {n1} sweeps (delta {d1:.1e}), then fp64tc {n2} sweeps (delta {d2:.1e}); oracle {n_ref}: "
          f"|dE|/|E| {abs(e - e_ref) / abs(e_ref):.1e}, spectra {s_err:.1e}")
    assert ok
    assert abs(e - e_ref) < TOL * abs(e_ref)
    assert rel_err(r["h"], rd["h"]) < TOL and rel_err(r["v"], rd["v"]) < TOL
    assert s_err < TOL
    gm.close()
    gp.close()


def test_two_corner_route():
    """The two-corner projectors (corners = 2, X = Q1^T Q4) in the FP64-accurate
    form against the exact-SVD oracle of that route, FP64 tolerances."""
    w = synth.workload("product_noise", seed=0, D=2, chi=16)
    g = gpu_ctm(w["tensors"], w["pattern"], 16, prec="fp64tc", corners=2)
    g.sweep(6)
    st = _oracle(w, 16, 6, corners=2)
    rd = O.bond_rdms(st, w["tensors"], w["pattern"])
    e_ref = O.energy_per_spin(rd, w["J"], 2, 2)
    e = g.energy(w["J"])
    r = g.rdms()
    s_err = spectra_err(g.spectra(), O.corner_spectra(st))
    print(f"two corners: |dE|/|E| {abs(e - e_ref) / abs(e_ref):.1e}, spectra {s_err:.1e}")
    assert abs(e - e_ref) < TOL * abs(e_ref)
    assert rel_err(r["h"], rd["h"]) < TOL and rel_err(r["v"], rd["v"]) < TOL
    assert s_err < TOL
    g.close()


def test_batch_of_uneven_instances():
    """The batched scan (one graph launch per move over instances of uneven D
    and chi) in the FP64-accurate form: every instance's energy and corner
    spectra against its own oracle run, FP64 tolerances."""
    from paper_1711_04798_gb300 import Batch
    from gpu_common import DEFAULTS
    insts = synth.scan(seed=5, n=4, Ds=(2, 3), chis=(9, 12, 16))
    b = Batch(insts, tune=False, prec="fp64tc", **DEFAULTS)
    b.sweep(1)
    b.sweep(1)  # the second call replays the captured graph
    e = b.energies([i["J"] for i in insts])
    for i, inst in enumerate(insts):
        st = _oracle(inst, inst["chi"], 2)
        e_ref = O.energy_per_spin(O.bond_rdms(st, inst["tensors"], inst["pattern"]), inst["J"], 2, 2)
        assert abs(e[i] - e_ref) < TOL * abs(e_ref), (i, e[i], e_ref)
        assert spectra_err(b.instance(i).spectra(), O.corner_spectra(st)) < TOL, i
    b.close()
