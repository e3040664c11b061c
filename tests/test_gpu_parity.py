"""GPU (CUDA library, through the C ABI) against the FP64 oracle on the same
seeded inputs.  The oracle truncates with the exact SVD of the ring across
each cut (Sec. II.C); the GPU with its randomized range finder.  FP64 path
tolerance: 1e-10 relative on energies and RDM elements, and 1e-10 on the
corner spectra s_i/s_0 (relative to the largest value s_0) wherever
s_i/s_0 >= 1e-8."""
import numpy as np
import pytest

import oracle as O
import synth
from gpu_common import gpu_ctm, oracle_options, rel_err, spectra_err

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _oracle_run(w, chi, moves, **kw):
    st = O.make_state(w["tensors"], w["pattern"], w["D"], chi)
    opt = oracle_options(chi, w["D"], **kw)
    for m in moves:
        st = O.sweep(st, opt) if m == "sweep" else O.move(st, m, opt)
    return st


def _compare_rdms(g, st, w, tol=TOL):
    r_gpu = g.rdms()
    r_ref = O.bond_rdms(st, w["tensors"], w["pattern"])
    for key in ("h", "v"):
        assert rel_err(r_gpu[key], r_ref[key]) < tol, key


def _compare_site_rdms(g, st, w, tol=TOL):
    r_ref = O.site_rdms(st, w["tensors"], w["pattern"])
    assert rel_err(g.site_rdms(), r_ref) < tol


def _compare_spectra(g, st, floor=1e-8, tol=TOL):
    assert spectra_err(g.spectra(), O.corner_spectra(st), floor) < tol


def test_trace_init_environment_matches():
    w = synth.workload("real", seed=3)
    g = gpu_ctm(w["tensors"], w["pattern"], 8)
    st = O.make_state(w["tensors"], w["pattern"], w["D"], 8)
    for role in range(8):
        for y in range(2):
            for x in range(2):
                ref = st.C[role][y][x] if role < 4 else st.T[role - 4][y][x]
                assert np.max(np.abs(g.env(role, x, y) - ref)) < 1e-14


@pytest.mark.parametrize("direction", ["L", "R", "U", "D"])
def test_single_move_each_direction(direction):
    w = synth.workload("real", seed=1, chi=12)
    g = gpu_ctm(w["tensors"], w["pattern"], 12)
    g.move(direction, 1)
    st = _oracle_run(w, 12, [direction])
    _compare_rdms(g, st, w)
    _compare_spectra(g, st)


def test_real_D2_chi16_twenty_sweeps_energy_rdms_spectra():
    """Real iid tensors, d=8, D=2, chi=16, 20 sweeps, J=(1,1,1)."""
    w = synth.workload("real", seed=0)
    g = gpu_ctm(w["tensors"], w["pattern"], 16)
    g.sweep(20)
    st = _oracle_run(w, 16, ["sweep"] * 20)
    e_ref = O.energy_per_spin(O.bond_rdms(st, w["tensors"], w["pattern"]), w["J"], 2, 2)
    e_gpu = g.energy(w["J"])
    assert abs(e_gpu - e_ref) < TOL * abs(e_ref)
    _compare_rdms(g, st, w)
    _compare_site_rdms(g, st, w)
    _compare_spectra(g, st)


def test_product_noise_D3_chi18_complex():
    """Complex product state + 0.1 noise, D=3, chi=18, 3 sweeps."""
    w = synth.workload("product_noise", seed=2, D=3, chi=18)
    g = gpu_ctm(w["tensors"], w["pattern"], 18)
    g.sweep(3)
    st = _oracle_run(w, 18, ["sweep"] * 3)
    e_ref = O.energy_per_spin(O.bond_rdms(st, w["tensors"], w["pattern"]), w["J"], 2, 2)
    assert abs(g.energy(w["J"]) - e_ref) < TOL * abs(e_ref)
    _compare_rdms(g, st, w)
    _compare_site_rdms(g, st, w)
    _compare_spectra(g, st)


def test_site_rdms_at_trace_init_and_on_a_1x1_cell():
    w = synth.workload("product_noise", seed=7, D=3, chi=9)
    g = gpu_ctm(w["tensors"], w["pattern"], 9)
    _compare_site_rdms(g, O.make_state(w["tensors"], w["pattern"], 3, 9), w)
    rng = np.random.default_rng(31)
    A = rng.standard_normal((2, 2, 2, 2, 2)) + 1j * rng.standard_normal((2, 2, 2, 2, 2))
    w1 = {"tensors": [A / np.abs(A).max()], "pattern": [[0]], "D": 2}
    g1 = gpu_ctm(w1["tensors"], w1["pattern"], 8)
    g1.sweep(2)
    _compare_site_rdms(g1, _oracle_run(w1, 8, ["sweep"] * 2), w1)


def test_ising_onsager_on_gpu():
    from test_oracle_pins import ising_tensor, onsager_minus_beta_f
    beta = 0.3
    A = ising_tensor(beta)
    g = gpu_ctm([A], [[0]], 16, cutoff=1e-12)
    g.sweep(30)
    assert abs(np.log(abs(g.kappa())) / 4 - onsager_minus_beta_f(beta)) < 1e-9


def test_kappa_and_fidelity_match_oracle():
    w1 = synth.workload("product_noise", seed=4, D=2, chi=8)
    w2 = synth.workload("product_noise", seed=5, D=2, chi=8)
    t1, t2, pat = w1["tensors"], w2["tensors"], w1["pattern"]
    hs = [gpu_ctm(t1, pat, 8, bra=t2), gpu_ctm(t1, pat, 8), gpu_ctm(t2, pat, 8)]
    ks_ref = []
    for a, b in ((t1, t2), (t1, t1), (t2, t2)):
        st = O.make_state(a, pat, 2, 8, mixed_with=b)
        opt = oracle_options(8, 2)
        for _ in range(4):
            st = O.sweep(st, opt)
        ks_ref.append(O.kappa(st))
    for hnd in hs:
        hnd.sweep(4)
    for hnd, kr in zip(hs, ks_ref):
        assert abs(hnd.kappa() - kr) < TOL * abs(kr)
    from paper_1711_04798_gb300 import CTM
    d_gpu = CTM.fidelity(*hs)
    d_ref = O.fidelity(*ks_ref)
    assert abs(d_gpu[0] - d_ref[0]) < TOL and abs(d_gpu[1] - d_ref[1]) < TOL


@pytest.mark.parametrize("Nv", [2, 4])
def test_boundary_rho_matches_oracle(Nv):
    w = synth.workload("product_noise", seed=6, D=2, chi=8)
    g = gpu_ctm(w["tensors"], w["pattern"], 8)
    g.sweep(3)
    st = _oracle_run(w, 8, ["sweep"] * 3)
    lam_gpu, S_gpu = g.boundary_rho(0, Nv)
    lam_ref = O.boundary_spectrum(st, 0, Nv)
    assert np.max(np.abs(lam_gpu - lam_ref)) < 1e-10
    assert abs(S_gpu - O.entropy(lam_ref)) < 1e-10


def test_errors_are_reported_not_fatal():
    from paper_1711_04798_gb300 import CTMError
    w = synth.workload("real", seed=0)
    with pytest.raises(CTMError):
        gpu_ctm(w["tensors"], w["pattern"], 3)  # chi < D^2
    g = gpu_ctm(w["tensors"], w["pattern"], 8)
    with pytest.raises(CTMError):
        g.boundary_rho(0, 3)  # not a multiple of Ly
    g.sweep(1)  # the handle is still usable


@pytest.mark.parametrize("chi", [33, 40])
def test_cluster_sized_cores_match_oracle(chi):
    """chi >= 32: the projector core (k = chi + 16 rows), the CholeskyQR
    factorisations and the corner spectra (chi x chi) run on the 16-CTA cluster
    kernels; odd chi leaves a dummy player in the Jacobi pair schedule."""
    w = synth.workload("product_noise", seed=6, D=2, chi=chi)
    g = gpu_ctm(w["tensors"], w["pattern"], chi)
    g.sweep(2)
    st = _oracle_run(w, chi, ["sweep"] * 2)
    e_ref = O.energy_per_spin(O.bond_rdms(st, w["tensors"], w["pattern"]), w["J"], 2, 2)
    assert abs(g.energy(w["J"]) - e_ref) < TOL * abs(e_ref)
    _compare_rdms(g, st, w)
    _compare_spectra(g, st)
    g.close()
    gp = gpu_ctm(w["tensors"], w["pattern"], chi, prec="bf16x3", cutoff=1e-6)
    gp.sweep(2)
    st6 = _oracle_run(w, chi, ["sweep"] * 2, cutoff=1e-6)
    e6 = O.energy_per_spin(O.bond_rdms(st6, w["tensors"], w["pattern"]), w["J"], 2, 2)
    assert abs(gp.energy(w["J"]) - e6) < 1e-5
    gp.close()


@pytest.mark.parametrize("recipe", ["real_D2_chi16_sweeps3", "product_noise_D3_chi18_sweeps3"])
def test_against_the_oracles_range_finder(recipe):
    """Secondary check: the oracle's restatement of the GPU's own projector
    route (randomized range finder, the same seeded test matrix, k = chi + 16,
    q = 2) agrees with the GPU to the same tolerances."""
    if recipe.startswith("real"):
        w, chi = synth.workload("real", seed=0), 16
    else:
        w, chi = synth.workload("product_noise", seed=2, D=3, chi=18), 18
    g = gpu_ctm(w["tensors"], w["pattern"], chi)
    g.sweep(3)
    st = _oracle_run(w, chi, ["sweep"] * 3, proj="rsvd")
    e_ref = O.energy_per_spin(O.bond_rdms(st, w["tensors"], w["pattern"]), w["J"], 2, 2)
    assert abs(g.energy(w["J"]) - e_ref) < TOL * abs(e_ref)
    _compare_rdms(g, st, w)
    _compare_spectra(g, st)
    g.close()


def test_converge_matches_oracle():
    """ipeps_ctm_converge: sweeps until the corner spectra change by less than
    tol (max over corners of ||s/s_0 - s_old/s_old_0||_2), the oracle's
    ctm_converge with the exact SVD.  The sweep counts may differ by one where
    the last delta lies close to tol; the converged readouts agree to 1e-10."""
    w, chi = synth.workload("real", seed=0), 16
    g = gpu_ctm(w["tensors"], w["pattern"], chi)
    n_gpu, delta_gpu, ok = g.converge(1e-10, 100)
    st = O.make_state(w["tensors"], w["pattern"], w["D"], chi)
    st, n_ref, delta_ref = O.ctm_converge(st, oracle_options(chi, w["D"]), 1e-10, 100)
    print(f"converge: gpu {n_gpu} sweeps (delta {delta_gpu:.2e}), oracle {n_ref} ({delta_ref:.2e})")
    assert ok and delta_gpu < 1e-10 and delta_ref < 1e-10
    assert abs(n_gpu - n_ref) <= 1
    e_ref = O.energy_per_spin(O.bond_rdms(st, w["tensors"], w["pattern"]), w["J"], 2, 2)
    assert abs(g.energy(w["J"]) - e_ref) < TOL * abs(e_ref)
    _compare_rdms(g, st, w)
    _compare_site_rdms(g, st, w)
    _compare_spectra(g, st)
    # a budget too small to converge reports ENOCONV with the sweeps it took
    g2 = gpu_ctm(w["tensors"], w["pattern"], chi)
    n2, d2, ok2 = g2.converge(1e-10, 2)
    assert not ok2 and n2 == 2 and d2 > 1e-10
    g.close()
    g2.close()


@pytest.mark.parametrize("D,chi,seed,sweeps,spec_tol", [(2, 16, 0, 6, TOL), (3, 18, 2, 3, 1e-7)])
def test_two_corner_projectors_match_oracle(D, chi, seed, sweeps, spec_tol):
    """The two-corner projector option (ipeps_options.corners = 2, X = Q1^T Q4:
    the ring opened on the cut's own side, Sec. II.C): energy and RDMs at 1e-10
    against the exact-SVD oracle of the same route; the corner spectra at 1e-10
    at D = 2, chi = 16, and at D = 3, chi = 18 within the range finder's own
    distance from the exact SVD on this route (4e-8 in the spectra, recorded
    in tests/test_projector_routes.py; the slower decay of the two-corner
    ring's singular values leaves the range finder short of convergence, and
    the GPU's FP64 route lies 2e-8 from the oracle's restatement of it)."""
    w = synth.workload("product_noise", seed=seed, D=D, chi=chi)
    g = gpu_ctm(w["tensors"], w["pattern"], chi, corners=2)
    g.sweep(sweeps)
    st = _oracle_run(w, chi, ["sweep"] * sweeps, corners=2)
    e_ref = O.energy_per_spin(O.bond_rdms(st, w["tensors"], w["pattern"]), w["J"], 2, 2)
    e = g.energy(w["J"])
    err = spectra_err(g.spectra(), O.corner_spectra(st))
    print(f"two corners D{D} chi{chi}: E gpu {e:.15f} oracle {e_ref:.15f}, spectra {err:.1e}")
    assert abs(e - e_ref) < TOL * abs(e_ref)
    _compare_rdms(g, st, w)
    assert err < spec_tol
    g.close()


def test_two_corner_projectors_in_the_precision_form():
    """BF16x6 with the two-corner projectors against the oracle of that route
    at the same cutoff: the 1e-6 energy target."""
    w = synth.workload("product_noise", seed=2, D=3, chi=18)
    g = gpu_ctm(w["tensors"], w["pattern"], 18, corners=2, prec="bf16x6", cutoff=1e-6)
    g.sweep(3)
    st = _oracle_run(w, 18, ["sweep"] * 3, corners=2, cutoff=1e-6)
    e_ref = O.energy_per_spin(O.bond_rdms(st, w["tensors"], w["pattern"]), w["J"], 2, 2)
    e = g.energy(w["J"])
    print(f"two corners BF16x6: |dE| {abs(e - e_ref):.1e}")
    assert abs(e - e_ref) < 1e-6
    g.close()
