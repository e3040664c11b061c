"""Leading boundary spectrum of long cylinders (Sec. IV) on the GPU: dense
rings from one product of two half rings, Lanczos in the sigma_R inner
product, against the oracle's plain definition (all eigenvalues of the dense
product sigma_L^T sigma_R, the k largest kept)."""
import numpy as np
import pytest

import oracle as O
import synth
from gpu_common import gpu_ctm, oracle_options

pytestmark = pytest.mark.gpu


def _pair(D, chi, sweeps, seed=2, prec="fp64"):
    w = synth.workload("product_noise", seed=seed, D=D, chi=chi)
    g = gpu_ctm(w["tensors"], w["pattern"], chi, prec=prec)
    g.sweep(sweeps)
    st = O.make_state(w["tensors"], w["pattern"], D, chi)
    opt = oracle_options(chi, D)
    for _ in range(sweeps):
        st = O.sweep(st, opt)
    return g, st


@pytest.mark.parametrize("D,chi,Nv,k", [(2, 12, 4, 4), (2, 12, 8, 12), (3, 18, 6, 16)])
def test_topk_matches_oracle_definition(D, chi, Nv, k):
    g, st = _pair(D, chi, 5)
    lam, S, rest, nconv = g.boundary_rho_topk(0, Nv, k, max_iter=min(D ** Nv, 400), tol=1e-12)
    ref, S_ref, rest_ref = O.boundary_spectrum_topk(st, 0, Nv, k)
    assert nconv == k
    assert np.max(np.abs(lam - ref)) < 1e-9 * ref[0], (lam, ref)
    assert abs(S - S_ref) < 1e-9 and abs(rest - rest_ref) < 1e-9
    assert np.all(np.diff(lam) <= 1e-15)
    g.close()


def test_topk_agrees_with_dense_route_in_precision_form():
    """Both GPU routes (dense Jacobi spectrum and Lanczos) on one BF16x3 environment."""
    g, _ = _pair(3, 18, 4, prec="bf16x3")
    dense, _ = g.boundary_rho(0, 4)
    lam, _, rest, nconv = g.boundary_rho_topk(0, 4, 10, max_iter=81, tol=1e-12)
    assert nconv == 10
    # same operators up to the precision form's rounding of the ring products
    assert np.max(np.abs(lam - dense[:10])) < 1e-6 * dense[0]
    assert abs(rest - dense[10:].sum()) < 1e-6
    g.close()


def test_topk_argument_errors():
    from paper_1711_04798_gb300 import CTMError
    g, _ = _pair(2, 8, 1)
    with pytest.raises(CTMError) as ei:
        g.boundary_rho_topk(0, 4, 8, max_iter=4)  # k > max_iter
    assert ei.value.status == 1
    with pytest.raises(CTMError):
        g.boundary_rho_topk(0, 3, 2)  # Nv not a multiple of Ly = 2
    lam, _, _, _ = g.boundary_rho_topk(0, 2, 2, max_iter=4)  # the handle stays usable
    assert np.all(np.isfinite(lam))
    g.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("bf16x6", 1e-5)])
@pytest.mark.parametrize("Nv", [2, 4])
def test_boundary_renyi2_matches_oracle(prec, tol, Nv):
    """Second Renyi entropy from the traces of M = sigma_L^T sigma_R (Sec. IV)
    against the oracle's, and against the dense spectrum's purity on the GPU."""
    w = synth.workload("product_noise", seed=6, D=2, chi=8)
    g = gpu_ctm(w["tensors"], w["pattern"], 8, prec=prec, cutoff=1e-6 if prec != "fp64" else 1e-8)
    g.sweep(3)
    st = O.make_state(w["tensors"], w["pattern"], 2, 8)
    opt = oracle_options(8, 2, cutoff=1e-6 if prec != "fp64" else 1e-8)
    for _ in range(3):
        st = O.sweep(st, opt)
    S2, p = g.boundary_renyi2(0, Nv)
    S2_ref, p_ref = O.boundary_renyi2(st, 0, Nv)
    lam, _ = g.boundary_rho(0, Nv)
    print(f"{prec} Nv={Nv}: S2 {S2:.12f} oracle {S2_ref:.12f}; purity vs dense spectrum "
          f"{abs(p - np.sum(lam ** 2)):.1e}")
    assert abs(S2 - S2_ref) < tol and abs(p - p_ref) < tol
    assert abs(p - np.sum(lam ** 2)) < tol
    g.close()


@pytest.mark.parametrize("Nv", [2, 4, 8])
def test_refined_boundary_spectrum_matches_oracle(Nv):
    """Sec. IV beyond the ring approximation: the rings refined by power
    iteration with the exact column transfer matrices (the same fixed number
    of iterations on both sides), against the oracle's refinement, up to the
    literal circumference of eight block sites (D = 2: a 256 x 256 operator)."""
    w = synth.workload("product_noise", seed=6, D=2, chi=8)
    g = gpu_ctm(w["tensors"], w["pattern"], 8)
    g.sweep(3)
    st = O.make_state(w["tensors"], w["pattern"], 2, 8)
    opt = oracle_options(8, 2)
    for _ in range(3):
        st = O.sweep(st, opt)
    iters = 12
    lam, S, it, ch = g.boundary_rho_refined(0, Nv, iters=iters, tol=0.0)
    lam_ref, it_ref, ch_ref = O.refined_boundary_spectrum(st, 0, Nv, iters, tol=0.0)
    lam_ring = O.boundary_spectrum(st, 0, Nv)
    print(f"Nv={Nv}: refined S {S:.12f} (oracle {O.entropy(lam_ref):.12f}), ring approximation "
          f"{O.entropy(lam_ring):.12f}; last change gpu {ch:.2e} oracle {ch_ref:.2e}")
    assert it == iters == it_ref
    assert np.max(np.abs(lam - lam_ref)) < 1e-10 and abs(S - O.entropy(lam_ref)) < 1e-10
    g.close()
