"""Shared helpers of the GPU parity tests: the library handle and the
oracle configured with the same truncation options.

The oracle's projectors default to the exact truncated SVD of the ring
across the cut (Sec. II.C: the projectors keep the chi largest singular
directions of that ring).  The CUDA path reaches the same truncation through a
randomized range finder with subspace iteration; its distance to the exact
SVD on every parity recipe is recorded by ``tests/test_projector_routes.py``.
``proj="rsvd"`` gives the oracle's restatement of that range finder (same
test matrix, k = chi + 16, q = 2), the secondary check."""
import os

import numpy as np

import oracle as O
import synth

DEFAULTS = dict(oversample=16, power=2, cutoff=1e-8, orth_tol=1e-14, omega_seed=7)
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def oracle_options(chi, D, proj="svd", **kw):
    o = dict(DEFAULTS)
    o.update(kw)
    K, k = chi * D * D, chi + o["oversample"]
    omega = synth.omega(o["omega_seed"], K, k) if proj == "rsvd" else None
    return O.CTMOptions(chi=chi, proj=proj, oversample=o["oversample"], power=o["power"],
                        cutoff=o["cutoff"], orth_tol=o["orth_tol"], omega=omega, corners=o.get("corners", 4))


def gpu_ctm(tensors, pattern, chi, **kw):
    from paper_1711_04798_gb300 import CTM
    o = dict(DEFAULTS)
    o.update(kw)
    return CTM(tensors, pattern, chi, **o)


def rel_err(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def spectra_err(s, s_ref, floor=1e-8):
    """Largest |s_i/s_0 - s_ref_i/s_ref_0| over the values s_ref_i/s_ref_0 >= floor
    (both sides already normalised by their largest value)."""
    mask = np.asarray(s_ref) > floor
    return float(np.max(np.abs(np.asarray(s) - np.asarray(s_ref))[mask]))


def golden(name):
    """A stored oracle record written by tests/golden/make_golden.py."""
    path = os.path.join(GOLDEN, name + ".npz")
    if not os.path.exists(path):
        import pytest
        pytest.fail(f"missing oracle record {path}: run tests/golden/make_golden.py {name}")
    with np.load(path) as z:
        return {k: z[k] for k in z.files}
