"""Shared helpers of the GPU parity tests: the library handle and the
oracle configured with the same projector options."""
import numpy as np

import oracle as O
import synth

DEFAULTS = dict(oversample=16, power=2, cutoff=1e-8, orth_tol=1e-14, omega_seed=7)


def oracle_options(chi, D, proj="rsvd", **kw):
    o = dict(DEFAULTS)
    o.update(kw)
    K, k = chi * D * D, chi + o["oversample"]
    return O.CTMOptions(chi=chi, proj=proj, oversample=o["oversample"], power=o["power"],
                        cutoff=o["cutoff"], orth_tol=o["orth_tol"],
                        omega=synth.omega(o["omega_seed"], K, k))


def gpu_ctm(tensors, pattern, chi, **kw):
    from paper_1711_04798_gb300 import CTM
    o = dict(DEFAULTS)
    o.update(kw)
    return CTM(tensors, pattern, chi, **o)


def rel_err(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
