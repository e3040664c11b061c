"""Write the stored oracle values of the full-size GPU parity tests.

Only ``oracle/`` (the FP64 CPU CTM) and ``synth/`` (the seeded inputs) are
used; nothing here touches the CUDA library.  Each record is an ``.npz`` file
beside this script, named for its workload:

``product_noise_D4_chi64_converged``
    Complex all-up product state + 0.1 complex normal noise, d = 8, D = 4,
    chi = 64, 2x2 cell, seed 0 (psi1) and seed 1 (psi2).  Exact truncated SVD
    projectors (Sec. II.C; the truncation to chi of the ring across the cut),
    cutoff 1e-8, swept from the trace initialisation until the corner spectra
    change by less than 1e-10 (Sec. II.C, environment iterated to
    convergence).  Energy per spin at (Jx, Jy, Jz) = (1, 1, 0.5) (Eq. H-KR,
    App. A), bond and site RDMs, corner spectra, and the fidelity per site of
    psi1 against psi2 from the converged mixed network (Sec. III, Eq.
    "fidelity", Fig. 4).

``product_noise_D5_chi100_cut8``
    The same recipe at D = 5, chi = 100, seed 0, cutoff 1e-8 (the FP64
    path), exact SVD projectors: the state after one sweep.

``product_noise_D5_chi100_cut6``
    The same at cutoff 1e-6 (the precision form's cutoff): the state after
    one sweep and the converged state (1e-10), with the number of sweeps
    taken.

``product_noise_D5_chi100_rsvd_sweep1``
    One sweep of the D = 5, chi = 100 recipe with the randomized range finder
    (k = chi + 16, q = 2, test matrix from seed 7), for the record of how far
    that projector route lies from the exact SVD at full size.

Usage: ``python tests/golden/make_golden.py NAME [NAME ...]`` (names as
above without the file suffix; ``all`` for every record).  Runs for minutes
(D = 4) to hours (D = 5 converged) on a CPU.
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import synth  # noqa: E402

TOL = 1e-10
MAX_SWEEPS = 120


def _readouts(st, w, J):
    rd = O.bond_rdms(st, w["tensors"], w["pattern"])
    return {
        "E": O.energy_per_spin(rd, J, 2, 2),
        "rho_h": rd["h"],
        "rho_v": rd["v"],
        "rho_site": O.site_rdms(st, w["tensors"], w["pattern"]),
        "spectra": O.corner_spectra(st),
    }


def _converge(st, opt, log, on_sweep=None):
    s_old = O.corner_spectra(st)
    delta, n = np.inf, 0
    while n < MAX_SWEEPS:
        t = time.time()
        st = O.sweep(st, opt)
        n += 1
        s_new = O.corner_spectra(st)
        delta = O.spectra_delta(s_new, s_old)
        s_old = s_new
        print(f"  {log}: sweep {n} delta {delta:.3e} ({time.time() - t:.1f} s)", flush=True)
        if on_sweep:
            on_sweep(n, st)
        if delta < TOL:
            break
    return st, n, delta


def d4_chi64(path):
    D, chi = 4, 64
    w1 = synth.workload("product_noise", seed=0, D=D, chi=chi)
    w2 = synth.workload("product_noise", seed=1, D=D, chi=chi)
    J = w1["J"]
    out = {"tol": TOL, "cutoff": 1e-8, "J": np.array(J)}
    kap = {}
    for tag, a, b in (("11", w1, None), ("22", w2, None), ("12", w1, w2)):
        opt = O.CTMOptions(chi=chi, proj="svd", cutoff=1e-8)
        st = O.make_state(a["tensors"], a["pattern"], D, chi,
                          mixed_with=None if b is None else b["tensors"])
        st, n, delta = _converge(st, opt, f"D4 chi64 psi{tag}")
        kap[tag] = O.kappa(st)
        out[f"sweeps_{tag}"] = n
        out[f"delta_{tag}"] = delta
        out[f"kappa_{tag}"] = kap[tag]
        out[f"ties_{tag}"] = len(opt.ties)
        out[f"spectra_{tag}"] = O.corner_spectra(st)
        if b is None:
            r = _readouts(st, a, J)
            for key, val in r.items():
                out[f"{key}_{tag}"] = val
    d_block, d_spin = O.fidelity(kap["12"], kap["11"], kap["22"])
    out["d_block"], out["d_spin"] = d_block, d_spin
    np.savez_compressed(path, **out)


def d5_chi100(path, cutoff, converge=True):
    D, chi = 5, 100
    w = synth.workload("product_noise", seed=0, D=D, chi=chi)
    opt = O.CTMOptions(chi=chi, proj="svd", cutoff=cutoff)
    st = O.make_state(w["tensors"], w["pattern"], D, chi)
    out = {"tol": TOL, "cutoff": cutoff, "J": np.array(w["J"])}

    def first(n, s):
        if n == 1:
            for key, val in _readouts(s, w, w["J"]).items():
                out[f"{key}_sweep1"] = val
            np.savez_compressed(path, **out)  # partial record while converging

    if not converge:
        st = O.sweep(st, opt)
        first(1, st)
        return
    st, n, delta = _converge(st, opt, f"D5 chi100 cut {cutoff:g}", first)
    for key, val in _readouts(st, w, w["J"]).items():
        out[f"{key}_conv"] = val
    out["sweeps"], out["delta"], out["ties"] = n, delta, len(opt.ties)
    np.savez_compressed(path, **out)


def d5_rsvd_sweep1(path):
    D, chi = 5, 100
    w = synth.workload("product_noise", seed=0, D=D, chi=chi)
    K, k = chi * D * D, chi + 16
    opt = O.CTMOptions(chi=chi, proj="rsvd", cutoff=1e-8, omega=synth.omega(7, K, k))
    st = O.sweep(O.make_state(w["tensors"], w["pattern"], D, chi), opt)
    out = {"cutoff": 1e-8, "J": np.array(w["J"])}
    for key, val in _readouts(st, w, w["J"]).items():
        out[f"{key}_sweep1"] = val
    np.savez_compressed(path, **out)


RECORDS = {
    "product_noise_D4_chi64_converged": d4_chi64,
    "product_noise_D5_chi100_cut8": lambda p: d5_chi100(p, 1e-8, converge=False),
    "product_noise_D5_chi100_cut6": lambda p: d5_chi100(p, 1e-6),
    "product_noise_D5_chi100_rsvd_sweep1": d5_rsvd_sweep1,
}


def main(names):
    if names == ["all"]:
        names = list(RECORDS)
    for name in names:
        t = time.time()
        RECORDS[name](os.path.join(HERE, name + ".npz"))
        print(f"{name}: written in {time.time() - t:.0f} s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["all"])
