"""FP64 CTM oracle (test infrastructure only: see the package docstring).

The paper (Sec. II.C, Fig. 3) fixes WHAT is computed: an environment of four
chi x chi corner matrices C1..C4 and eight chi x chi x D^2 half-row/column
tensors T around a 2x2 unit cell of double-layer tensors a = sum_s A_s A_s^*
(Fig. 3a), obtained with the directional CTM of its refs. Orus2009 and
Corboz2010a.  It prints no move details, so the steps below are this oracle's reading of
those references, written out plainly:

* one environment set {C1..C4, T1..T4} per cell position (x, y) (x to the
  right, y downwards): C1 upper-left, C2 upper-right, C3 lower-right, C4
  lower-left; T1 above, T2 right, T3 below, T4 left of the site.
* legs are listed clockwise-covariantly: C1[d,r] C2[l,d] C3[u,l] C4[r,u];
  T1[l,d,r] T2[u,l,d] T3[r,u,l] T4[d,r,u]; a[u,l,d,r].  Every D^2 leg is the
  fused (ket, bra) pair, index ket*D + bra.  Rotating the lattice by 90 degrees
  counter-clockwise therefore only relabels: C'_j = C_{j+1}, T'_j = T_{j+1},
  a' = a with legs (r,u,l,d), site (x,y) -> (y, -x).
* a left move absorbs the unit-cell columns x = 0 .. Lx-1 in turn; the other
  three directions are the left move in a rotated frame.  One sweep is
  L, R, U, D.
* projectors come from the four enlarged corners of the 2x2 plaquette on each
  cut (upper half Q1 Q2, lower half Q4 Q3^T), truncated SVD of the ring matrix
  X = (Q1 Q2)^T (Q4 Q3^T) to chi, keeping s_i > cutoff * s_0.
* environment tensors are zero-padded to chi from the trace initialisation
  (boundary bonds of the initial tensors traced ket against bra).
* each renormalised tensor is divided by its Frobenius norm.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "CTMOptions",
    "CTMState",
    "double_layer",
    "trace_init",
    "rotate",
    "rotate_k",
    "enlarged_corners",
    "ring_matrix_factors",
    "truncated_svd",
    "projectors",
    "left_move",
    "move",
    "sweep",
    "corner_spectra",
    "spectra_delta",
    "ctm_converge",
    "make_state",
]

DIRS = {"L": 0, "U": 1, "R": 2, "D": 3}
SWEEP_ORDER = ("L", "R", "U", "D")


@dataclass
class CTMOptions:
    """Projector choices.

    ``proj``: ``"svd"`` = exact truncated SVD of X (LAPACK), ``"rsvd"`` = the
    randomized range finder with subspace iteration (Halko, Martinsson & Tropp
    2011, Alg. 4.4 + 5.1) using the fixed test matrix ``omega``.

    ``corners``: 4 (default) builds the projectors from the full ring of the
    four enlarged corners; 2 from the left half only, R_up = Q1 and R_dn = Q4
    (the two-corner variant, about a third of the cost): untruncated both are
    exact, truncated they differ by the truncation error.

    ``ties`` collects every cut where the chi-th and (chi+1)-th singular values
    agree to a relative ``tie_tol``: the truncation then splits a multiplet,
    the kept subspace is not unique, and the environment (and every readout
    after it) depends on rounding, so a run that records a tie is not a parity
    reference at that chi.  Recording changes nothing in the arithmetic.
    """

    chi: int
    proj: str = "rsvd"
    oversample: int = 16
    power: int = 2
    cutoff: float = 1e-8
    orth_tol: float = 1e-14
    omega: np.ndarray | None = None
    tie_tol: float = 1e-10
    ties: list = field(default_factory=list)  # (chi, s_chi, s_chi+1) per tied cut
    corners: int = 4  # 4: four-corner ring; 2: two-corner (left half) projectors


@dataclass
class CTMState:
    Lx: int
    Ly: int
    D: int
    chi: int
    a: list  # a[y][x] -> (D2, D2, D2, D2)
    C: list = field(default_factory=list)  # C[j][y][x] -> (chi, chi), j = 0..3 for C1..C4
    T: list = field(default_factory=list)  # T[j][y][x] -> (chi, D2, chi)

    @property
    def D2(self) -> int:
        return self.D * self.D


# ---------------------------------------------------------------------------
# Fig. 3(a): double-layer (reduced) tensor a = sum_s A_s conj(A_s); Fig. 4 /
# Sec. III uses the mixed version sum_s A_s(lambda1) conj(B_s(lambda2)).
# ---------------------------------------------------------------------------
def double_layer(A: np.ndarray, B: np.ndarray | None = None) -> np.ndarray:
    """a[(u u'), (l l'), (d d'), (r r')] = sum_p A[p,u,l,d,r] conj(B[p,u',l',d',r'])."""
    if B is None:
        B = A
    D = A.shape[1]
    a = np.einsum("pulsr,pULSR->uUlLsSrR", A.astype(np.complex128), np.conj(B.astype(np.complex128)), optimize=True)
    return a.reshape(D * D, D * D, D * D, D * D)


def _pad(t: np.ndarray, shape) -> np.ndarray:
    out = np.zeros(shape, dtype=np.complex128)
    out[tuple(slice(0, s) for s in t.shape)] = t
    return out


def _normalize(t: np.ndarray) -> np.ndarray:
    n = np.linalg.norm(t)
    return t / n if n > 0 else t


def trace_init(a_cell, D: int, chi: int):
    """Initial environment: each C/T is the neighbouring double-layer tensor
    with its outward legs traced ket against bra (open boundary), padded to chi.

    C1[x,y] <- site (x-1,y-1), legs u,l traced;  C2 <- (x+1,y-1), u,r traced;
    C3 <- (x+1,y+1), d,r;  C4 <- (x-1,y+1), l,d;  T1 <- (x,y-1), u;
    T2 <- (x+1,y), r;  T3 <- (x,y+1), d;  T4 <- (x-1,y), l.
    """
    Ly, Lx = len(a_cell), len(a_cell[0])
    D2 = D * D
    if chi < D2:
        raise ValueError("chi must be >= D^2 for the trace initialisation")

    def site(x, y):
        return a_cell[y % Ly][x % Lx]

    C = [[[None] * Lx for _ in range(Ly)] for _ in range(4)]
    T = [[[None] * Lx for _ in range(Ly)] for _ in range(4)]
    for y in range(Ly):
        for x in range(Lx):
            s = site(x - 1, y - 1).reshape(D, D, D, D, D2, D2)
            C[0][y][x] = np.einsum("iijjdr->dr", s, optimize=True)
            s = site(x + 1, y - 1).reshape(D, D, D2, D2, D, D)
            C[1][y][x] = np.einsum("iildjj->ld", s, optimize=True)
            s = site(x + 1, y + 1).reshape(D2, D2, D, D, D, D)
            C[2][y][x] = np.einsum("uliijj->ul", s, optimize=True)
            s = site(x - 1, y + 1).reshape(D2, D, D, D, D, D2)
            C[3][y][x] = np.einsum("uiijjr->ru", s, optimize=True)
            s = site(x, y - 1).reshape(D, D, D2, D2, D2)
            T[0][y][x] = np.einsum("iildr->ldr", s, optimize=True)
            s = site(x + 1, y).reshape(D2, D2, D2, D, D)
            T[1][y][x] = np.einsum("uldii->uld", s, optimize=True)
            s = site(x, y + 1).reshape(D2, D2, D, D, D2)
            T[2][y][x] = np.einsum("uliir->rul", s, optimize=True)
            s = site(x - 1, y).reshape(D2, D, D, D2, D2)
            T[3][y][x] = np.einsum("uiidr->dru", s, optimize=True)
    for j in range(4):
        for y in range(Ly):
            for x in range(Lx):
                C[j][y][x] = _normalize(_pad(C[j][y][x], (chi, chi)))
                T[j][y][x] = _normalize(_pad(T[j][y][x], (chi, D2, chi)))
    return C, T


def make_state(tensors, pattern, D: int, chi: int, mixed_with=None) -> CTMState:
    """Build a CTMState from host tensors A[p,u,l,d,r] and pattern[y][x] -> id.

    With ``mixed_with`` (a second tensor list) the network is the fidelity
    network of Sec. III: e = sum_s A_s conj(B_s) at every site.
    """
    Ly, Lx = len(pattern), len(pattern[0])
    if mixed_with is None:
        a_list = [double_layer(A) for A in tensors]
    else:
        a_list = [double_layer(A, B) for A, B in zip(tensors, mixed_with)]
    a_cell = [[a_list[pattern[y][x]] for x in range(Lx)] for y in range(Ly)]
    C, T = trace_init(a_cell, D, chi)
    return CTMState(Lx=Lx, Ly=Ly, D=D, chi=chi, a=a_cell, C=C, T=T)


# ---------------------------------------------------------------------------
# Lattice rotation (relabelling only; see module docstring).
# ---------------------------------------------------------------------------
def rotate(st: CTMState) -> CTMState:
    """Rotate the whole network by 90 degrees counter-clockwise."""
    Lx, Ly = st.Lx, st.Ly
    nLx, nLy = Ly, Lx
    a = [[None] * nLx for _ in range(nLy)]
    C = [[[None] * nLx for _ in range(nLy)] for _ in range(4)]
    T = [[[None] * nLx for _ in range(nLy)] for _ in range(4)]
    for yp in range(nLy):
        for xp in range(nLx):
            x, y = (-yp) % Lx, xp % Ly
            a[yp][xp] = np.ascontiguousarray(np.transpose(st.a[y][x], (3, 0, 1, 2)))
            for j in range(4):
                C[j][yp][xp] = st.C[(j + 1) % 4][y][x]
                T[j][yp][xp] = st.T[(j + 1) % 4][y][x]
    return CTMState(Lx=nLx, Ly=nLy, D=st.D, chi=st.chi, a=a, C=C, T=T)


def rotate_k(st: CTMState, k: int) -> CTMState:
    for _ in range(k % 4):
        st = rotate(st)
    return st


# ---------------------------------------------------------------------------
# Enlarged corners of the 2x2 plaquette with upper-left site (x, y).
# Row/column fusions: every cut leg is (boundary chi, D^2) with chi slow.
# ---------------------------------------------------------------------------
def enlarged_corners(st: CTMState, x: int, y: int):
    """Return Q1..Q4 as (chi*D2, chi*D2) matrices.

    Q1[(d_T4,d_a),(r_T1,r_a)]  upper-left  (C1, T1, T4, a at (x,y))
    Q2[(l_T1,l_a),(d_T2,d_a)]  upper-right (T1, C2, T2, a at (x+1,y))
    Q3[(u_T2,u_a),(l_T3,l_a)]  lower-right (T2, C3, T3, a at (x+1,y+1))
    Q4[(u_T4,u_a),(r_T3,r_a)]  lower-left  (T4, C4, T3, a at (x,y+1))
    """
    Lx, Ly = st.Lx, st.Ly
    x0, x1 = x % Lx, (x + 1) % Lx
    y0, y1 = y % Ly, (y + 1) % Ly
    C, T, a = st.C, st.T, st.a
    N = st.chi * st.D2
    # each corner as three pairwise contractions: C.T, then .T, then .a
    CT = np.einsum("ab,bcr->acr", C[0][y0][x0], T[0][y0][x0], optimize=True)
    CTT = np.einsum("dea,acr->decr", T[3][y0][x0], CT, optimize=True)
    Q1 = np.einsum("decr,ceDR->dDrR", CTT, a[y0][x0], optimize=True)
    TC = np.einsum("Ltg,gh->Lth", T[0][y0][x1], C[1][y0][x1], optimize=True)
    TCT = np.einsum("Lth,hmE->LtmE", TC, T[1][y0][x1], optimize=True)
    Q2 = np.einsum("LtmE,tKem->LKEe", TCT, a[y0][x1], optimize=True)
    TC = np.einsum("Umh,hg->Umg", T[1][y1][x1], C[2][y1][x1], optimize=True)
    TCT = np.einsum("Umg,gtL->UmtL", TC, T[2][y1][x1], optimize=True)
    Q3 = np.einsum("UmtL,uKtm->UuLK", TCT, a[y1][x1], optimize=True)
    CT = np.einsum("gh,hmU->gmU", C[3][y1][x0], T[3][y1][x0], optimize=True)
    TCT = np.einsum("gmU,Rtg->mUtR", CT, T[2][y1][x0], optimize=True)
    Q4 = np.einsum("mUtR,umtr->UuRr", TCT, a[y1][x0], optimize=True)
    return (Q1.reshape(N, N), Q2.reshape(N, N), Q3.reshape(N, N), Q4.reshape(N, N))


def ring_matrix_factors(Q1, Q2, Q3, Q4):
    """Upper half R_up = Q1 Q2, lower half R_dn = Q4 Q3^T (rows: the left cut),
    and the ring opened on the right cut, X = R_up^T R_dn."""
    R_up = Q1 @ Q2
    R_dn = Q4 @ Q3.T
    X = R_up.T @ R_dn
    return R_up, R_dn, X


def _orth(Y: np.ndarray, tol: float) -> np.ndarray:
    """Orthonormal basis of the numerical range of Y (columns with
    singular value above tol * largest)."""
    U, s, _ = np.linalg.svd(Y, full_matrices=False)
    if s.size == 0 or s[0] == 0.0:
        return U[:, :0]
    return U[:, s > tol * s[0]]


def truncated_svd(X: np.ndarray, opt: CTMOptions):
    """Return (U, s, V) of X, singular values descending (all that the method
    produces; truncation happens in ``projectors``)."""
    if opt.proj == "svd":
        U, s, Vh = np.linalg.svd(X)
        return U, s, Vh.conj().T
    if opt.proj != "rsvd":
        raise ValueError(opt.proj)
    K = X.shape[0]
    k = opt.chi + opt.oversample
    Om = opt.omega
    if Om is None or Om.shape != (K, k):
        raise ValueError(f"rsvd needs omega of shape {(K, k)}")
    Q = _orth(X @ Om, opt.orth_tol)
    for _ in range(opt.power):
        Z = _orth(X.conj().T @ Q, opt.orth_tol)
        Q = _orth(X @ Z, opt.orth_tol)
    W = X.conj().T @ Q  # = B^H with B = Q^H X
    Uw, s, Vwh = np.linalg.svd(W, full_matrices=False)
    U = Q @ Vwh.conj().T
    V = Uw
    return U, s, V


def projectors(Q1, Q2, Q3, Q4, opt: CTMOptions):
    """Projector pair for the left cut of the plaquette.

    With the ring X = R_up^T R_dn = U S V^H truncated to chi_eff values
    (s_i > cutoff * s_0, at most chi):
        P  = R_dn V S^{-1/2}      (N x chi)   -> tensors above the cut
        Pt = S^{-1/2} U^H R_up^T  (chi x N)   -> tensors below the cut
    so that R_up^T (P Pt) R_dn = U_chi S_chi V_chi^H.
    """
    if opt.corners == 4:
        R_up, R_dn, X = ring_matrix_factors(Q1, Q2, Q3, Q4)
    elif opt.corners == 2:
        R_up, R_dn = Q1, Q4
        X = R_up.T @ R_dn
    else:
        raise ValueError(f"corners must be 4 or 2, not {opt.corners}")
    U, s, V = truncated_svd(X, opt)
    chi = opt.chi
    N = X.shape[0]
    keep = 0
    if s.size and s[0] > 0:
        keep = int(min(chi, np.count_nonzero(s > opt.cutoff * s[0])))
    if keep == chi and s.size > chi and s[chi] > opt.cutoff * s[0] and s[chi - 1] - s[chi] <= opt.tie_tol * s[chi]:
        opt.ties.append((chi, float(s[chi - 1]), float(s[chi])))
    P = np.zeros((N, chi), dtype=np.complex128)
    Pt = np.zeros((chi, N), dtype=np.complex128)
    if keep:
        isq = 1.0 / np.sqrt(s[:keep])
        P[:, :keep] = (R_dn @ V[:, :keep]) * isq[None, :]
        Pt[:keep, :] = isq[:, None] * (U[:, :keep].conj().T @ R_up.T)
    return P, Pt, s


def left_move(st: CTMState, opt: CTMOptions, columns=None) -> CTMState:
    """Absorb the unit-cell columns x = 0..Lx-1 from the left, one after another
    (``columns`` restricts the absorption to the listed columns, in order)."""
    Lx, Ly, chi, D2 = st.Lx, st.Ly, st.chi, st.D2
    C = [[row[:] for row in Cj] for Cj in st.C]
    T = [[row[:] for row in Tj] for Tj in st.T]
    st = CTMState(Lx=Lx, Ly=Ly, D=st.D, chi=chi, a=st.a, C=C, T=T)
    for x in (range(Lx) if columns is None else columns):
        Pm, Ptm = [], []
        for y in range(Ly):
            P, Pt, _ = projectors(*enlarged_corners(st, x, y), opt)
            Pm.append(P.reshape(chi, D2, chi))
            Ptm.append(Pt.reshape(chi, chi, D2))
        xn = (x + 1) % Lx
        newC1, newT4, newC4 = [], [], []
        for y in range(Ly):
            ym = (y - 1) % Ly
            c1 = np.einsum("asr,asn->nr", np.einsum("ab,bsr->asr", C[0][y][x], T[0][y][x]), Pm[ym], optimize=True)
            t4 = np.einsum("emf,ehb->mfhb", T[3][y][x], Pm[y], optimize=True)
            t4 = np.einsum("mfhb,gmhr->fbgr", t4, st.a[y][x], optimize=True)
            t4 = np.einsum("fbgr,afg->bra", t4, Ptm[ym], optimize=True)
            c4 = np.einsum("rsu,aus->ra", np.einsum("gu,rsg->rsu", C[3][y][x], T[2][y][x]), Ptm[y], optimize=True)
            newC1.append(_normalize(c1))
            newT4.append(_normalize(t4))
            newC4.append(_normalize(c4))
        for y in range(Ly):
            C[0][y][xn] = newC1[y]
            T[3][y][xn] = newT4[y]
            C[3][y][xn] = newC4[y]
    return st


def move(st: CTMState, direction: str, opt: CTMOptions) -> CTMState:
    k = DIRS[direction]
    return rotate_k(left_move(rotate_k(st, k), opt), 4 - k)


def sweep(st: CTMState, opt: CTMOptions) -> CTMState:
    for dname in SWEEP_ORDER:
        st = move(st, dname, opt)
    return st


def corner_spectra(st: CTMState) -> np.ndarray:
    """Singular values of every corner, normalised by the largest:
    array [4, Ly, Lx, chi] (C1..C4)."""
    out = np.zeros((4, st.Ly, st.Lx, st.chi))
    for j in range(4):
        for y in range(st.Ly):
            for x in range(st.Lx):
                s = np.linalg.svd(st.C[j][y][x], compute_uv=False)
                out[j, y, x] = s / s[0] if s[0] > 0 else s
    return out


def spectra_delta(s_new: np.ndarray, s_old: np.ndarray) -> float:
    """max over corners of || s/s_0 - s_old/s_old_0 ||_2."""
    d = np.linalg.norm((s_new - s_old).reshape(-1, s_new.shape[-1]), axis=1)
    return float(d.max())


def ctm_converge(st: CTMState, opt: CTMOptions, tol: float, max_sweeps: int):
    """Sweep until the corner spectra change by less than tol."""
    s_old = corner_spectra(st)
    delta = np.inf
    n = 0
    while n < max_sweeps:
        st = sweep(st, opt)
        n += 1
        s_new = corner_spectra(st)
        delta = spectra_delta(s_new, s_old)
        s_old = s_new
        if delta < tol:
            break
    return st, n, delta
