"""Readouts from a converged CTM environment (oracle; test infrastructure only).

* nearest-neighbour reduced density matrices and the energy of the ruby model
  (Eq. H-KR of Sec. IV in block-site form, App. A),
* the fidelity per site (Sec. III, Eq. "fidelity" and Fig. 4),
* the boundary density operator spectrum and entanglement entropy on an
  infinite cylinder (Sec. IV, Eq. "rho" and Fig. "cylinder").
"""
from __future__ import annotations

import numpy as np

from .ctm import CTMState, rotate_k

__all__ = [
    "rdm_horizontal",
    "bond_rdms",
    "rdm_site",
    "site_rdms",
    "pauli_block_ops",
    "ruby_bond_hamiltonians",
    "star_bond_hamiltonians",
    "xyz_all_edges_bond_hamiltonians",
    "energy_per_spin",
    "site_type",
    "partition_ratios",
    "kappa",
    "fidelity",
    "ring_sigma",
    "boundary_spectrum",
    "spectrum_of_rings",
    "boundary_renyi2",
    "column_transfer_apply",
    "refined_rings",
    "refined_boundary_spectrum",
    "boundary_spectrum_topk",
    "fixed_rings",
    "entropy",
]


def _split(t: np.ndarray, axis: int, D: int) -> np.ndarray:
    """Split a fused (ket, bra) leg of length D*D into two legs."""
    shape = list(t.shape)
    shape[axis:axis + 1] = [D, D]
    return t.reshape(shape)


def rdm_horizontal(st: CTMState, A_cell, x: int, y: int) -> np.ndarray:
    """Two-site RDM of the horizontal bond (x,y)-(x+1,y), normalised to trace 1.

    Returned as a (d^2, d^2) matrix with rows (p_left, q_right) (ket) and
    columns (p', q') (bra): rho[(p q),(p' q')].
    """
    Lx, Ly, D = st.Lx, st.Ly, st.D
    x0, x1, y0 = x % Lx, (x + 1) % Lx, y % Ly
    C, T = st.C, st.T
    A = A_cell[y0][x0].astype(np.complex128)
    B = A_cell[y0][x1].astype(np.complex128)
    t1 = _split(T[0][y0][x0], 1, D)   # [l, u, u', r]
    t4 = _split(T[3][y0][x0], 1, D)   # [d, l, l', u]
    t3 = _split(T[2][y0][x0], 1, D)   # [r, d, d', l]
    # left half: (C1 T1) T4, open A and conj(A), then (C4 T3)
    L = np.einsum("ab,bUVh->aUVh", C[0][y0][x0], t1, optimize=True)
    L = np.einsum("eLMa,aUVh->eLMUVh", t4, L, optimize=True)
    L = np.einsum("eLMUVh,pULSr->eMVhpSr", L, A, optimize=True)
    L = np.einsum("eMVhpSr,qVMTs->ehpSrqTs", L, np.conj(A), optimize=True)
    CB = np.einsum("ge,kSTg->ekST", C[3][y0][x0], t3, optimize=True)
    left = np.einsum("ehpSrqTs,ekST->hrskpq", L, CB, optimize=True)
    u1 = _split(T[0][y0][x1], 1, D)   # [l, u, u', r]
    t2 = _split(T[1][y0][x1], 1, D)   # [u, r, r', d]
    b3 = _split(T[2][y0][x1], 1, D)   # [r, d, d', l]
    # right half: (T1 C2) T2, open B and conj(B), then (C3 T3)
    R = np.einsum("hUVc,cf->hUVf", u1, C[1][y0][x1], optimize=True)
    R = np.einsum("hUVf,fRSg->hUVRSg", R, t2, optimize=True)
    R = np.einsum("hUVRSg,pUlXR->hVSgplX", R, B, optimize=True)
    R = np.einsum("hVSgplX,qVmYS->hgplXqmY", R, np.conj(B), optimize=True)
    CB = np.einsum("gi,iXYk->gXYk", C[2][y0][x1], b3, optimize=True)
    right = np.einsum("hgplXqmY,gXYk->hlmkpq", R, CB, optimize=True)
    rho = np.einsum("hrskpq,hrskPQ->pPqQ", left, right, optimize=True)
    d = A.shape[0]
    rho = rho.reshape(d * d, d * d)
    return rho / np.trace(rho)


def rdm_site(st: CTMState, A_cell, x: int, y: int) -> np.ndarray:
    """One-site RDM at (x,y), normalised to trace 1, as a (d, d) matrix
    rho[p, p'] (row ket, column bra).

    Sec. II.C: a local expectation value is the network with the site's
    physical legs left open, the rest of the plane replaced by its environment
    (Fig. 3b).  Written as its definition: the eight environment tensors of
    the site are contracted into one ring E over the site's four double
    legs, then closed with A and conj(A):

        C1 T1 C2
        T4  .  T2        E[(u u'), (l l'), (d d'), (r r')]
        C4 T3 C3
    """
    Lx, Ly, D = st.Lx, st.Ly, st.D
    x0, y0 = x % Lx, y % Ly
    C = [st.C[j][y0][x0] for j in range(4)]
    T = [st.T[j][y0][x0] for j in range(4)]
    # C1[d,r] T1[l,u,r] C2[l,d]: a = C1 down, U = site up leg, e = C2 down
    top = np.einsum("ab,bUc->aUc", C[0], T[0])
    top = np.einsum("aUc,ce->aUe", top, C[1])
    # C4[r,u] T3[r,u,l] C3[u,l]: f = C4 up, V = site down leg, g = C3 up
    bottom = np.einsum("hf,iVh->fVi", C[3], T[2])
    bottom = np.einsum("fVi,gi->fVg", bottom, C[2])
    # T4[d,r,u] = [f, L, a], T2[u,l,d] = [e, R, g]
    E = np.einsum("aUe,fLa->UefL", top, T[3])
    E = np.einsum("UefL,eRg->UfLRg", E, T[1])
    E = np.einsum("UfLRg,fVg->ULVR", E, bottom)
    E = E.reshape(D, D, D, D, D, D, D, D)  # u u' l l' d d' r r'
    A = A_cell[y0][x0].astype(np.complex128)
    half = np.einsum("uUlLsSrR,pulsr->pULSR", E, A)
    rho = np.einsum("pULSR,qULSR->pq", half, np.conj(A))
    return rho / np.trace(rho)


def site_rdms(st: CTMState, tensors, pattern) -> np.ndarray:
    """One-site RDMs of every cell position: array [Ly, Lx, d, d]."""
    Lx, Ly = st.Lx, st.Ly
    A_cell = [[tensors[pattern[y][x]] for x in range(Lx)] for y in range(Ly)]
    d = A_cell[0][0].shape[0]
    out = np.zeros((Ly, Lx, d, d), dtype=np.complex128)
    for y in range(Ly):
        for x in range(Lx):
            out[y, x] = rdm_site(st, A_cell, x, y)
    return out


def _rotate_tensor(A: np.ndarray) -> np.ndarray:
    """A[p,u,l,d,r] of the network rotated 90 degrees counter-clockwise."""
    return np.ascontiguousarray(np.transpose(A, (0, 4, 1, 2, 3)))


def bond_rdms(st: CTMState, tensors, pattern):
    """All nearest-neighbour RDMs of the cell.

    Returns dict with 'h' -> array [Ly, Lx, d^2, d^2] for bonds (x,y)-(x+1,y)
    (left site first) and 'v' -> [Ly, Lx, d^2, d^2] for bonds (x,y)-(x,y+1)
    (upper site first).  Vertical bonds are horizontal bonds of the network
    rotated by 90 degrees counter-clockwise, where (x,y) -> (y, -x).
    """
    Lx, Ly = st.Lx, st.Ly
    A_cell = [[tensors[pattern[y][x]] for x in range(Lx)] for y in range(Ly)]
    d = A_cell[0][0].shape[0]
    h = np.zeros((Ly, Lx, d * d, d * d), dtype=np.complex128)
    v = np.zeros_like(h)
    for y in range(Ly):
        for x in range(Lx):
            h[y, x] = rdm_horizontal(st, A_cell, x, y)
    rst = rotate_k(st, 1)
    rA = [[None] * Ly for _ in range(Lx)]
    for yp in range(Lx):
        for xp in range(Ly):
            rA[yp][xp] = _rotate_tensor(A_cell[xp % Ly][(-yp) % Lx])
    for y in range(Ly):
        for x in range(Lx):
            v[y, x] = rdm_horizontal(rst, rA, y, (-x) % Lx)
    return {"h": h, "v": v}


# ---------------------------------------------------------------------------
# Ruby model in block-site form (App. A).  Block-site basis p = 4 b1 + 2 b2 + b3
# (spin 1 most significant), b = 0 meaning sigma^z = +1.
# ---------------------------------------------------------------------------
def pauli_block_ops():
    sx = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    sy = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
    sz = np.array([[1, 0], [0, -1]], dtype=np.complex128)
    I2 = np.eye(2, dtype=np.complex128)
    ops = {}
    for name, s in (("x", sx), ("y", sy), ("z", sz)):
        for k in (1, 2, 3):
            f = [I2, I2, I2]
            f[k - 1] = s
            ops[name + str(k)] = np.kron(np.kron(f[0], f[1]), f[2])
    return ops


def site_type(x: int, y: int) -> str:
    """Checkerboard block-site type of the 2x2 cell (Sec. II.B): A when x+y even."""
    return "A" if (x + y) % 2 == 0 else "B"


def ruby_bond_hamiltonians(J):
    """Bond operators (64x64, left/upper site first) of H_R = -sum J_a s^a s^a.

    Each sigma^a sigma^a link of App. A carries -J_a.  Horizontal bond with the
    A site on the left: H_r = h^x_{iA,jB}; with B on the left: H_l = 0 (the
    trivial auxiliary bond).  Vertical bonds: H_u / H_d = (h_A + h_B)/2 + h^y,
    where h_A = h_B = -Jz (z1 z2 + z1 z3 + z2 z3) and h^y couples the upper
    site's spin 3 to the lower site's spin 2 by x and spin 2 to spin 1 by y
    (the same form for A-over-B and B-over-A).
    """
    Jx, Jy, Jz = J
    o = pauli_block_ops()
    I8 = np.eye(8, dtype=np.complex128)
    h_site = -Jz * (o["z1"] @ o["z2"] + o["z1"] @ o["z3"] + o["z2"] @ o["z3"])
    H_r = -Jx * np.kron(o["x1"], o["x1"]) - Jy * np.kron(o["y3"], o["y3"])
    H_l = np.zeros((64, 64), dtype=np.complex128)
    H_v = 0.5 * (np.kron(h_site, I8) + np.kron(I8, h_site)) \
        - Jx * np.kron(o["x3"], o["x2"]) - Jy * np.kron(o["y2"], o["y1"])
    return {"H_r": H_r, "H_l": H_l, "H_u": H_v, "H_d": H_v.copy(), "h_site": h_site}


def xyz_all_edges_bond_hamiltonians(J):
    """Bond operators of the literal reading -sum_edges (Jx xx + Jy yy + Jz zz):
    the links of ``ruby_bond_hamiltonians`` (triangle edges inside a block
    site, spin 1-1 and 3-3 across a horizontal A-B bond, upper 3 - lower 2 and
    upper 2 - lower 1 across a vertical bond), each carrying all three terms
    instead of its own colour's."""
    Jx, Jy, Jz = J
    o = pauli_block_ops()
    I8 = np.eye(8, dtype=np.complex128)

    def link_in(a, b):
        return -sum(Jc * o[f"{al}{a}"] @ o[f"{al}{b}"] for al, Jc in (("x", Jx), ("y", Jy), ("z", Jz)))

    def link_across(a, b):
        return -sum(Jc * np.kron(o[f"{al}{a}"], o[f"{al}{b}"]) for al, Jc in (("x", Jx), ("y", Jy), ("z", Jz)))

    h_site = link_in(1, 2) + link_in(1, 3) + link_in(2, 3)
    H_r = link_across(1, 1) + link_across(3, 3)
    H_l = np.zeros((64, 64), dtype=np.complex128)
    H_v = 0.5 * (np.kron(h_site, I8) + np.kron(I8, h_site)) + link_across(3, 2) + link_across(2, 1)
    return {"H_r": H_r, "H_l": H_l, "H_u": H_v, "H_d": H_v.copy(), "h_site": h_site}


def star_bond_hamiltonians(J):
    """Bond operators of a Heisenberg model on the star lattice (App. B), on
    the same 2x2 cell of triangle block sites: J = (J_t, J_e) couple Pauli
    vectors s.s inside each triangle and between triangles.  Reading of the
    block structure (the figure is absent from the text): spins 1, 2, 3 of a
    triangle link to the left, right and vertical neighbour of the brick wall;
    A sites link down, B sites up, so the vertical bond with B on top is the
    trivial (D = 1) edge and carries no term.  Horizontal bonds (either type on
    the left) hold half of each site's triangle term plus the link of the left
    site's spin 2 to the right site's spin 1; the vertical bond with A on top
    links spin 3 to spin 3."""
    Jt, Je = J
    o = pauli_block_ops()
    I8 = np.eye(8, dtype=np.complex128)

    def dot_in(a, b):
        return sum(o[f"{al}{a}"] @ o[f"{al}{b}"] for al in "xyz")

    def dot_across(a, b):
        return sum(np.kron(o[f"{al}{a}"], o[f"{al}{b}"]) for al in "xyz")

    h_site = Jt * (dot_in(1, 2) + dot_in(1, 3) + dot_in(2, 3))
    H_h = 0.5 * (np.kron(h_site, I8) + np.kron(I8, h_site)) + Je * dot_across(2, 1)
    H_v = Je * dot_across(3, 3)
    return {"H_r": H_h, "H_l": H_h.copy(), "H_u": H_v, "H_d": np.zeros((64, 64), dtype=np.complex128),
            "h_site": h_site}


def energy_per_spin(rdms, J, Lx: int, Ly: int, model: str = "ruby") -> float:
    """(1/(3 Lx Ly)) * sum over the cell's 2 Lx Ly bonds of Re tr(rho_b H_b).

    model: "ruby" (each link its own colour's term, Eq. H-KR),
    "xyz_all_edges" (every link all three terms, for comparison) or "star"
    (the Heisenberg star-lattice model of ``star_bond_hamiltonians``, App. B;
    J = (J_t, J_e))."""
    if model == "ruby":
        H = ruby_bond_hamiltonians(J)
    elif model == "xyz_all_edges":
        H = xyz_all_edges_bond_hamiltonians(J)
    elif model == "star":
        H = star_bond_hamiltonians(J)
    else:
        raise ValueError(model)
    e = 0.0
    for y in range(Ly):
        for x in range(Lx):
            Hh = H["H_r"] if site_type(x, y) == "A" else H["H_l"]
            e += np.real(np.trace(rdms["h"][y, x] @ Hh))
            Hv = H["H_u"] if site_type(x, y) == "A" else H["H_d"]
            e += np.real(np.trace(rdms["v"][y, x] @ Hv))
    return e / (3 * Lx * Ly)


# ---------------------------------------------------------------------------
# Sec. III: fidelity per site.  For a network with environment, the per-cell
# "free energy" kappa = Z(cell) Z(corners) / (Z(columns only) Z(rows only)),
# Eq. (fidelity) written with C1..C4, T (Fig. 4).
# ---------------------------------------------------------------------------
WINDOW = 2  # kappa uses a 2x2 window of sites for every cell (Lx, Ly in {1, 2})


def _window_contract(st: CTMState, with_rows: bool, with_cols: bool) -> complex:
    """Contract the environment of the 2x2 window of sites at (0,0) row by row.

    with_cols: the window's two columns (T1 on top, T3 at the bottom, a's
    inside) are present; with_rows: its two rows (T4 on the left, T2 on the
    right) are present.  The four corners are always present.  Cell indices
    are taken mod (Lx, Ly).  The boundary array B carries axes
    [vl, v_0 .. v_{n-1}, vr] (left bond, column bonds, right bond).
    """
    Lx, Ly = st.Lx, st.Ly
    C, T, a = st.C, st.T, st.a
    n = WINDOW if with_cols else 0
    xr, yb = (WINDOW - 1) % Lx, (WINDOW - 1) % Ly
    B = C[0][0][0]                                   # [vl, ht]
    for x in range(n):
        B = np.tensordot(B, T[0][0][x % Lx], axes=([B.ndim - 1], [0]))  # T1[l,d,r]
    B = np.tensordot(B, C[1][0][xr], axes=([B.ndim - 1], [0]))          # C2[l,d]
    for y in range(WINDOW if with_rows else 0):
        B = np.tensordot(T[3][y % Ly][0], B, axes=([2], [0]))  # T4[d,r,u]: [vl', h, v.., vr]
        for x in range(n):
            B = np.tensordot(B, a[y % Ly][x % Lx], axes=([1 + x, 2 + x], [1, 0]))
            B = np.moveaxis(B, [B.ndim - 2, B.ndim - 1], [1 + x, 2 + x])
        B = np.tensordot(B, T[1][y % Ly][xr], axes=([1 + n, 2 + n], [1, 0]))  # T2[u,l,d]
    B = np.tensordot(C[3][yb][0], B, axes=([1], [0]))    # C4[r,u]: [hb, v.., vr]
    for x in range(n):
        B = np.tensordot(B, T[2][yb][x % Lx], axes=([0, 1], [2, 1]))    # T3[r,u,l]
        B = np.moveaxis(B, B.ndim - 1, 0)
    return complex(np.einsum("hv,vh->", B, C[2][yb][xr]))  # C3[u,l]


def partition_ratios(st: CTMState):
    """(Z_window, Z_00, Z_cols, Z_rows) for the 2x2 window at (0,0)."""
    return (_window_contract(st, True, True), _window_contract(st, False, False),
            _window_contract(st, False, True), _window_contract(st, True, False))


def kappa(st: CTMState) -> complex:
    """kappa of the 2x2 window = Z_window Z_00 / (Z_cols Z_rows): the
    partition function of its four sites per unit of infinite lattice."""
    Zc, Z00, Zcol, Zrow = partition_ratios(st)
    return Zc * Z00 / (Zcol * Zrow)


def fidelity(k12: complex, k11: complex, k22: complex, n_sites: int = WINDOW * WINDOW):
    """Fidelity per block site d = |k12|^(1/n) / (|k11| |k22|)^(1/(2n)) and per
    spin d^(1/3) (three spins per block site)."""
    d_block = np.exp((np.log(abs(k12)) - 0.5 * (np.log(abs(k11)) + np.log(abs(k22)))) / n_sites)
    return float(d_block), float(d_block ** (1.0 / 3.0))


# ---------------------------------------------------------------------------
# Sec. IV: boundary density operator.  sigma_R = ring of N_v tensors T2 at
# column x, sigma_L = ring of N_v tensors T4 at column x+1 (Fig. "cylinder" b),
# both read as D^Nv x D^Nv operators (ket index rows, bra index columns).
# ---------------------------------------------------------------------------
def ring_sigma(st: CTMState, which: str, x: int, Nv: int) -> np.ndarray:
    Lx, Ly, D = st.Lx, st.Ly, st.D
    if Nv % Ly:
        raise ValueError("Nv must be a multiple of the cell height")
    if which == "R":
        ts = [_split(st.T[1][i % Ly][x % Lx], 1, D) for i in range(Nv)]  # [u, k, b, d]
    else:
        ts = [np.transpose(_split(st.T[3][i % Ly][(x + 1) % Lx], 1, D), (3, 1, 2, 0)) for i in range(Nv)]
    R = ts[0]  # [c0, K, B, c1]
    for t in ts[1:]:
        R = np.einsum("aKBc,ckbe->aKkBbe", R, t, optimize=True)
        s = R.shape
        R = R.reshape(s[0], s[1] * s[2], s[3] * s[4], s[5])
    return np.einsum("aKBa->KB", R, optimize=True)


def fixed_rings(st: CTMState, x: int, Nv: int):
    """sigma_L and sigma_R of the cut between columns x and x+1 (rings of T4
    and T2, Fig. "cylinder"), each multiplied by the phase that makes its trace
    real positive and replaced by its Hermitian part."""
    sL = ring_sigma(st, "L", x, Nv)
    sR = ring_sigma(st, "R", x, Nv)
    sL = sL * np.exp(-1j * np.angle(np.trace(sL)))
    sR = sR * np.exp(-1j * np.angle(np.trace(sR)))
    return 0.5 * (sL + sL.conj().T), 0.5 * (sR + sR.conj().T)


def boundary_spectrum_topk(st: CTMState, x: int, Nv: int, k: int):
    """The k largest eigenvalues of M = sigma_L^T sigma_R divided by tr M,
    their entropy -sum lam ln lam and the weight 1 - sum lam they leave out.

    Sec. IV: the spectrum of the boundary density operator is that of
    sigma_L^T sigma_R (the identity after Eq. "rho"); for long cylinders only
    its leading part is computed (iteratively, with the rings as structured
    operators).  Written here as its plain definition: all eigenvalues of the
    dense product (LAPACK), sorted by real part, the k largest kept; tr M is
    the sum of all of them.
    """
    sL, sR = fixed_rings(st, x, Nv)
    M = sL.T @ sR
    ev = np.sort(np.real(np.linalg.eigvals(M)))[::-1]
    lam = ev[:k] / np.real(np.trace(M))
    return lam, entropy(lam), float(1.0 - lam.sum())


def boundary_spectrum(st: CTMState, x: int, Nv: int):
    """Spectrum of sigma_L^T sigma_R normalised to sum 1, descending.

    Computed through the similar operator |sigma_L^T|^(1/2) sigma_R
    |sigma_L^T|^(1/2) (Eq. "rho" and the spectrum identity after it): both
    rings are phase-fixed so their traces are real positive and Hermitised;
    |S|^(1/2) comes from the SVD S = U s V^H as V s^(1/2) V^H; the spectrum is
    the singular values of the resulting Hermitian operator (its eigenvalues
    when it is positive, as for an exact environment).
    """
    sL, sR = fixed_rings(st, x, Nv)
    return spectrum_of_rings(sL, sR)


def spectrum_of_rings(sL: np.ndarray, sR: np.ndarray) -> np.ndarray:
    """The boundary spectrum of ``boundary_spectrum`` for given Hermitian rings.

    Eq. "rho" needs sqrt(sigma_L^T), defined for a positive sigma_L.  A ring
    built from truncated edge tensors can carry small negative eigenvalues;
    the square root used here is that of |sigma_L^T| = (S^H S)^(1/2), which is
    sqrt(sigma_L^T) itself whenever sigma_L^T is positive (so on positive rings
    every route -- eigenvalues of sigma_L^T sigma_R, of the similar operator,
    or these singular values -- gives the same numbers), and which keeps the
    weights non-negative otherwise.
    """
    _, s, Vh = np.linalg.svd(sL.T)
    W = (Vh.conj().T * np.sqrt(s)[None, :]) @ Vh
    H = W @ sR @ W
    lam = np.linalg.svd(H, compute_uv=False)
    return lam / lam.sum()


_LETTERS = "abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ"


def column_transfer_apply(a_col, v: np.ndarray, side: str) -> np.ndarray:
    """The cylinder's column transfer matrix (Sec. IV: sigma_L, sigma_R are its
    dominant left and right eigenvectors) applied to a boundary vector.

    a_col[i] is the double-layer tensor a[u, l, d, r] at row i of the column
    (periodic vertically: the d leg of row Nv-1 meets the u leg of row 0); v
    has one D^2 index per row.  side "R": (E v)(l_1..l_Nv) = sum over r, u of
    prod_i a_i[u_i, l_i, u_{i+1}, r_i] v(r_1..r_Nv); side "L": the same sum
    over l with v(l), leaving r.  Contracted row by row, the open up leg of
    row 0 traced against the last row's down leg at the end
    (``column_transfer_apply_dense`` writes the same sum as one einsum)."""
    Nv = len(a_col)
    D2 = a_col[0].shape[0]
    w = v.reshape(D2, -1)
    w = np.einsum("ulvr,rR->ulvR" if side == "R" else "ulvr,lR->urvR", a_col[0], w)
    for i in range(1, Nv):
        w = w.reshape(D2, D2 ** i, D2, D2, -1)
        w = np.einsum("ALurR,ulvr->ALlvR" if side == "R" else "ALulR,ulvr->ALrvR", w, a_col[i])
    w = w.reshape(D2, D2 ** Nv, D2)
    return np.einsum("ALA->L", w).reshape([D2] * Nv)


def column_transfer_apply_dense(a_col, v: np.ndarray, side: str) -> np.ndarray:
    """``column_transfer_apply`` as a single einsum over the whole ring (for
    small Nv: the check of the row-by-row order)."""
    Nv = len(a_col)
    L = _LETTERS
    u, l, r = L[:Nv], L[Nv:2 * Nv], L[2 * Nv:3 * Nv]
    ops = [f"{u[i]}{l[i]}{u[(i + 1) % Nv]}{r[i]}" for i in range(Nv)]
    vin, vout = (r, l) if side == "R" else (l, r)
    spec = ",".join(ops + [vin]) + "->" + vout
    return np.einsum(spec, *a_col, v, optimize=True)


def _ring_to_vector(S: np.ndarray, D: int, Nv: int) -> np.ndarray:
    """Operator S[(k_1..k_Nv), (b_1..b_Nv)] as a vector over (k_i b_i) per row."""
    t = S.reshape([D] * (2 * Nv))
    perm = [q for i in range(Nv) for q in (i, Nv + i)]
    return np.transpose(t, perm).reshape([D * D] * Nv)


def _vector_to_ring(v: np.ndarray, D: int, Nv: int) -> np.ndarray:
    t = v.reshape([D] * (2 * Nv))
    perm = [2 * i for i in range(Nv)] + [2 * i + 1 for i in range(Nv)]
    n = D ** Nv
    return np.transpose(t, perm).reshape(n, n)


def refined_rings(st: CTMState, x: int, Nv: int, iters: int, tol: float = 0.0):
    """sigma_L and sigma_R of the cut between columns x and x+1 refined beyond
    the ring approximation of Sec. IV: starting from the CTM rings (T4 at
    column x+1, T2 at column x), power iteration with the exact column
    transfer matrices of one cell period (sigma_R <- E_{x+1} ... E_{x+Lx}
    sigma_R, sigma_L <- sigma_L E_{x-Lx+1} ... E_x), each iterate normalised
    and its phase aligned with the previous one, until both change by less
    than tol (Frobenius) or after iters iterations.  Returns (sigma_L,
    sigma_R, iterations, last change) with the rings as D^Nv x D^Nv
    operators."""
    Lx, Ly, D = st.Lx, st.Ly, st.D
    if Nv % Ly:
        raise ValueError("Nv must be a multiple of the cell height")
    col = {c: [st.a[i % Ly][c % Lx] for i in range(Nv)] for c in range(Lx)}
    vs = {"L": _ring_to_vector(ring_sigma(st, "L", x, Nv), D, Nv),
          "R": _ring_to_vector(ring_sigma(st, "R", x, Nv), D, Nv)}
    for k in vs:
        vs[k] = vs[k] / np.linalg.norm(vs[k])
    it, change = 0, np.inf
    while it < iters:
        change = 0.0
        for side in ("L", "R"):
            v = vs[side]
            cols = [(x + c) % Lx for c in range(Lx, 0, -1)] if side == "R" else \
                   [(x - Lx + 1 + c) % Lx for c in range(Lx)]
            for c in cols:
                v = column_transfer_apply(col[c], v, side)
            v = v / np.linalg.norm(v)
            ov = np.vdot(vs[side], v)
            v = v * (np.conj(ov) / abs(ov))
            change = max(change, float(np.linalg.norm(v - vs[side])))
            vs[side] = v
        it += 1
        if change < tol:
            break
    return _vector_to_ring(vs["L"], D, Nv), _vector_to_ring(vs["R"], D, Nv), it, change


def refined_boundary_spectrum(st: CTMState, x: int, Nv: int, iters: int, tol: float = 0.0):
    """The boundary spectrum (as ``boundary_spectrum``) of the refined rings,
    and the iterations and last change of the refinement."""
    sL, sR, it, change = refined_rings(st, x, Nv, iters, tol)
    sL = sL * np.exp(-1j * np.angle(np.trace(sL)))
    sR = sR * np.exp(-1j * np.angle(np.trace(sR)))
    return spectrum_of_rings(0.5 * (sL + sL.conj().T), 0.5 * (sR + sR.conj().T)), it, change


def boundary_renyi2(st: CTMState, x: int, Nv: int):
    """Second Renyi entropy of the boundary density operator of Sec. IV,
    S_2 = -ln sum_i lam_i^2 with lam the eigenvalues of M = sigma_L^T sigma_R
    divided by tr M: written through traces as the purity
    tr(M^2) / (tr M)^2 (real part), which needs no eigenvalues and so is
    available for cylinders whose spectrum is only known in part.
    Returns (S_2, purity)."""
    sL, sR = fixed_rings(st, x, Nv)
    M = sL.T @ sR
    tr = np.trace(M)
    purity = float(np.real(np.trace(M @ M)) / np.real(tr) ** 2)
    return float(-np.log(purity)), purity


def entropy(lam: np.ndarray) -> float:
    """Von Neumann entropy -sum lam ln lam over the positive eigenvalues."""
    p = lam[lam > 0]
    return float(-np.sum(p * np.log(p)))
