"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types an oracle formula: each compares the oracle with a
closed form (Onsager's solution of the 2D Ising model, product states), a
brute-force contraction written here independently, or an invariance of the
exact network (gauge, lattice symmetry, the spectrum identity of Sec. IV).
"""
import numpy as np
import pytest
import scipy.integrate as si
import scipy.linalg as sla
import scipy.special as ss

import oracle as O
import synth


# ---------------------------------------------------------------------------
# helpers (independent of the oracle's contraction code)
# ---------------------------------------------------------------------------
def ising_tensor(beta):
    """d=2, D=2 PEPS whose norm network is the classical Ising model at beta:
    A_s[u,l,d,r] = W_su W_sl W_sd W_sr with W = sqrt(B(beta/2)), so each bond of
    the double layer carries B(beta/2)_{ss'}^2 = exp(beta s s')."""
    B = np.array([[np.exp(beta / 2), np.exp(-beta / 2)], [np.exp(-beta / 2), np.exp(beta / 2)]])
    W = np.real(sla.sqrtm(B))
    return np.einsum("pu,pl,pd,pr->puldr", W, W, W, W)


def onsager_minus_beta_f(beta):
    """-beta f per site of the square-lattice Ising model (J = 1), Onsager 1944,
    with the inner angular integral done in closed form."""
    c2, s = np.cosh(2 * beta) ** 2, np.sinh(2 * beta)

    def f(t):
        c = c2 - s * np.cos(t)
        return np.log((c + np.sqrt(c * c - s * s)) / 2)

    val, _ = si.quad(f, 0, 2 * np.pi, epsabs=1e-14, epsrel=1e-14, limit=400)
    return np.log(2) + val / (4 * np.pi)


def onsager_nn_corr(beta):
    """<s_i s_j> on a nearest-neighbour bond, closed form with the complete
    elliptic integral K of modulus k = 2 sinh(2b)/cosh^2(2b)."""
    k = 2 * np.sinh(2 * beta) / np.cosh(2 * beta) ** 2
    return (0.5 + (2 * np.tanh(2 * beta) ** 2 - 1) * ss.ellipk(k * k) / np.pi) / np.tanh(2 * beta)


def random_tensors(seed, n, d, D, cplx=True):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        A = rng.standard_normal((d, D, D, D, D))
        if cplx:
            A = A + 1j * rng.standard_normal((d, D, D, D, D))
        out.append(A / np.abs(A).max())
    return out


def brute_force_rdm(tensors, pattern, xs, ys, open_sites):
    """Reduced density matrix of ``open_sites`` in the finite patch of sites
    xs x ys (ranges), every outer virtual leg traced ket against bra, by plain
    row-by-row contraction of the ket/bra layers (D legs kept separate)."""
    Ly, Lx = len(pattern), len(pattern[0])
    D = tensors[0].shape[1]
    d = tensors[0].shape[0]
    W = len(xs)
    # state axes: [(k_x, b_x) for each column x] + open legs (p, p') in order;
    # the top legs are traced: only k == b survives.
    state = np.ones([D, D] * W)
    for x in range(W):
        state = state * np.eye(D).reshape([1] * (2 * x) + [D, D] + [1] * (2 * (W - x - 1)))
    n_open = 0
    for y in ys:
        # horizontal ket/bra bond entering from the left: traced
        h = np.eye(D)  # axes (k, b)
        cur = np.einsum("...,kb->...kb", state, h)  # [col legs..., open..., hk, hb]
        for ix, x in enumerate(xs):
            A = tensors[pattern[y % Ly][x % Lx]]
            op = (x, y) in open_sites
            # axes of cur: column legs (2W), open legs (2 n_open), hk, hb
            ncol = 2 * W
            nopen = 2 * n_open
            ku, bu = 2 * ix, 2 * ix + 1
            hk, hb = ncol + nopen, ncol + nopen + 1
            if op:
                ket = A
                bra = np.conj(A)
                # contract ket: A[p,u,l,d,r] with (u=ku, l=hk)
                cur = np.tensordot(cur, ket, axes=([ku, hk], [1, 2]))  # appends p, d, r
                # remaining axes shift: remove ku and hk
                bu2 = bu - 1
                hb2 = hb - 2
                cur = np.tensordot(cur, bra, axes=([bu2, hb2], [1, 2]))  # appends p', d', r'
            else:
                # sum_p A conj(A): contract ket with the physical index shared
                cur = np.tensordot(cur, A, axes=([ku, hk], [1, 2]))  # appends p, d, r
                bu2 = bu - 1
                hb2 = hb - 2
                cur = np.tensordot(cur, np.conj(A), axes=([bu2, hb2, cur.ndim - 3], [1, 2, 0]))  # appends d', r'
            # reorder: new column legs (d, d') into position ix, open (p,p') appended, (r, r') last
            nd = cur.ndim
            if op:
                # tail axes: p, d, r, p', d', r'
                p, dk, rk, pb, db, rb = range(nd - 6, nd)
                rest = list(range(nd - 6))
                # rest holds: column legs except ix (2W-2), open legs, nothing else
                cols = rest[:2 * ix] + [dk, db] + rest[2 * ix:2 * W - 2]
                opens = rest[2 * W - 2:] + [p, pb]
                cur = np.transpose(cur, cols + opens + [rk, rb])
            else:
                dk, rk, db, rb = range(nd - 4, nd)
                rest = list(range(nd - 4))
                cols = rest[:2 * ix] + [dk, db] + rest[2 * ix:2 * W - 2]
                opens = rest[2 * W - 2:]
                cur = np.transpose(cur, cols + opens + [rk, rb])
            if op:
                n_open += 1
        # right boundary traced
        state = np.einsum("...kb,kb->...", cur, np.eye(D))
    # bottom legs traced
    for x in range(W):
        state = np.einsum("kb...,kb->...", state, np.eye(D))
    # state axes: open legs in order of appearance (p1, p1', p2, p2', ...)
    rho = state
    if n_open == 2:
        rho = np.transpose(rho, (0, 2, 1, 3)).reshape(d * d, d * d)
    else:
        rho = rho.reshape(d, d)
    return rho / np.trace(rho)


# ---------------------------------------------------------------------------
# a1: double layer (Fig. 3a)
# ---------------------------------------------------------------------------
def test_double_layer_hermitian_and_norm():
    A = random_tensors(1, 1, 3, 2)[0]
    a = O.double_layer(A)
    D = 2
    a8 = a.reshape([D] * 8)  # u u' l l' d d' r r'
    # swapping ket and bra on every leg conjugates a
    assert np.allclose(a8, np.conj(np.transpose(a8, (1, 0, 3, 2, 5, 4, 7, 6))), atol=1e-14)
    # tracing every leg ket against bra gives the squared norm of A
    tr = np.einsum("aabbccdd->", a8)
    assert abs(tr - np.vdot(A, A)) < 1e-12


# ---------------------------------------------------------------------------
# lattice rotation (relabelling only)
# ---------------------------------------------------------------------------
def test_rotation_is_a_relabelling():
    ts = random_tensors(2, 4, 2, 2)
    pat = [[0, 1], [2, 3]]
    st = O.make_state(ts, pat, 2, 8)
    st4 = O.rotate_k(st, 4)
    for j in range(4):
        for y in range(2):
            for x in range(2):
                assert np.array_equal(st4.C[j][y][x], st.C[j][y][x])
                assert np.array_equal(st4.T[j][y][x], st.T[j][y][x])
    # trace initialisation commutes with rotating the tensors themselves
    rot = lambda A: np.transpose(A, (0, 4, 1, 2, 3))
    r1 = O.rotate(st)
    rpat_tensors = [rot(ts[pat[x % 2][(-y) % 2]]) for y in range(2) for x in range(2)]
    rst = O.make_state(rpat_tensors, [[0, 1], [2, 3]], 2, 8)
    for j in range(4):
        for y in range(2):
            for x in range(2):
                assert np.allclose(r1.C[j][y][x], rst.C[j][y][x], atol=1e-14)
                assert np.allclose(r1.T[j][y][x], rst.T[j][y][x], atol=1e-14)


# ---------------------------------------------------------------------------
# Whole CTM + kappa + RDMs on a correlated network: 2D classical Ising model
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("beta", [0.3, 0.6])
def test_ising_free_energy_and_bond_correlation(beta):
    A = ising_tensor(beta)
    st = O.make_state([A], [[0]], 2, 16)
    st, n, _ = O.ctm_converge(st, O.CTMOptions(chi=16, proj="svd", cutoff=1e-12), 1e-9, 80)
    lnk = np.log(abs(O.kappa(st))) / 4  # 2x2 window
    assert abs(lnk - onsager_minus_beta_f(beta)) < 1e-10
    r = O.bond_rdms(st, [A], [[0]])
    zz = np.array([1.0, -1.0, -1.0, 1.0])
    for key in ("h", "v"):
        corr = np.real(np.diag(r[key][0, 0])) @ zz
        assert abs(corr - onsager_nn_corr(beta)) < 1e-9


@pytest.mark.parametrize("beta", [0.5, 0.6])
def test_ising_spontaneous_magnetisation_from_spin_up_boundary(beta):
    """Ordered phase (beta > beta_c = ln(1 + sqrt 2) / 2): an environment
    started from spin-up boundary sites (the user-supplied initial environment)
    converges to the + phase, whose one-site RDM gives Yang's (1952)
    M = (1 - sinh(2 beta)^-4)^(1/8); the symmetric trace initialisation keeps
    the Z2 symmetry and gives M = 0."""
    A = ising_tensor(beta)
    A_up = A.copy()
    A_up[1] = 0.0  # boundary sites fixed to s = +1
    opt = O.CTMOptions(chi=16, proj="svd", cutoff=1e-12)
    st = O.make_state([A], [[0]], 2, 16)
    st.C, st.T = O.trace_init([[O.double_layer(A_up)]], 2, 16)
    st, _, _ = O.ctm_converge(st, opt, 1e-10, 200)
    rho = O.site_rdms(st, [A], [[0]])[0, 0]
    M = np.real(rho[0, 0] - rho[1, 1])
    assert abs(M - (1.0 - np.sinh(2 * beta) ** -4) ** 0.125) < 1e-9
    st0, _, _ = O.ctm_converge(O.make_state([A], [[0]], 2, 16), opt, 1e-10, 200)
    rho0 = O.site_rdms(st0, [A], [[0]])[0, 0]
    assert abs(np.real(rho0[0, 0] - rho0[1, 1])) < 1e-6
    assert opt.ties == []


def test_ising_fidelity_closed_form():
    """Overlap of Ising PEPS at b1 and b2 is the Ising model at (b1+b2)/2, so
    d = Z((b1+b2)/2) / sqrt(Z(b1) Z(b2)) per site (Sec. III with Onsager)."""
    b1, b2 = 0.25, 0.35
    A1, A2 = ising_tensor(b1), ising_tensor(b2)
    opt = O.CTMOptions(chi=16, proj="svd", cutoff=1e-12)
    ks = []
    for ta, tb in ((A1, A2), (A1, A1), (A2, A2)):
        st = O.make_state([ta], [[0]], 2, 16, mixed_with=[tb])
        st, _, _ = O.ctm_converge(st, opt, 1e-9, 80)
        ks.append(O.kappa(st))
    d_block, _ = O.fidelity(ks[0], ks[1], ks[2])
    exact = np.exp(onsager_minus_beta_f((b1 + b2) / 2)
                   - 0.5 * (onsager_minus_beta_f(b1) + onsager_minus_beta_f(b2)))
    assert abs(d_block - exact) < 1e-10


# ---------------------------------------------------------------------------
# D = 1 product states: the environment is exact and everything is closed form
# ---------------------------------------------------------------------------
def product_tensors(seed, n=4, d=8):
    rng = np.random.default_rng(seed)
    phis = [rng.standard_normal(d) + 1j * rng.standard_normal(d) for _ in range(n)]
    return phis, [phi.reshape(d, 1, 1, 1, 1) for phi in phis]


# ruby bonds of one 2x2 cell as (site1, spin1, site2, spin2, alpha), sites given
# as (x, y); written from App. A: triangle z-links inside every block site,
# inter-block x/y links on the right bond of an A site and on vertical bonds.
def ruby_links():
    links = []
    sites = [(0, 0), (1, 0), (0, 1), (1, 1)]
    for s in sites:
        links += [(s, 1, s, 2, "z"), (s, 1, s, 3, "z"), (s, 2, s, 3, "z")]
    for (x, y) in sites:
        t = "A" if (x + y) % 2 == 0 else "B"
        right = ((x + 1) % 2, y)
        below = (x, (y + 1) % 2)
        if t == "A":
            links += [((x, y), 1, right, 1, "x"), ((x, y), 3, right, 3, "y")]
        # vertical: upper spin 3 -- lower spin 2 by x, upper 2 -- lower 1 by y
        links += [((x, y), 3, below, 2, "x"), ((x, y), 2, below, 1, "y")]
    return links


def spin_expect(phi, k, alpha):
    """<phi| sigma^alpha on spin k |phi> / <phi|phi> for a block-site vector."""
    s = {"x": np.array([[0, 1], [1, 0]]), "y": np.array([[0, -1j], [1j, 0]]), "z": np.diag([1, -1])}[alpha]
    psi = phi.reshape(2, 2, 2)
    out = np.tensordot(s, psi, axes=([1], [k - 1]))
    out = np.moveaxis(out, 0, k - 1)
    return np.real(np.vdot(psi, out) / np.vdot(psi, psi))


def pair_expect(phi, k1, k2, alpha):
    """<phi| sigma^alpha_k1 sigma^alpha_k2 |phi> / <phi|phi> inside one block site."""
    s = {"x": np.array([[0, 1], [1, 0]]), "y": np.array([[0, -1j], [1j, 0]]), "z": np.diag([1, -1])}[alpha]
    psi = phi.reshape(2, 2, 2)
    out = psi
    for k in (k1, k2):
        out = np.moveaxis(np.tensordot(s, out, axes=([1], [k - 1])), 0, k - 1)
    return np.real(np.vdot(psi, out) / np.vdot(psi, psi))


def test_product_state_rdm_and_energy_closed_form():
    phis, ts = product_tensors(3)
    pat = [[0, 1], [2, 3]]
    J = (0.7, 1.3, 0.9)
    st = O.make_state(ts, pat, 1, 2)
    opt = O.CTMOptions(chi=2, proj="svd")
    for _ in range(2):
        st = O.sweep(st, opt)
    r = O.bond_rdms(st, ts, pat)
    rho1 = [np.outer(p, p.conj()) / np.vdot(p, p) for p in phis]
    for y in range(2):
        for x in range(2):
            exp_h = np.kron(rho1[pat[y][x]], rho1[pat[y][(x + 1) % 2]])
            exp_v = np.kron(rho1[pat[y][x]], rho1[pat[(y + 1) % 2][x]])
            assert np.allclose(r["h"][y, x], exp_h, atol=1e-13)
            assert np.allclose(r["v"][y, x], exp_v, atol=1e-13)
    e = O.energy_per_spin(r, J, 2, 2)
    Jd = {"x": J[0], "y": J[1], "z": J[2]}
    site_phi = {(x, y): phis[pat[y][x]] for x in range(2) for y in range(2)}
    links = ruby_links()
    assert len(links) == 24  # 12 spins, four-valent lattice
    def term(s1, k1, s2, k2, al):
        if s1 == s2:  # two spins of the same block site
            return pair_expect(site_phi[s1], k1, k2, al)
        return spin_expect(site_phi[s1], k1, al) * spin_expect(site_phi[s2], k2, al)
    e_exact = sum(-Jd[l[4]] * term(*l) for l in links) / 12
    assert abs(e - e_exact) < 1e-13


def test_xyz_all_edges_reading_product_states():
    """The literal all-edges reading: every ruby link carries all three terms;
    checked on D=1 product states against the independent link list."""
    phis, ts = product_tensors(4)
    pat = [[0, 1], [2, 3]]
    J = (0.7, 1.3, 0.9)
    st = O.sweep(O.make_state(ts, pat, 1, 2), O.CTMOptions(chi=2, proj="svd"))
    r = O.bond_rdms(st, ts, pat)
    site_phi = {(x, y): phis[pat[y][x]] for x in range(2) for y in range(2)}

    def term(s1, k1, s2, k2, al):
        if s1 == s2:
            return pair_expect(site_phi[s1], k1, k2, al)
        return spin_expect(site_phi[s1], k1, al) * spin_expect(site_phi[s2], k2, al)

    Jd = {"x": J[0], "y": J[1], "z": J[2]}
    e_exact = sum(-Jd[al] * term(l[0], l[1], l[2], l[3], al) for l in ruby_links() for al in "xyz") / 12
    assert abs(O.energy_per_spin(r, J, 2, 2, model="xyz_all_edges") - e_exact) < 1e-13
    # all spins up: every one of the 24 links gives <zz> = 1
    A = np.zeros((8, 1, 1, 1, 1))
    A[0] = 1.0
    st = O.sweep(O.make_state([A] * 4, pat, 1, 1), O.CTMOptions(chi=1, proj="svd"))
    r = O.bond_rdms(st, [A] * 4, pat)
    assert abs(O.energy_per_spin(r, (0.3, 0.4, 0.37), 2, 2, model="xyz_all_edges") + 2 * 0.37) < 1e-14
    assert abs(O.energy_per_spin(r, (0.3, 0.4, 0.37), 2, 2) + 0.37) < 1e-14


def test_all_up_energy_is_minus_Jz():
    d = 8
    A = np.zeros((d, 1, 1, 1, 1))
    A[0] = 1.0
    st = O.make_state([A] * 4, [[0, 1], [2, 3]], 1, 1)
    st = O.sweep(st, O.CTMOptions(chi=1, proj="svd"))
    r = O.bond_rdms(st, [A] * 4, [[0, 1], [2, 3]])
    assert abs(O.energy_per_spin(r, (1.0, 1.0, 0.37), 2, 2) + 0.37) < 1e-14


def test_product_state_fidelity_closed_form():
    phis1, t1 = product_tensors(5)
    phis2, t2 = product_tensors(6)
    pat = [[0, 1], [2, 3]]
    opt = O.CTMOptions(chi=1, proj="svd")
    ks = []
    for a, b in ((t1, t2), (t1, t1), (t2, t2)):
        st = O.make_state(a, pat, 1, 1, mixed_with=b)
        st = O.sweep(st, opt)
        ks.append(O.kappa(st))
    d_block, d_spin = O.fidelity(*ks)
    ov = [abs(np.vdot(q, p)) / (np.linalg.norm(p) * np.linalg.norm(q)) for p, q in zip(phis1, phis2)]
    exact = np.prod(ov) ** 0.25
    assert abs(d_block - exact) < 1e-13
    assert abs(d_spin - exact ** (1 / 3)) < 1e-13
    st = O.make_state(t1, pat, 1, 1, mixed_with=t1)
    st = O.sweep(st, opt)
    k = O.kappa(st)
    assert abs(O.fidelity(k, k, k)[0] - 1.0) < 1e-14


# ---------------------------------------------------------------------------
# Untruncated moves equal the exact contraction of the finite patch
# ---------------------------------------------------------------------------
def test_trace_init_rdm_equals_bruteforce_patch():
    ts = random_tensors(7, 4, 2, 2)
    pat = [[0, 1], [2, 3]]
    st = O.make_state(ts, pat, 2, 4)
    A_cell = [[ts[pat[y][x]] for x in range(2)] for y in range(2)]
    rho = O.rdm_horizontal(st, A_cell, 0, 0)
    ref = brute_force_rdm(ts, pat, range(-1, 3), range(-1, 2), [(0, 0), (1, 0)])
    assert np.allclose(rho, ref, atol=1e-13)


def test_trace_init_site_rdm_equals_bruteforce_patch():
    """At the trace initialisation the one-site window is the 3x3 open patch."""
    ts = random_tensors(17, 4, 2, 2)
    pat = [[0, 1], [2, 3]]
    st = O.make_state(ts, pat, 2, 4)
    A_cell = [[ts[pat[y][x]] for x in range(2)] for y in range(2)]
    for (x, y) in ((0, 0), (1, 0), (0, 1), (1, 1)):
        rho = O.rdm_site(st, A_cell, x, y)
        ref = brute_force_rdm(ts, pat, range(x - 1, x + 2), range(y - 1, y + 2), [(x, y)])
        assert np.allclose(rho, ref, atol=1e-13), (x, y)


@pytest.mark.parametrize("direction", ["L", "R", "U", "D"])
def test_untruncated_move_site_rdm_equals_bruteforce_patch(direction):
    ts = random_tensors(19, 1, 3, 2)
    st = O.make_state(ts, [[0]], 2, 64)
    st = O.move(st, direction, O.CTMOptions(chi=64, proj="svd", cutoff=1e-14))
    rho = O.rdm_site(st, [[ts[0]]], 0, 0)
    xs = {"L": range(-2, 2), "R": range(-1, 3)}.get(direction, range(-1, 2))
    ys = {"U": range(-2, 2), "D": range(-1, 3)}.get(direction, range(-1, 2))
    ref = brute_force_rdm(ts, [[0]], xs, ys, [(0, 0)])
    assert np.allclose(rho, ref, atol=1e-9)


def test_product_state_site_rdm():
    phis, ts = product_tensors(21)
    pat = [[0, 1], [2, 3]]
    st = O.sweep(O.make_state(ts, pat, 1, 2), O.CTMOptions(chi=2, proj="svd"))
    r = O.site_rdms(st, ts, pat)
    for y in range(2):
        for x in range(2):
            phi = phis[pat[y][x]]
            assert np.allclose(r[y, x], np.outer(phi, phi.conj()) / np.vdot(phi, phi), atol=1e-14)


def test_site_rdm_is_partial_trace_of_bond_rdms_when_converged():
    """At a converged environment the one-site window and the two-site windows
    describe the same state: tracing either site out of a bond RDM gives the
    site RDM (up to the truncation error)."""
    w = synth.workload("product_noise", seed=23, D=2, chi=16)
    st = O.make_state(w["tensors"], w["pattern"], 2, 16)
    opt = O.CTMOptions(chi=16, proj="svd", cutoff=1e-12)
    for _ in range(12):
        st = O.sweep(st, opt)
    rs = O.site_rdms(st, w["tensors"], w["pattern"])
    rb = O.bond_rdms(st, w["tensors"], w["pattern"])
    d = 8
    for y in range(2):
        for x in range(2):
            h = rb["h"][y, x].reshape(d, d, d, d)  # [p q, p' q']
            v = rb["v"][y, x].reshape(d, d, d, d)
            assert np.allclose(np.einsum("pqrq->pr", h), rs[y, x], atol=1e-9)
            assert np.allclose(np.einsum("pqpr->qr", h), rs[y, (x + 1) % 2], atol=1e-9)
            assert np.allclose(np.einsum("pqrq->pr", v), rs[y, x], atol=1e-9)
            assert np.allclose(np.einsum("pqpr->qr", v), rs[(y + 1) % 2, x], atol=1e-9)
            herm = rs[y, x]
            assert np.allclose(herm, herm.conj().T, atol=1e-13)
            assert np.min(np.linalg.eigvalsh(herm)) > -1e-12


def test_untruncated_column_absorption_equals_bruteforce_patch():
    """2x2 cell, four tensors: absorbing column 0 without truncation gives the
    environment of the patch one column wider (bond (1,0)-(2,0))."""
    ts = random_tensors(8, 4, 4, 2)
    pat = [[0, 1], [2, 3]]
    st = O.make_state(ts, pat, 2, 64)
    st = O.left_move(st, O.CTMOptions(chi=64, proj="svd", cutoff=1e-14), columns=[0])
    A_cell = [[ts[pat[y][x]] for x in range(2)] for y in range(2)]
    rho = O.rdm_horizontal(st, A_cell, 1, 0)
    ref = brute_force_rdm(ts, pat, range(-1, 4), range(-1, 2), [(1, 0), (2, 0)])
    assert np.allclose(rho, ref, atol=1e-9)


@pytest.mark.parametrize("corners", [4, 2])
@pytest.mark.parametrize("direction", ["L", "R", "U", "D"])
def test_untruncated_move_equals_bruteforce_patch(direction, corners):
    """1x1 cell: one move in each direction widens the patch on that side
    (four-corner and two-corner projectors alike: untruncated, both exact)."""
    ts = random_tensors(9, 1, 4, 2)
    st = O.make_state(ts, [[0]], 2, 64)
    st = O.move(st, direction, O.CTMOptions(chi=64, proj="svd", cutoff=1e-14, corners=corners))
    rho = O.rdm_horizontal(st, [[ts[0]]], 0, 0)
    xs = {"L": range(-2, 3), "R": range(-1, 4)}.get(direction, range(-1, 3))
    ys = {"U": range(-2, 2), "D": range(-1, 3)}.get(direction, range(-1, 2))
    ref = brute_force_rdm(ts, [[0]], xs, ys, [(0, 0), (1, 0)])
    assert np.allclose(rho, ref, atol=1e-9)


# ---------------------------------------------------------------------------
# Invariances of the exact network
# ---------------------------------------------------------------------------
def random_unitary(rng, n):
    q, r = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    return q * (np.diag(r) / np.abs(np.diag(r)))[None, :]


def test_unitary_gauge_invariance():
    ts = random_tensors(10, 4, 8, 2)
    pat = [[0, 1], [2, 3]]
    rng = np.random.default_rng(11)
    g = [t.copy() for t in ts]
    for y in range(2):
        for x in range(2):
            U = random_unitary(rng, 2)  # bond (x,y) -> (x+1,y)
            L, R = pat[y][x], pat[y][(x + 1) % 2]
            g[L] = np.einsum("puldr,rs->pulds", g[L], U)
            g[R] = np.einsum("sl,puldr->pusdr", U.conj().T, g[R])
            V = random_unitary(rng, 2)  # bond (x,y) -> (x,y+1)
            T_, B_ = pat[y][x], pat[(y + 1) % 2][x]
            g[T_] = np.einsum("puldr,ds->pulsr", g[T_], V)
            g[B_] = np.einsum("su,puldr->psldr", V.conj().T, g[B_])
    opt = O.CTMOptions(chi=12, proj="svd")
    res = []
    for tens in (ts, g):
        st = O.make_state(tens, pat, 2, 12)
        for _ in range(3):
            st = O.sweep(st, opt)
        r = O.bond_rdms(st, tens, pat)
        res.append((O.corner_spectra(st), r, O.energy_per_spin(r, (1, 1, 1), 2, 2)))
    assert np.allclose(res[0][0], res[1][0], atol=1e-10)
    assert np.allclose(res[0][1]["h"], res[1][1]["h"], atol=1e-10)
    assert np.allclose(res[0][1]["v"], res[1][1]["v"], atol=1e-10)
    assert abs(res[0][2] - res[1][2]) < 1e-12


def test_invertible_gauge_energy_gap_shrinks_with_chi():
    """Random invertible (non-unitary) gauges on every bond leave the state
    unchanged but not the truncation: the energies of the two networks agree
    only up to a truncation error that shrinks as chi grows (reported)."""
    w = synth.workload("real", seed=0)
    ts, pat = w["tensors"], w["pattern"]
    rng = np.random.default_rng(5)
    g = [t.copy() for t in ts]
    for y in range(2):
        for x in range(2):
            G = np.eye(2) + 0.3 * rng.standard_normal((2, 2))
            L, R = pat[y][x], pat[y][(x + 1) % 2]
            g[L] = np.einsum("puldr,rs->pulds", g[L], G)
            g[R] = np.einsum("sl,puldr->pusdr", np.linalg.inv(G), g[R])
            G = np.eye(2) + 0.3 * rng.standard_normal((2, 2))
            T_, B_ = pat[y][x], pat[(y + 1) % 2][x]
            g[T_] = np.einsum("puldr,ds->pulsr", g[T_], G)
            g[B_] = np.einsum("su,puldr->psldr", np.linalg.inv(G), g[B_])
    gaps = []
    for chi in (4, 8, 16):
        es = []
        for tens in (ts, g):
            opt = O.CTMOptions(chi=chi, proj="svd", cutoff=1e-12)
            st = O.make_state(tens, pat, 2, chi)
            for _ in range(20):
                st = O.sweep(st, opt)
            es.append(O.energy_per_spin(O.bond_rdms(st, tens, pat), w["J"], 2, 2))
        gaps.append(abs(es[0] - es[1]))
    print("invertible-gauge energy gaps at chi = 4, 8, 16:", gaps)
    assert gaps[0] > gaps[1] > gaps[2]
    assert gaps[2] < 1e-9


def c4v_symmetrize(A):
    rot = lambda t: np.transpose(t, (0, 4, 1, 2, 3))       # (u,l,d,r) -> (r,u,l,d)
    ref = lambda t: np.transpose(t, (0, 1, 4, 3, 2))       # swap l <-> r
    out = np.zeros_like(A)
    t = A
    for _ in range(4):
        out = out + t + ref(t)
        t = rot(t)
    return out / 8


def test_c4v_symmetric_tensor_gives_symmetric_environment():
    A = c4v_symmetrize(random_tensors(12, 1, 2, 2, cplx=False)[0])
    st = O.make_state([A], [[0]], 2, 12)
    opt = O.CTMOptions(chi=12, proj="svd")
    st, _, _ = O.ctm_converge(st, opt, 1e-11, 200)
    s = O.corner_spectra(st)
    nz = s[0, 0, 0] > 1e-8
    for j in range(1, 4):
        assert np.allclose(s[j, 0, 0][nz], s[0, 0, 0][nz], atol=1e-10)
    r = O.bond_rdms(st, [A], [[0]])
    assert np.allclose(r["h"], r["v"], atol=1e-10)


# ---------------------------------------------------------------------------
# Projectors: the randomized range finder is exact once it spans everything,
# and converges to the exact truncated SVD with more subspace iterations.
# ---------------------------------------------------------------------------
def _ring_with_spectrum(s, seed=0):
    """Corners with Q2 = Q3 = Q4 = 1, so the ring X = Q1^T has singular values s."""
    rng = np.random.default_rng(seed)
    n = len(s)
    U, V = random_unitary(rng, n), random_unitary(rng, n)
    X = (U * np.asarray(s)[None, :]) @ V.conj().T
    eye = np.eye(n, dtype=np.complex128)
    return X.T, eye, eye, eye


@pytest.mark.parametrize("proj", ["svd", "rsvd"])
def test_split_multiplet_at_the_cut_is_recorded(proj):
    s = [1.0, 0.5, 0.3, 0.3, 0.1, 0.05]
    Q = _ring_with_spectrum(s)

    def run(chi, cutoff):
        opt = O.CTMOptions(chi=chi, proj=proj, oversample=4, cutoff=cutoff,
                           omega=synth.omega(3, 6, chi + 4))
        P, Pt, sv = O.projectors(*Q, opt)
        assert np.allclose(sv[:len(s)], s, atol=1e-12)
        return opt.ties

    ties = run(3, 1e-8)  # k = chi + 4 >= 6: full span, exact values  # cut between the two 0.3's
    assert len(ties) == 1 and ties[0][0] == 3 and abs(ties[0][1] - 0.3) < 1e-12
    assert run(2, 1e-8) == []  # 0.5 | 0.3: distinct
    assert run(4, 1e-8) == []  # 0.3 | 0.1: distinct
    assert run(3, 0.35) == []  # truncated by the cutoff (keep 2), not by chi


def test_random_parity_recipes_record_no_ties():
    for w, chi in ((synth.workload("real", seed=0), 16),
                   (synth.workload("product_noise", seed=2, D=2, chi=12), 12)):
        D = w["D"]
        opt = O.CTMOptions(chi=chi, omega=synth.omega(7, chi * D * D, chi + 16))
        st = O.make_state(w["tensors"], w["pattern"], D, chi)
        for _ in range(3):
            st = O.sweep(st, opt)
        assert opt.ties == []


def test_two_corner_projectors_approach_the_four_corner_energy():
    """Truncated, the two-corner projectors see less of the environment; the
    energy gap to the four-corner result shrinks as chi grows."""
    w = synth.workload("real", seed=0)
    gaps = []
    for chi in (8, 16, 24):
        es = []
        for corners in (4, 2):
            opt = O.CTMOptions(chi=chi, proj="svd", cutoff=1e-12, corners=corners)
            st = O.make_state(w["tensors"], w["pattern"], 2, chi)
            for _ in range(20):
                st = O.sweep(st, opt)
            es.append(O.energy_per_spin(O.bond_rdms(st, w["tensors"], w["pattern"]), w["J"], 2, 2))
        gaps.append(abs(es[0] - es[1]))
    print("two- vs four-corner energy gaps at chi = 8, 16, 24:", gaps)
    assert gaps[0] > gaps[1] > gaps[2]
    assert gaps[2] < 1e-9
    with pytest.raises(ValueError):
        O.projectors(*(np.eye(2),) * 4, O.CTMOptions(chi=1, proj="svd", corners=3))


def test_energy_converges_with_chi():
    """chi-convergence (reported): on the real iid workload the energy's
    distance to its chi = 24 value shrinks monotonically with chi."""
    w = synth.workload("real", seed=0)
    es = {}
    for chi in (4, 8, 16, 24):
        opt = O.CTMOptions(chi=chi, proj="svd", cutoff=1e-12)
        st = O.make_state(w["tensors"], w["pattern"], 2, chi)
        for _ in range(20):
            st = O.sweep(st, opt)
        es[chi] = O.energy_per_spin(O.bond_rdms(st, w["tensors"], w["pattern"]), w["J"], 2, 2)
    gaps = [abs(es[c] - es[24]) for c in (4, 8, 16)]
    print("E(chi):", es, "gaps to chi=24:", gaps)
    assert gaps[0] > gaps[1] > gaps[2]
    assert gaps[2] < 1e-9


def test_rsvd_full_span_equals_svd():
    ts = random_tensors(13, 4, 8, 2)
    pat = [[0, 1], [2, 3]]
    chi = 4
    K = chi * 4
    es = []
    for proj, over in (("svd", 0), ("rsvd", 16)):
        opt = O.CTMOptions(chi=chi, proj=proj, oversample=over, omega=synth.omega(1, K, chi + over))
        st = O.make_state(ts, pat, 2, chi)
        for _ in range(3):
            st = O.sweep(st, opt)
        es.append(O.energy_per_spin(O.bond_rdms(st, ts, pat), (1, 1, 1), 2, 2))
    assert abs(es[0] - es[1]) < 1e-12


def test_rsvd_converges_to_svd_with_power_iterations():
    rng = np.random.default_rng(4)
    n, k = 120, 30
    U = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))[0]
    V = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))[0]
    s = 0.8 ** np.arange(n)
    X = (U * s) @ V.conj().T
    opt = O.CTMOptions(chi=20, proj="rsvd", oversample=10, power=6, omega=synth.omega(2, n, k))
    Ur, sr, Vr = O.truncated_svd(X, opt)
    assert np.allclose(sr[:20], s[:20], rtol=1e-12)
    # the kept left subspace matches
    Pr = Ur[:, :20] @ Ur[:, :20].conj().T
    Pe = U[:, :20] @ U[:, :20].conj().T
    assert np.linalg.norm(Pr - Pe) < 1e-10


# ---------------------------------------------------------------------------
# Sec. IV: boundary density operator
# ---------------------------------------------------------------------------
def test_spectrum_identity_of_eq_rho():
    """spec(sigma_L^T sigma_R) = spec(sqrt(sigma_L^T) sigma_R sqrt(sigma_L^T))
    for Hermitian positive sigma's (the identity used after Eq. rho)."""
    rng = np.random.default_rng(5)
    n = 16
    G = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    H = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    sL, sR = G @ G.conj().T, H @ H.conj().T
    ev = np.sort(np.real(np.linalg.eigvals(sL.T @ sR)))[::-1]
    w, V = np.linalg.eigh(sL.T)
    Wh = (V * np.sqrt(w)) @ V.conj().T
    ev2 = np.sort(np.linalg.eigvalsh(Wh @ sR @ Wh))[::-1]
    assert np.allclose(ev, ev2, rtol=1e-10)


def test_ring_sigma_at_trace_init_is_column_of_sites():
    ts = random_tensors(14, 4, 2, 2)
    pat = [[0, 1], [2, 3]]
    st = O.make_state(ts, pat, 2, 4)
    D = 2
    # T2[0, y] at trace init = site (1, y) with its right leg traced
    sR = O.ring_sigma(st, "R", 0, 2)
    a = [O.double_layer(ts[pat[y][1]]).reshape(D, D, D, D, D, D, D, D) for y in range(2)]
    # sites (1,0), (1,1) stacked on a periodic column of height 2, right legs traced,
    # left legs open (ket k, bra b); T's are normalised, so compare up to scale.
    ref = np.einsum("aAkKbBrr,bBlLaAss->klKL", a[0], a[1]).reshape(4, 4)
    # st tensors are padded/normalised copies: compare the normalised operators
    assert np.allclose(sR / np.linalg.norm(sR), ref / np.linalg.norm(ref), atol=1e-13)


def _exact_cylinder_spectrum(A):
    """Boundary spectrum of the exact infinite cylinder of circumference 2:
    sigma_L, sigma_R = left / right fixed points of the column transfer matrix
    E[(l0 l1), (r0 r1)] = sum_{u, c} a[u,l0,c,r0] a[c,l1,u,r1] (periodic
    vertical bonds), each reshaped to a (ket..., bra...) operator, phase-fixed
    to a positive trace and Hermitised; eigenvalues of sigma_L^T sigma_R / tr."""
    D = A.shape[1]
    a = O.double_layer(A)
    E = np.einsum("alcr,cmas->lmrs", a, a).reshape(D ** 4, D ** 4)
    ops = []
    for M in (E.T, E):  # left fixed point: eigenvector of E^T
        w, V = np.linalg.eig(M)
        v = V[:, np.argmax(np.abs(w))].reshape(D, D, D, D)  # k0 b0 k1 b1
        m = np.transpose(v, (0, 2, 1, 3)).reshape(D * D, D * D)
        m = m * np.exp(-1j * np.angle(np.trace(m)))
        ops.append(0.5 * (m + m.conj().T))
    sL, sR = ops
    M = sL.T @ sR
    return np.sort(np.real(np.linalg.eigvals(M)))[::-1] / np.real(np.trace(M))


@pytest.mark.parametrize("case", ["ising_0.3", "random_complex"])
def test_ctm_ring_approximates_the_exact_cylinder(case):
    """Sec. IV approximates the cylinder's boundary operators by rings of the
    converged half-plane edge tensors; on a circumference-2 cylinder the
    exact ones come from the column transfer matrix.  Sanity tolerances: the
    approximation is close where the correlation length is short."""
    A = ising_tensor(0.3) if case == "ising_0.3" else random_tensors(4, 1, 2, 2)[0]
    lam_x = _exact_cylinder_spectrum(A)
    st = O.make_state([A], [[0]], 2, 16)
    st, _, _ = O.ctm_converge(st, O.CTMOptions(chi=16, proj="svd", cutoff=1e-12), 1e-10, 200)
    lam_c = O.boundary_spectrum(st, 0, 2)
    S_x, S_c = O.entropy(lam_x[lam_x > 0]), O.entropy(lam_c)
    print(case, "exact", lam_x, "ring", lam_c, "S", S_x, S_c)
    if case == "ising_0.3":
        assert np.max(np.abs(lam_c - lam_x)) < 1e-5 and abs(S_c - S_x) < 1e-4
    else:
        assert abs(S_c - S_x) < 0.02 * S_x


def test_product_state_boundary_entropy_is_zero():
    _, ts = product_tensors(15)
    pat = [[0, 1], [2, 3]]
    st = O.make_state(ts, pat, 1, 1)
    st = O.sweep(st, O.CTMOptions(chi=1, proj="svd"))
    lam = O.boundary_spectrum(st, 0, 2)
    assert np.allclose(lam, [1.0]) and abs(O.entropy(lam)) < 1e-15


def _converged_state(seed, D, chi, sweeps):
    w = synth.workload("product_noise", seed=seed, D=D, chi=chi)
    st = O.make_state(w["tensors"], w["pattern"], D, chi)
    opt = O.CTMOptions(chi=chi, proj="rsvd", omega=synth.omega(7, chi * D * D, chi + 16))
    for _ in range(sweeps):
        st = O.sweep(st, opt)
    return st


def test_topk_boundary_spectrum_equals_similar_operator_spectrum():
    """The leading eigenvalues of sigma_L^T sigma_R (eig of the product) equal
    the leading eigenvalues of |sigma_L^T|^(1/2) sigma_R |sigma_L^T|^(1/2)
    (SVD route) when both rings are positive, as they are here."""
    st = _converged_state(2, 2, 12, 6)
    for Nv in (2, 4):
        sL, sR = O.fixed_rings(st, 0, Nv)
        assert np.linalg.eigvalsh(sL).min() > 0 and np.linalg.eigvalsh(sR).min() > 0
        full = O.boundary_spectrum(st, 0, Nv)
        n = len(full)
        lam, S, rest = O.boundary_spectrum_topk(st, 0, Nv, n)
        assert np.allclose(lam, full, rtol=1e-10, atol=1e-14) and abs(rest) < 1e-12
        assert abs(S - O.entropy(full)) < 1e-10
        k = n // 3
        lk, Sk, restk = O.boundary_spectrum_topk(st, 0, Nv, k)
        assert np.allclose(lk, full[:k], rtol=1e-10)
        assert abs(restk - full[k:].sum()) < 1e-10
        assert 0 < Sk < O.entropy(full)


def test_topk_product_state_single_eigenvalue():
    _, ts = product_tensors(15)
    pat = [[0, 1], [2, 3]]
    st = O.make_state(ts, pat, 1, 1)
    st = O.sweep(st, O.CTMOptions(chi=1, proj="svd"))
    lam, S, rest = O.boundary_spectrum_topk(st, 0, 2, 1)
    assert np.allclose(lam, [1.0]) and abs(S) < 1e-15 and abs(rest) < 1e-14


@pytest.mark.parametrize("build", ["ruby_bond_hamiltonians", "xyz_all_edges_bond_hamiltonians"])
def test_hamiltonian_terms_hermitian_and_trivial_bond(build):
    H = getattr(O, build)((0.3, 0.5, 0.7))
    for k in ("H_r", "H_u", "H_d"):
        assert np.allclose(H[k], H[k].conj().T)
    assert not np.any(H["H_l"])
    # each Pauli-product term is traceless: trace of every bond operator vanishes
    for k in ("H_r", "H_u", "H_d"):
        assert abs(np.trace(H[k])) < 1e-12


def _exact_cylinder_rings(A):
    """sigma_L, sigma_R of the exact circumference-2 cylinder (fixed points of
    the column transfer matrix, as in _exact_cylinder_spectrum)."""
    D = A.shape[1]
    a = O.double_layer(A)
    E = np.einsum("alcr,cmas->lmrs", a, a).reshape(D ** 4, D ** 4)
    ops = []
    for M in (E.T, E):
        w, V = np.linalg.eig(M)
        v = V[:, np.argmax(np.abs(w))].reshape(D, D, D, D)
        m = np.transpose(v, (0, 2, 1, 3)).reshape(D * D, D * D)
        m = m * np.exp(-1j * np.angle(np.trace(m)))
        ops.append(0.5 * (m + m.conj().T))
    return ops


def test_boundary_spectrum_route_on_positive_rings():
    """Eq. "rho": on positive rings (the exact cylinder's fixed points are
    positive: they are reduced density operators of the virtual space) the
    oracle's route -- singular values of |sigma_L^T|^(1/2) sigma_R
    |sigma_L^T|^(1/2) -- gives the eigenvalues of sigma_L^T sigma_R, the
    quantity Sec. IV diagonalises, and the eigenvalues of the similar operator
    built from the positive square root."""
    for A in (ising_tensor(0.3), ising_tensor(0.5)):
        sL, sR = _exact_cylinder_rings(A)
        assert np.linalg.eigvalsh(sL).min() > -1e-14 and np.linalg.eigvalsh(sR).min() > -1e-14
        lam = O.spectrum_of_rings(sL, sR)
        M = sL.T @ sR
        ev = np.sort(np.real(np.linalg.eigvals(M)))[::-1] / np.real(np.trace(M))
        w, V = np.linalg.eigh(sL.T)
        Wh = (V * np.sqrt(np.clip(w, 0, None))) @ V.conj().T
        ev2 = np.sort(np.linalg.eigvalsh(Wh @ sR @ Wh))[::-1]
        ev2 = ev2 / ev2.sum()
        assert np.allclose(lam, ev, atol=1e-12) and np.allclose(lam, ev2, atol=1e-12)
        assert np.allclose(lam, _exact_cylinder_spectrum(A), atol=1e-12)


def test_boundary_spectrum_route_on_an_indefinite_ring():
    """Where a ring has a negative eigenvalue (possible for rings of truncated
    edge tensors) sqrt(sigma_L^T) is undefined; the oracle's |sigma_L^T|^(1/2)
    keeps every weight non-negative and summing to one, and it differs from
    dropping the negative part (clamping), which changes the operator: the
    two routes are told apart here."""
    rng = np.random.default_rng(8)
    n = 6
    U, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    sL = (U * np.array([1.0, 0.5, 0.3, 0.2, 0.1, -0.05])) @ U.conj().T
    G = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    sR = G @ G.conj().T
    lam = O.spectrum_of_rings(sL, sR)
    assert lam.min() >= 0 and abs(lam.sum() - 1) < 1e-14
    w, V = np.linalg.eig(sL.T)
    absL = (V * np.sqrt(np.abs(w))) @ np.linalg.inv(V)  # |sigma_L^T|^(1/2) by eigenvectors
    ref = np.linalg.svd(absL @ sR @ absL, compute_uv=False)
    assert np.allclose(lam, ref / ref.sum(), atol=1e-12)
    wh, Vh = np.linalg.eigh(sL.T)
    clamp = (Vh * np.sqrt(np.clip(wh, 0, None))) @ Vh.conj().T
    ev_c = np.sort(np.linalg.eigvalsh(clamp @ sR @ clamp))[::-1]
    assert np.max(np.abs(lam - ev_c / ev_c.sum())) > 1e-3


def test_boundary_renyi2_equals_the_spectrum_purity():
    """S_2 from traces equals -ln sum lam^2 of the boundary spectrum (Sec. IV)
    on positive rings of a converged environment, and vanishes for a product
    state (D = 1)."""
    st = _converged_state(2, 2, 12, 6)
    for Nv in (2, 4):
        lam = O.boundary_spectrum(st, 0, Nv)
        S2, p = O.boundary_renyi2(st, 0, Nv)
        assert abs(p - np.sum(lam ** 2)) < 1e-12 and abs(S2 + np.log(np.sum(lam ** 2))) < 1e-10
        assert 0 < S2 <= O.entropy(lam) + 1e-12  # Renyi-2 never exceeds von Neumann
    _, ts = product_tensors(15)
    pst = O.sweep(O.make_state(ts, [[0, 1], [2, 3]], 1, 1), O.CTMOptions(chi=1, proj="svd"))
    S2, p = O.boundary_renyi2(pst, 0, 2)
    assert abs(S2) < 1e-14 and abs(p - 1) < 1e-14


# ---------------------------------------------------------------------------
# App. B: star lattice on the same block-site engine
# ---------------------------------------------------------------------------
def _star_link_energy(phis, Jt, Je):
    """Energy per spin of a product of block-site states phi (8-vectors at
    pattern [[0, 1], [2, 3]]) from an explicit list of the star lattice's
    links in the cell: the three triangle edges of every site, the two
    horizontal links per row (left site's spin 2 to right site's spin 1) and
    the vertical links below the A sites (spin 3 to spin 3)."""
    o = O.pauli_block_ops()

    def ev(phi, op):
        return np.vdot(phi, op @ phi).real / np.vdot(phi, phi).real

    def spin(phi, k):
        return np.array([ev(phi, o[f"{al}{k}"]) for al in "xyz"])

    pat = [[0, 1], [2, 3]]
    e = 0.0
    for y in range(2):
        for x in range(2):
            p = phis[pat[y][x]]
            e += Jt * sum(ev(p, sum(o[f"{al}{a}"] @ o[f"{al}{b}"] for al in "xyz"))
                          for a, b in ((1, 2), (1, 3), (2, 3)))
            right = phis[pat[y][(x + 1) % 2]]
            e += Je * spin(p, 2) @ spin(right, 1)
            if (x + y) % 2 == 0:  # A site: its link goes down
                below = phis[pat[(y + 1) % 2][x]]
                e += Je * spin(p, 3) @ spin(below, 3)
    return e / 12.0


def test_star_hamiltonian_terms():
    H = O.star_bond_hamiltonians((0.7, 0.4))
    for k in ("H_r", "H_l", "H_u"):
        assert np.allclose(H[k], H[k].conj().T)
    assert not np.any(H["H_d"])  # the trivial edge carries no term


def test_star_product_states_closed_forms():
    """D = 1 products: the CTM energy equals the link-list energy; the all-up
    state gives J_t + J_e/2 per spin; a triangle in its total-spin-1/2 ground
    space with J_e = 0 gives -J_t (sum_{i<j} s_i.s_j = 2 S(S+1) - 9/2 = -3 per
    triangle)."""
    rng = np.random.default_rng(17)
    Jt, Je = 0.8, 0.35
    phis = [rng.standard_normal(8) + 1j * rng.standard_normal(8) for _ in range(4)]
    ts = [p.reshape(8, 1, 1, 1, 1) for p in phis]
    pat = [[0, 1], [2, 3]]
    st = O.sweep(O.make_state(ts, pat, 1, 1), O.CTMOptions(chi=1, proj="svd"))
    e = O.energy_per_spin(O.bond_rdms(st, ts, pat), (Jt, Je), 2, 2, model="star")
    assert abs(e - _star_link_energy(phis, Jt, Je)) < 1e-13
    up = np.zeros(8)
    up[0] = 1.0
    st = O.sweep(O.make_state([up.reshape(8, 1, 1, 1, 1)] * 4, pat, 1, 1), O.CTMOptions(chi=1, proj="svd"))
    e_up = O.energy_per_spin(O.bond_rdms(st, [up.reshape(8, 1, 1, 1, 1)] * 4, pat), (Jt, Je), 2, 2, model="star")
    assert abs(e_up - (Jt + Je / 2)) < 1e-14
    h = O.star_bond_hamiltonians((1.0, 0.0))["h_site"]
    w, V = np.linalg.eigh(h)
    assert abs(w[0] + 3.0) < 1e-12 and np.sum(np.abs(w + 3.0) < 1e-9) == 4  # S = 1/2 twice
    gs = [V[:, 0].reshape(8, 1, 1, 1, 1)] * 4
    st = O.sweep(O.make_state(gs, pat, 1, 1), O.CTMOptions(chi=1, proj="svd"))
    e_gs = O.energy_per_spin(O.bond_rdms(st, gs, pat), (Jt, 0.0), 2, 2, model="star")
    assert abs(e_gs + Jt) < 1e-13


def test_star_tensors_trivial_legs():
    """synth.star_tensors: the empty edge of each block site has dimension 1
    (u for A sites, d for B sites), the product-state entry sits at index 0."""
    ts = synth.star_tensors(seed=2, D=3)
    assert [t.shape for t in ts] == [(8, 1, 3, 3, 3), (8, 3, 3, 1, 3), (8, 3, 3, 1, 3), (8, 1, 3, 3, 3)]
    for t in ts:
        assert abs(t[0, 0, 0, 0, 0] - 1.0) < 0.5


def test_refined_rings_reach_the_exact_cylinder():
    """Sec. IV: sigma_L, sigma_R are the dominant eigenvectors of the column
    transfer matrix.  Power iteration with the exact transfer matrix, started
    from the CTM rings, reaches the fixed points that a dense eigensolver of
    that matrix gives on the circumference-2 cylinder (Ising beta = 0.3 and a
    random complex tensor): the refined spectrum equals the exact one to
    1e-10, where the plain ring approximation was off by up to 3e-6."""
    for A in (ising_tensor(0.3), random_tensors(4, 1, 2, 2)[0]):
        lam_x = _exact_cylinder_spectrum(A)
        st = O.make_state([A], [[0]], 2, 16)
        st, _, _ = O.ctm_converge(st, O.CTMOptions(chi=16, proj="svd", cutoff=1e-12), 1e-10, 200)
        lam_r, it, change = O.refined_boundary_spectrum(st, 0, 2, 400, tol=1e-13)
        print("refined", it, change, np.max(np.abs(lam_r - lam_x)))
        assert change < 1e-12 and np.max(np.abs(lam_r - lam_x)) < 1e-10


def test_refined_rings_are_eigenvectors_of_the_transfer_matrix():
    """On a 2x2 cell (two columns per period) the refined rings satisfy the
    eigen-equations of the one-period transfer matrix E_{x+1} E_{x+2} to the
    iteration's tolerance, at circumference 2 and 4."""
    st = _converged_state(2, 2, 12, 6)
    D = st.D
    for Nv in (2, 4):
        sL, sR, it, change = O.refined_rings(st, 0, Nv, 500, tol=1e-12)
        assert change < 1e-12, (Nv, it, change)
        col = {c: [st.a[i % 2][c] for i in range(Nv)] for c in range(2)}
        vR = O.readout._ring_to_vector(sR, D, Nv)
        wR = O.column_transfer_apply(col[1], O.column_transfer_apply(col[0], vR, "R"), "R")
        lamR = np.vdot(vR, wR) / np.vdot(vR, vR)
        assert np.linalg.norm(wR - lamR * vR) < 1e-10 * np.linalg.norm(wR)
        vL = O.readout._ring_to_vector(sL, D, Nv)
        wL = O.column_transfer_apply(col[0], O.column_transfer_apply(col[1], vL, "L"), "L")
        lamL = np.vdot(vL, wL) / np.vdot(vL, vL)
        assert np.linalg.norm(wL - lamL * vL) < 1e-10 * np.linalg.norm(wL)
        assert abs(lamL - lamR) < 1e-10 * abs(lamR)  # one dominant eigenvalue, left and right


def test_column_transfer_row_by_row_equals_the_ring_einsum():
    """The row-by-row contraction of the column transfer matrix equals the
    single einsum over the ring (both sides, circumference 2 and 4, two
    different tensors in the column)."""
    rng = np.random.default_rng(44)
    D2 = 4
    for Nv in (2, 4):
        a = [rng.standard_normal((D2,) * 4) + 1j * rng.standard_normal((D2,) * 4) for _ in range(2)]
        col = [a[i % 2] for i in range(Nv)]
        v = rng.standard_normal([D2] * Nv) + 1j * rng.standard_normal([D2] * Nv)
        for side in ("L", "R"):
            x = O.column_transfer_apply(col, v, side)
            y = O.readout.column_transfer_apply_dense(col, v, side)
            assert np.allclose(x, y, rtol=1e-12, atol=1e-12 * np.abs(y).max())
