"""A CPU model of the precision form's rounding.

The BF16x3 path splits every operand x into bf16 parts hi = bf16(x) and
lo = bf16(x - hi), forms hi*hi + hi*lo + lo*hi and accumulates in FP32.  Here
that arithmetic is emulated in numpy (bf16 by round-to-nearest-even on the top
16 bits of an FP32 word, products summed in complex64 so the accumulation is
FP32) and substituted into the oracle's own pairwise contractions: the moves
(enlarged corners, absorption, the ring matrix) and/or the readouts (RDM
contractions), while orthonormalisation, SVDs and normalisation stay FP64.

The oracle's contraction sequence is not the GPU's (the GPU never forms the
ring matrix and sends small products to its FP64 GEMM), so the model sizes the
arithmetic's effect rather than reproducing the GPU's error budget: at the GPU
precision test's workload (D = 3, chi = 18, six sweeps, cutoff 1e-8) it gives
|dE| 1.1e-6 for BF16x3 where the GB300 measured 1.1e-6, but overestimates the
TF32 path's error by tens.  What it does establish is a property of the
arithmetic: BF16x3's error comes from its two-part split (16 significand
bits), not from FP32 accumulation, and a three-way split cuts it about ten
times.  The oracle itself is unchanged (the substitution is undone after each
run)."""
import functools
import types

import numpy as np

import oracle as O
import oracle.ctm as OC
import oracle.readout as OR
import synth
from gpu_common import oracle_options


def bf16(x):
    """Round FP32 values to bfloat16 (nearest, ties to even), returned as FP32."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32)
    u = (u + (((u >> 16) & 1) + 0x7FFF)) & np.uint32(0xFFFF0000)
    return u.view(np.float32)


def _split(a):
    re, im = np.real(a).astype(np.float64), np.imag(a).astype(np.float64)
    hr, hi = bf16(re.astype(np.float32)), bf16(im.astype(np.float32))
    lr, li = bf16((re - hr).astype(np.float32)), bf16((im - hi).astype(np.float32))
    return (hr + 1j * hi).astype(np.complex64), (lr + 1j * li).astype(np.complex64)


def _bf16x3_einsum(spec, *ops, **kw):
    if len(ops) != 2:
        return np.einsum(spec, *ops, **kw)
    (ah, al), (bh, bl) = _split(np.asarray(ops[0])), _split(np.asarray(ops[1]))
    r = (np.einsum(spec, ah, bh, optimize=True) + np.einsum(spec, ah, bl, optimize=True)
         + np.einsum(spec, al, bh, optimize=True))
    return r.astype(np.complex128)


def _bf16x3_fp64_accumulate_einsum(spec, *ops, **kw):
    """The same three bf16 products, summed exactly (FP64) instead of in FP32."""
    if len(ops) != 2:
        return np.einsum(spec, *ops, **kw)
    (ah, al), (bh, bl) = _split(np.asarray(ops[0])), _split(np.asarray(ops[1]))
    c = lambda t: t.astype(np.complex128)
    return sum(np.einsum(spec, c(x), c(y), optimize=True) for x, y in ((ah, bh), (ah, bl), (al, bh)))


def _split3(a):
    """Three bf16 parts x = p0 + p1 + p2 + O(2^-24 |x|) (24 significand bits)."""
    re, im = np.real(a).astype(np.float64), np.imag(a).astype(np.float64)
    parts = []
    for _ in range(3):
        pr, pi = bf16(re.astype(np.float32)), bf16(im.astype(np.float32))
        parts.append((pr + 1j * pi).astype(np.complex64))
        re, im = re - pr, im - pi
    return parts


def _bf16x6_einsum(spec, *ops, **kw):
    """Three-way split, the six products p_i q_j with i + j <= 2, FP32 accumulation."""
    if len(ops) != 2:
        return np.einsum(spec, *ops, **kw)
    A, B = _split3(np.asarray(ops[0])), _split3(np.asarray(ops[1]))
    r = sum(np.einsum(spec, A[i], B[j], optimize=True) for i in range(3) for j in range(3) if i + j <= 2)
    return r.astype(np.complex128)


class _Numpy(types.ModuleType):
    """numpy with einsum replaced by an emulated product."""

    def __getattr__(self, name):
        return getattr(np, name)


def _numpy_with(einsum):
    m = _Numpy("numpy_emulated")
    m.einsum = einsum
    return m


def _ring_with(einsum):
    def ring(Q1, Q2, Q3, Q4):
        R_up = einsum("ij,jk->ik", Q1, Q2)
        R_dn = einsum("ij,kj->ik", Q4, Q3)
        return R_up, R_dn, einsum("ji,jk->ik", R_up, R_dn)
    return ring


def _sweeps_and_readouts():
    """Six sweeps at D = 3, chi = 18, then site RDMs and the energy."""
    w = synth.workload("product_noise", seed=2, D=3, chi=18)
    opt = oracle_options(18, 3, cutoff=1e-8)
    st = O.make_state(w["tensors"], w["pattern"], 3, 18)
    for _ in range(6):
        st = O.sweep(st, opt)
    rs = O.site_rdms(st, w["tensors"], w["pattern"])
    return rs, O.energy_per_spin(O.bond_rdms(st, w["tensors"], w["pattern"]), w["J"], 2, 2)


@functools.lru_cache(maxsize=1)
def _exact():
    """The plain FP64 oracle (computed once)."""
    return _sweeps_and_readouts()


def _run(monkeypatch, moves, readouts, einsum=_bf16x3_einsum):
    """The same run with `einsum` in the moves and/or the readout contractions."""
    with monkeypatch.context() as m:
        if moves:
            m.setattr(OC, "np", _numpy_with(einsum))
            m.setattr(OC, "ring_matrix_factors", _ring_with(einsum))
        if readouts:
            m.setattr(OR, "np", _numpy_with(einsum))
        return _sweeps_and_readouts()


def test_bf16_rounding():
    one = np.float32(1.0)
    assert bf16(one) == one
    assert bf16(np.float32(1 + 2 ** -8)) == one                       # tie -> even
    assert bf16(np.float32(1 + 3 * 2 ** -9)) == np.float32(1 + 2 ** -7)
    assert bf16(np.float32(-2.5)) == np.float32(-2.5)
    x = np.float32(0.1234567)
    assert abs(float(bf16(x)) - float(x)) <= 2 ** -9 * abs(float(x))


def test_bf16x3_rounding_in_moves_and_readouts(monkeypatch):
    rs0, e0 = _exact()
    rs_all, e_all = _run(monkeypatch, True, True)
    rs_ro, e_ro = _run(monkeypatch, False, True)
    err_all, err_ro = np.max(np.abs(rs_all - rs0)), np.max(np.abs(rs_ro - rs0))
    print(f"emulated BF16x3 everywhere: |dE| {abs(e_all - e0):.2e}, site RDM {err_all:.2e}; "
          f"readouts only: |dE| {abs(e_ro - e0):.2e}, site RDM {err_ro:.2e}")
    # the size the GB300 measured (1.1e-6 / 6.8e-6) is of this order
    assert 3e-7 < abs(e_all - e0) < 3e-6
    assert 1e-6 < err_all < 2e-5
    # the readout contractions alone exceed 1e-6 in RDM elements but not in energy
    assert 5e-7 < err_ro < 1e-5 and abs(e_ro - e0) < abs(e_all - e0)
    # the oracle is back to plain FP64
    assert OC.np is np and OR.np is np and OC.ring_matrix_factors is O.ring_matrix_factors


def test_bf16x3_is_limited_by_its_split_not_by_accumulation(monkeypatch):
    """hi + lo keeps 16 significand bits, so summing the three products exactly
    does not help; a three-way split (24 bits) with six products reaches the
    1e-6 RDM target at twice the tensor-core work of BF16x3."""
    rs0, e0 = _exact()
    rs3, e3 = _run(monkeypatch, True, True)
    rs_acc, e_acc = _run(monkeypatch, True, True, _bf16x3_fp64_accumulate_einsum)
    rs6, e6 = _run(monkeypatch, True, True, _bf16x6_einsum)
    d3, d_acc, d6 = (np.max(np.abs(r - rs0)) for r in (rs3, rs_acc, rs6))
    print(f"site RDM error: BF16x3 {d3:.2e}, exact accumulation {d_acc:.2e}, three-way split {d6:.2e}; "
          f"|dE| {abs(e3 - e0):.2e}, {abs(e_acc - e0):.2e}, {abs(e6 - e0):.2e}")
    assert d_acc > 0.5 * d3
    assert d6 < 1e-6 and d6 < 0.2 * d3 and abs(e6 - e0) < 0.2 * abs(e3 - e0)
