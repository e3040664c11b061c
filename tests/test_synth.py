"""The seeded input generator shared by the oracle and the CUDA tests.

SplitMix64 (Steele, Lea & Flood 2014) with state 0 produces the well-known
first outputs below; the counter form used here (state = seed + (n + 1) *
golden gamma) reproduces them, so the stream is the published generator."""
import numpy as np

import synth


def test_splitmix64_published_first_outputs():
    out = synth.splitmix64(0, np.arange(3, dtype=np.uint64))
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform53_exact_and_in_range():
    u = synth.uniform53(5, 10000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert np.all(u * 2.0 ** 53 == np.floor(u * 2.0 ** 53))  # exact multiples of 2^-53
    assert abs(u.mean() - 0.5) < 0.01
    assert np.array_equal(synth.uniform53(5, 4, offset=3), u[3:7])


def test_normal_moments():
    g = synth.normal(9, 200000)
    assert abs(g.mean()) < 0.01 and abs(g.var() - 1.0) < 0.01
    assert abs(np.mean(g ** 4) - 3.0) < 0.05


def test_omega_layout_and_range():
    om = synth.omega(7, 5, 3)
    u = synth.uniform53(7, 30)
    assert np.array_equal(om.real.ravel(), 2.0 * u[0::2] - 1.0)
    assert np.array_equal(om.imag.ravel(), 2.0 * u[1::2] - 1.0)
    assert np.all(np.abs(om.real) <= 1.0) and np.all(np.abs(om.imag) <= 1.0)


def test_workload_recipes():
    w = synth.workload("real", seed=0)
    assert (w["D"], w["chi"], w["J"]) == (2, 16, (1.0, 1.0, 1.0))
    for A in w["tensors"]:
        assert A.shape == (8, 2, 2, 2, 2) and A.dtype == np.float64 and np.max(np.abs(A)) == 1.0
    w = synth.workload("product_noise", seed=1, D=3, chi=9)
    A = w["tensors"][0]
    assert A.shape == (8, 3, 3, 3, 3) and np.iscomplexobj(A)
    noise = A.copy()
    noise[0, 0, 0, 0, 0] -= 1.0
    assert abs(np.mean(np.abs(noise) ** 2) - 0.01) < 0.002  # 0.1 x unit complex normal
    assert w["tensors"][1] is not A and not np.array_equal(w["tensors"][1], A)  # per-tensor streams
    scan = synth.scan(seed=2, n=5, Ds=(2, 3), chis=(9, 12))
    assert [s["J"][2] for s in scan] == [0.0, 0.5, 1.0, 1.5, 2.0]
    assert all(abs(s["J"][0] - (2.0 - s["J"][2]) / 2) < 1e-15 for s in scan)


def test_fidelity_line_ends_are_the_product_noise_recipe():
    """Point 0 of the coupling line is the product-plus-noise state of stream
    seed, the last point that of stream seed + 1 (theta = 0 and pi/2), and
    the points in between keep the all-up entry and the noise norm."""
    seed, D = 4, 2
    line = synth.fidelity_line(seed=seed, n=5, D=D)
    for t in range(4):
        assert np.array_equal(line[0][t], synth.product_plus_noise(seed, t, 8, D))
        assert np.allclose(line[-1][t], synth.product_plus_noise(seed + 1, t, 8, D), rtol=0, atol=1e-16)
    # in between: all-up + eps (cos theta N1 + sin theta N2), N1, N2 the two ends' noise
    n1 = line[0][1] / 0.1
    n2 = line[-1][1] / 0.1
    e0 = np.zeros_like(n1)
    e0[0, 0, 0, 0, 0] = 1.0 / 0.1
    th = 0.5 * np.pi * 2 / 4
    assert np.allclose(line[2][1] / 0.1 - e0, np.cos(th) * (n1 - e0) + np.sin(th) * (n2 - e0), atol=1e-12)
