"""CPU-only checks of the C ABI: the library builds, loads, exports every
symbol declared in include/ipeps_ctm.h, and validates arguments before any
CUDA call."""
import ctypes
import os
import re
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ipeps_ctm.h")).read()
    return sorted(set(re.findall(r"\b(ipeps_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1711_04798_gb300 import build
    path = build.LIB
    if not os.path.exists(path):
        build.build()
    from paper_1711_04798_gb300 import load_library
    return load_library()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_argument_validation_without_gpu(lib):
    from paper_1711_04798_gb300.binding import Cell, Options
    cell = Cell()
    cell.Lx = cell.Ly = 2
    for i in range(4):
        cell.pattern[i] = i
    cell.n_tensors, cell.d, cell.D, cell.dtype = 4, 8, 4, 1
    ptrs = (ctypes.c_void_p * 4)(1, 1, 1, 1)
    cell.tensors = ctypes.cast(ptrs, ctypes.POINTER(ctypes.c_void_p))
    opt = Options()
    lib.ipeps_default_options(ctypes.byref(opt))
    assert opt.svd_cutoff == 0.0 and opt.rsvd_oversample == 16  # 0: chosen by precision
    opt.chi = 8  # < D^2 = 16
    n = ctypes.c_size_t()
    assert lib.ipeps_ctm_workspace_size(ctypes.byref(cell), ctypes.byref(opt), ctypes.byref(n)) == 1
    assert b"chi" in lib.ipeps_last_error()
    opt.chi = 64
    assert lib.ipeps_ctm_workspace_size(ctypes.byref(cell), ctypes.byref(opt), ctypes.byref(n)) == 0
    assert n.value > 64 * 16 * 64 * 16 * 16  # at least the four enlarged corners
    cell.pattern[3] = 7
    h = ctypes.c_void_p()
    assert lib.ipeps_ctm_create(ctypes.byref(cell), ctypes.byref(opt), ctypes.byref(h)) == 1


def _good(lib):
    """A valid 2x2, d=8, D=4, chi=64 cell (fake non-null tensor pointers)."""
    from paper_1711_04798_gb300.binding import Cell, Options
    cell = Cell()
    cell.Lx = cell.Ly = 2
    for i in range(4):
        cell.pattern[i] = i
    cell.n_tensors, cell.d, cell.D, cell.dtype = 4, 8, 4, 1
    ptrs = (ctypes.c_void_p * 4)(1, 1, 1, 1)
    cell.tensors = ctypes.cast(ptrs, ctypes.POINTER(ctypes.c_void_p))
    opt = Options()
    lib.ipeps_default_options(ctypes.byref(opt))
    opt.chi = 64
    return cell, opt, ptrs


_BAD_LEGS = (ctypes.c_int * 16)(*([4] * 7 + [2] + [4] * 8))  # leg 7 (tensor 1, r) neither 1 nor D


def _set(obj, field, value):
    if field == "pattern":
        obj.pattern[2] = value
    elif field == "tensors":
        obj.tensors = None
    elif field == "leg_dims":
        obj.leg_dims = ctypes.cast(_BAD_LEGS, ctypes.POINTER(ctypes.c_int))
    else:
        setattr(obj, field, value)


# (target, field, value, fragment of the error message)
_RULES = [
    ("cell", "Lx", 0, b"Lx"), ("cell", "Lx", 3, b"Lx"), ("cell", "Ly", 0, b"Ly"),
    ("cell", "n_tensors", 0, b"n_tensors"), ("cell", "n_tensors", 5, b"n_tensors"),
    ("cell", "pattern", 4, b"pattern"), ("cell", "pattern", -1, b"pattern"),
    ("cell", "d", 0, b"d in"), ("cell", "d", 65, b"d in"), ("cell", "D", 13, b"D in"),
    ("cell", "dtype", 9, b"dtype"), ("cell", "tensors", None, b"null tensors"),
    ("cell", "leg_dims", None, b"leg_dims[7] = 2"),
    ("opt", "chi", 15, b"chi"), ("opt", "chi", 1025, b"chi > 1024"),
    ("opt", "rsvd_oversample", -1, b"rsvd"), ("opt", "rsvd_power", -1, b"rsvd"),
    ("opt", "rsvd_oversample", 1000, b"oversample"), ("opt", "prec", 5, b"prec"),
    ("opt", "prec", -1, b"prec"), ("opt", "jacobi_max_sweeps", 0, b"jacobi"),
    ("opt", "corners", 3, b"corners"), ("opt", "corners", -4, b"corners"),
]


@pytest.mark.parametrize("target,field,value,frag", _RULES)
def test_each_create_rule_rejects_before_cuda(lib, target, field, value, frag):
    cell, opt, _keep = _good(lib)
    n = ctypes.c_size_t()
    assert lib.ipeps_ctm_workspace_size(ctypes.byref(cell), ctypes.byref(opt), ctypes.byref(n)) == 0
    _set(cell if target == "cell" else opt, field, value)
    assert lib.ipeps_ctm_workspace_size(ctypes.byref(cell), ctypes.byref(opt), ctypes.byref(n)) == 1
    assert frag in lib.ipeps_last_error(), lib.ipeps_last_error()
    h = ctypes.c_void_p()
    assert lib.ipeps_ctm_create(ctypes.byref(cell), ctypes.byref(opt), ctypes.byref(h)) == 1
    assert h.value is None


def test_workspace_grows_with_chi_and_D(lib):
    cell, opt, _keep = _good(lib)
    sizes = {}
    for D, chi in [(2, 16), (4, 64), (4, 100), (5, 100)]:
        cell.D, opt.chi = D, chi
        n = ctypes.c_size_t()
        assert lib.ipeps_ctm_workspace_size(ctypes.byref(cell), ctypes.byref(opt), ctypes.byref(n)) == 0
        sizes[(D, chi)] = n.value
        # at least the environment: 4 corners chi^2 and 4 edges chi^2 D^2 per site, complex
        assert n.value >= 4 * 16 * chi * chi * (1 + D * D)
    assert sizes[(2, 16)] < sizes[(4, 64)] < sizes[(4, 100)] < sizes[(5, 100)]


def test_null_handles_are_rejected(lib):
    D = ctypes.c_double
    buf = (D * 64)()
    i = ctypes.c_int()
    J = (D * 3)(1, 1, 1)
    calls = [
        lambda: lib.ipeps_ctm_move(None, 0, 1),
        lambda: lib.ipeps_ctm_spectra(None, buf),
        lambda: lib.ipeps_ctm_converge(None, 1e-10, 5, ctypes.byref(i), buf),
        lambda: lib.ipeps_rdm(None, buf, buf),
        lambda: lib.ipeps_rdm_site(None, buf),
        lambda: lib.ipeps_energy(None, J, buf),
        lambda: lib.ipeps_kappa(None, buf),
        lambda: lib.ipeps_fidelity(None, None, None, buf, buf),
        lambda: lib.ipeps_boundary_rho(None, 0, 2, buf, ctypes.byref(i), buf),
        lambda: lib.ipeps_boundary_rho_topk(None, 0, 2, 4, 50, 1e-10, buf, ctypes.byref(i), buf, buf),
        lambda: lib.ipeps_ctm_autotune(None),
        lambda: lib.ipeps_ctm_set_tensors(None, None, None),
        lambda: lib.ipeps_ctm_reset_env(None),
        lambda: lib.ipeps_ctm_sync(None),
        lambda: lib.ipeps_ctm_profile(None, 1),
        lambda: lib.ipeps_batch_move(None, 0, 1),
        lambda: lib.ipeps_batch_energy(None, J, buf),
        lambda: lib.ipeps_batch_sync(None),
    ]
    for k, call in enumerate(calls):
        assert call() == 1, (k, lib.ipeps_last_error())
        assert b"null" in lib.ipeps_last_error(), (k, lib.ipeps_last_error())
    # queries on null handles answer with neutral values, destroy is a no-op
    assert lib.ipeps_ctm_launch_count(None) == 0
    assert lib.ipeps_ctm_tuning_size(None) == 0
    assert lib.ipeps_batch_instance(None, 0) is None
    assert lib.ipeps_batch_launch_count(None) == 0
    assert lib.ipeps_batch_tuning_size(None) == 0
    assert lib.ipeps_batch_stream(None) is None
    lib.ipeps_ctm_destroy(None)
    lib.ipeps_batch_destroy(None)


def test_batch_create_rejects_empty(lib):
    cell, opt, _keep = _good(lib)
    b = ctypes.c_void_p()
    assert lib.ipeps_batch_create(0, ctypes.byref(cell), ctypes.byref(opt), 0, ctypes.byref(b)) == 1
    assert lib.ipeps_batch_create(1, None, ctypes.byref(opt), 0, ctypes.byref(b)) == 1
    assert b.value is None


def test_gemm_entry_points_reject_bad_shapes(lib):
    I, P = ctypes.c_int, ctypes.c_void_p
    one = P(16)
    # ipeps_zgemm(prec, M, N, K, A, opA, B, opB, C)
    assert lib.ipeps_zgemm(I(0), I(0), I(4), I(4), one, I(0), one, I(0), one) == 1
    assert lib.ipeps_zgemm(I(0), I(4), I(4), I(4), None, I(0), one, I(0), one) == 1
    assert lib.ipeps_zgemm(I(5), I(4), I(4), I(4), one, I(0), one, I(0), one) == 1
    assert lib.ipeps_zgemm(I(0), I(4), I(4), I(4), one, I(4), one, I(0), one) == 1
    # ipeps_zgemm_tile(prec, bn, splits, ...): tensor-core precisions and BN in {128, 256} only
    args = (I(4), I(4), I(4), one, I(0), one, I(0), one)
    assert lib.ipeps_zgemm_tile(I(0), I(128), I(1), *args) == 1
    assert lib.ipeps_zgemm_tile(I(2), I(64), I(1), *args) == 1
    assert lib.ipeps_zgemm_tile(I(2), I(128), I(0), *args) == 1
    assert b"tile" in lib.ipeps_last_error()
    assert lib.ipeps_zgemm_tile(I(3), I(192), I(1), *args) == 1
    assert b"tile" in lib.ipeps_last_error()


def test_noalloc_rejects_before_touching_scratch(lib):
    I, P = ctypes.c_int, ctypes.c_void_p
    assert lib.ipeps_corner_spectrum_noalloc(None, I(8), P(16), None) == 1
    assert b"null" in lib.ipeps_last_error()
    for chi in (0, -3, 257):
        assert lib.ipeps_corner_spectrum_noalloc(P(16), I(chi), P(16), None) == 1
        assert b"outside 1..256" in lib.ipeps_last_error()


def _fnv64_words(payload: np.ndarray) -> int:
    """The checkpoint checksum as the header states it (FNV-1a over 64-bit words)."""
    h = 0xCBF29CE484222325
    for w in payload.view(np.uint64).tolist():
        h = ((h ^ w) * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h


def _write_checkpoint(path, Lx, Ly, d, D, chi, pattern, seed=0, version=1):
    import struct
    rng = np.random.default_rng(seed)
    n = Lx * Ly * (4 * chi * chi + 4 * chi * D * D * chi)
    payload = rng.standard_normal(2 * n)
    with open(path, "wb") as f:
        f.write(b"IPEPSENV")
        f.write(struct.pack("<12i", version, Lx, Ly, d, D, chi, 4, *pattern, 0))
        f.write(payload.astype("<f8").tobytes())
        f.write(struct.pack("<Q", _fnv64_words(payload)))
    return payload


def test_checkpoint_header_and_checksum_verified_without_gpu(lib, tmp_path):
    from paper_1711_04798_gb300 import CTMError, env_file_info
    p = tmp_path / "env.ipeps"
    _write_checkpoint(p, 2, 2, 8, 2, 6, [0, 1, 1, 0])
    info = env_file_info(p)
    assert info == {"version": 1, "Lx": 2, "Ly": 2, "d": 8, "D": 2, "chi": 6, "n_tensors": 4,
                    "pattern": [0, 1, 1, 0]}
    raw = bytearray(p.read_bytes())
    # one flipped payload bit, a truncated file, a foreign file, a newer version
    bad = tmp_path / "bad.ipeps"
    flipped = bytearray(raw)
    flipped[56 + 100] ^= 0x10
    cases = {"checksum": bytes(flipped), "bytes, expected": bytes(raw[:-9]),
             "not an environment": b"NOTENV!!" + bytes(raw[8:]),
             "version": bytes(raw[:8]) + (2).to_bytes(4, "little") + bytes(raw[12:])}
    for frag, blob in cases.items():
        bad.write_bytes(blob)
        with pytest.raises(CTMError) as e:
            env_file_info(bad)
        assert e.value.status == 8 and frag in str(e.value), (frag, str(e.value))
    with pytest.raises(CTMError) as e:
        env_file_info(tmp_path / "missing.ipeps")
    assert e.value.status == 8


def test_checkpoint_calls_reject_null_handles(lib, tmp_path):
    buf = (ctypes.c_double * 8)()
    assert lib.ipeps_ctm_env_set(None, 0, 0, 0, buf) == 1
    assert lib.ipeps_ctm_env_copy(None, None) == 1
    assert lib.ipeps_ctm_save(None, str(tmp_path / "x").encode()) == 1
    assert lib.ipeps_ctm_load(None, str(tmp_path / "x").encode()) == 1
    assert lib.ipeps_env_file_info(None, (ctypes.c_int * 11)()) == 1
    assert not (tmp_path / "x").exists() and not (tmp_path / "x.part").exists()


def test_too_small_workspace_is_refused_before_cuda(lib):
    cell, opt, _keep = _good(lib)
    n = ctypes.c_size_t()
    assert lib.ipeps_ctm_workspace_size(ctypes.byref(cell), ctypes.byref(opt), ctypes.byref(n)) == 0
    opt.workspace = ctypes.c_void_p(4096)  # never touched: the size check comes first
    opt.workspace_bytes = n.value - 1
    h = ctypes.c_void_p()
    assert lib.ipeps_ctm_create(ctypes.byref(cell), ctypes.byref(opt), ctypes.byref(h)) == 2
    assert b"workspace too small" in lib.ipeps_last_error() and h.value is None


def test_product_path_never_loads_the_oracle():
    """The package (binding and build) neither imports the oracle nor has a CPU
    path: importing it leaves `oracle` unloaded, and no source mentions it."""
    import subprocess
    code = ("import sys; sys.path.insert(0, %r); import paper_1711_04798_gb300 as p; "
            "print('oracle' in sys.modules, 'synth' in sys.modules)" % ROOT)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, check=True)
    assert out.stdout.split() == ["False", "False"], out.stdout
    pkg = os.path.join(ROOT, "paper_1711_04798_gb300")
    for name in os.listdir(pkg):
        if name.endswith(".py"):
            src = open(os.path.join(pkg, name)).read()
            assert not re.search(r"^\s*(import|from)\s+(oracle|synth)\b", src, re.M), name


def test_missing_library_fails_loudly():
    from paper_1711_04798_gb300 import binding
    saved = binding._lib
    binding._lib = None
    try:
        with pytest.raises(RuntimeError, match="not built"):
            binding.load_library(os.path.join(ROOT, "no_such_dir", "libnothing.so"))
    finally:
        binding._lib = saved
