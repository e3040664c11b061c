"""ctypes binding of the C ABI in include/ipeps_ctm.h (argument marshalling
only; every step of the CTM path runs in the CUDA library)."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libipeps_ctm.so")

PREC = {"fp64": 0, "tf32": 1, "bf16x3": 2, "bf16x6": 3, "fp64tc": 4}
DIRS = {"L": 0, "U": 1, "R": 2, "D": 3, "sweep": 4}
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOCONV", 5: "ETIMEOUT",
          6: "ENUMERIC", 7: "EUNSUPPORTED", 8: "EIO"}

EXPORTS = [
    "ipeps_default_options", "ipeps_ctm_workspace_size", "ipeps_ctm_create",
    "ipeps_ctm_set_tensors", "ipeps_ctm_reset_env", "ipeps_ctm_move", "ipeps_ctm_spectra",
    "ipeps_ctm_converge", "ipeps_rdm", "ipeps_energy", "ipeps_kappa", "ipeps_fidelity",
    "ipeps_boundary_rho", "ipeps_ctm_env_get", "ipeps_ctm_sync", "ipeps_ctm_launch_count",
    "ipeps_ctm_destroy", "ipeps_last_error", "ipeps_ctm_profile", "ipeps_ctm_profile_read",
    "ipeps_batch_create", "ipeps_batch_move", "ipeps_batch_energy", "ipeps_batch_instance",
    "ipeps_batch_tuning_size", "ipeps_batch_tuning_entry", "ipeps_batch_launch_count",
    "ipeps_batch_sync", "ipeps_batch_destroy", "ipeps_batch_stream", "ipeps_boundary_rho_topk",
    "ipeps_ctm_autotune", "ipeps_ctm_tuning_size", "ipeps_zgemm_tile", "ipeps_ctm_env_set",
    "ipeps_ctm_save", "ipeps_ctm_load", "ipeps_env_file_info", "ipeps_rdm_site", "ipeps_batch_fidelity",
    "ipeps_boundary_renyi2", "ipeps_energy_star", "ipeps_boundary_rho_refined", "ipeps_ctm_env_copy",
]


class Cell(C.Structure):
    _fields_ = [("Lx", C.c_int), ("Ly", C.c_int), ("pattern", C.c_int * 4), ("n_tensors", C.c_int),
                ("d", C.c_int), ("D", C.c_int), ("dtype", C.c_int),
                ("tensors", C.POINTER(C.c_void_p)), ("tensors_bra", C.POINTER(C.c_void_p)),
                ("leg_dims", C.POINTER(C.c_int))]


class Options(C.Structure):
    _fields_ = [("chi", C.c_int), ("prec", C.c_int), ("rsvd_oversample", C.c_int),
                ("rsvd_power", C.c_int), ("svd_cutoff", C.c_double), ("orth_tol", C.c_double),
                ("omega_seed", C.c_uint64), ("jacobi_max_sweeps", C.c_int),
                ("stream", C.c_void_p), ("workspace", C.c_void_p), ("workspace_bytes", C.c_size_t),
                ("wait_cycles", C.c_longlong), ("corners", C.c_int)]


class CTMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH):
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = C.CDLL(path)
    P, I, D = C.c_void_p, C.c_int, C.c_double
    lib.ipeps_default_options.argtypes = [C.POINTER(Options)]
    lib.ipeps_default_options.restype = None
    lib.ipeps_ctm_workspace_size.argtypes = [C.POINTER(Cell), C.POINTER(Options), C.POINTER(C.c_size_t)]
    lib.ipeps_ctm_create.argtypes = [C.POINTER(Cell), C.POINTER(Options), C.POINTER(P)]
    lib.ipeps_ctm_set_tensors.argtypes = [P, C.POINTER(P), C.POINTER(P)]
    lib.ipeps_ctm_reset_env.argtypes = [P]
    lib.ipeps_ctm_move.argtypes = [P, I, I]
    lib.ipeps_ctm_spectra.argtypes = [P, C.POINTER(D)]
    lib.ipeps_ctm_converge.argtypes = [P, D, I, C.POINTER(I), C.POINTER(D)]
    lib.ipeps_rdm.argtypes = [P, C.POINTER(D), C.POINTER(D)]
    lib.ipeps_rdm_site.argtypes = [P, C.POINTER(D)]
    lib.ipeps_energy.argtypes = [P, C.POINTER(D), C.POINTER(D)]
    lib.ipeps_kappa.argtypes = [P, C.POINTER(D)]
    lib.ipeps_fidelity.argtypes = [P, P, P, C.POINTER(D), C.POINTER(D)]
    lib.ipeps_boundary_rho.argtypes = [P, I, I, C.POINTER(D), C.POINTER(I), C.POINTER(D)]
    lib.ipeps_ctm_env_get.argtypes = [P, I, I, I, C.POINTER(D)]
    lib.ipeps_ctm_env_set.argtypes = [P, I, I, I, C.POINTER(D)]
    lib.ipeps_ctm_env_copy.argtypes = [P, P]
    lib.ipeps_ctm_save.argtypes = [P, C.c_char_p]
    lib.ipeps_ctm_load.argtypes = [P, C.c_char_p]
    lib.ipeps_env_file_info.argtypes = [C.c_char_p, C.POINTER(I)]
    lib.ipeps_ctm_autotune.argtypes = [P]
    lib.ipeps_ctm_tuning_size.argtypes = [P]
    lib.ipeps_boundary_rho_topk.argtypes = [P, I, I, I, I, D, C.POINTER(D), C.POINTER(I), C.POINTER(D),
                                            C.POINTER(D)]
    lib.ipeps_ctm_sync.argtypes = [P]
    lib.ipeps_ctm_launch_count.argtypes = [P]
    lib.ipeps_ctm_launch_count.restype = C.c_uint64
    lib.ipeps_ctm_profile.argtypes = [P, I]
    lib.ipeps_ctm_profile_read.argtypes = [P, I, C.POINTER(D), C.POINTER(C.c_uint64), C.POINTER(D)]
    lib.ipeps_ctm_destroy.argtypes = [P]
    lib.ipeps_ctm_destroy.restype = None
    lib.ipeps_last_error.restype = C.c_char_p
    lib.ipeps_batch_create.argtypes = [I, C.POINTER(Cell), C.POINTER(Options), I, C.POINTER(P)]
    lib.ipeps_batch_move.argtypes = [P, I, I]
    lib.ipeps_batch_energy.argtypes = [P, C.POINTER(D), C.POINTER(D)]
    lib.ipeps_boundary_rho_refined.argtypes = [P, I, I, I, D, C.POINTER(D), C.POINTER(I), C.POINTER(D),
                                               C.POINTER(I), C.POINTER(D)]
    lib.ipeps_energy_star.argtypes = [P, C.POINTER(D), C.POINTER(D)]
    lib.ipeps_boundary_renyi2.argtypes = [P, I, I, C.POINTER(D), C.POINTER(D)]
    lib.ipeps_batch_fidelity.argtypes = [P, I, C.POINTER(I), C.POINTER(I), C.POINTER(I), C.POINTER(D),
                                         C.POINTER(D)]
    lib.ipeps_batch_instance.argtypes = [P, I]
    lib.ipeps_batch_instance.restype = P
    lib.ipeps_batch_tuning_size.argtypes = [P]
    lib.ipeps_batch_tuning_entry.argtypes = [P, I, C.POINTER(I), C.POINTER(D)]
    lib.ipeps_batch_launch_count.argtypes = [P]
    lib.ipeps_batch_launch_count.restype = C.c_uint64
    lib.ipeps_batch_sync.argtypes = [P]
    lib.ipeps_batch_stream.argtypes = [P]
    lib.ipeps_batch_stream.restype = P
    lib.ipeps_batch_destroy.argtypes = [P]
    lib.ipeps_batch_destroy.restype = None
    for name in EXPORTS:
        if name not in ("ipeps_default_options", "ipeps_ctm_destroy", "ipeps_last_error",
                        "ipeps_ctm_launch_count", "ipeps_batch_instance", "ipeps_batch_launch_count",
                        "ipeps_batch_destroy", "ipeps_batch_stream"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def env_file_info(path) -> dict:
    """Header of a verified environment checkpoint (no GPU needed)."""
    lib = load_library()
    info = (C.c_int * 11)()
    _check(lib.ipeps_env_file_info(os.fsencode(path), info))
    keys = ("version", "Lx", "Ly", "d", "D", "chi", "n_tensors")
    out = dict(zip(keys, info[:7]))
    out["pattern"] = list(info[7:11])
    return out


def _check(st: int):
    if st != 0:
        raise CTMError(st, _lib.ipeps_last_error().decode())


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _bond_dim(tensors):
    """D of a cell: the largest virtual leg (legs of size 1 are trivial bonds)."""
    return max(max(t.shape[1:]) for t in tensors)


def _make_cell(tensors, pattern, bra=None):
    """ipeps_cell for the host tensors (kept alive by the returned tuple)."""
    Ly, Lx = len(pattern), len(pattern[0])
    d, D = tensors[0].shape[0], _bond_dim(tensors)
    cplx = any(np.iscomplexobj(t) for t in tensors) or (bra is not None)
    dt = np.complex128 if cplx else np.float64
    keep = [np.ascontiguousarray(t, dtype=dt) for t in tensors]
    keep_bra = [np.ascontiguousarray(t, dtype=dt) for t in bra] if bra is not None else None
    cell = Cell()
    cell.Lx, cell.Ly = Lx, Ly
    for y in range(Ly):
        for x in range(Lx):
            cell.pattern[y * Lx + x] = pattern[y][x]
    cell.n_tensors = len(tensors)
    cell.d, cell.D = d, D
    cell.dtype = 1 if cplx else 0
    ptrs = (C.c_void_p * len(tensors))(*[t.ctypes.data for t in keep])
    cell.tensors = C.cast(ptrs, C.POINTER(C.c_void_p))
    bptrs = None
    if keep_bra is not None:
        bptrs = (C.c_void_p * len(tensors))(*[t.ctypes.data for t in keep_bra])
        cell.tensors_bra = C.cast(bptrs, C.POINTER(C.c_void_p))
    legs = None
    if any(t.shape[1:] != (D, D, D, D) for t in tensors):
        legs = (C.c_int * (4 * len(tensors)))(*[s for t in tensors for s in t.shape[1:]])
        cell.leg_dims = C.cast(legs, C.POINTER(C.c_int))
    return cell, (keep, keep_bra, ptrs, bptrs, dt, legs)


def _make_options(lib, chi, prec="fp64", oversample=16, power=2, cutoff=0.0, orth_tol=1e-14,
                  omega_seed=7, jacobi_max_sweeps=40, stream=None, workspace=None, wait_cycles=0, corners=4):
    opt = Options()
    lib.ipeps_default_options(C.byref(opt))
    opt.chi = chi
    opt.prec = PREC[prec]
    opt.rsvd_oversample, opt.rsvd_power = oversample, power
    opt.svd_cutoff, opt.orth_tol = cutoff, orth_tol
    opt.omega_seed = omega_seed
    opt.jacobi_max_sweeps = jacobi_max_sweeps
    opt.wait_cycles = wait_cycles
    opt.corners = corners
    opt.stream = stream
    if workspace is not None:
        opt.workspace = C.c_void_p(workspace[0])
        opt.workspace_bytes = workspace[1]
    return opt


class CTM:
    """One CTM environment on the GPU (handle of the C ABI).

    tensors: list of A[p,u,l,d,r] (float64 or complex128 numpy arrays);
    pattern: [[id at (x,y)]] rows y, columns x; bra: optional second list for
    the mixed network of the fidelity (Sec. III).
    """

    def __init__(self, tensors, pattern, chi, prec="fp64", bra=None, oversample=16, power=2,
                 cutoff=0.0, orth_tol=1e-14, omega_seed=7, jacobi_max_sweeps=40, stream=None,
                 workspace=None, wait_cycles=0, corners=4):
        lib = load_library()
        self.lib = lib
        self._borrowed = False
        cell, keep = _make_cell(tensors, pattern, bra)
        self._keep, self._keep_bra, self._ptrs, self._bptrs, self._dtype, self._legs = keep
        self._set_meta(tensors, pattern, chi)
        opt = _make_options(lib, chi, prec, oversample, power, cutoff, orth_tol, omega_seed,
                            jacobi_max_sweeps, stream, workspace, wait_cycles, corners)
        self._cell, self._opt = cell, opt
        h = C.c_void_p()
        _check(lib.ipeps_ctm_create(C.byref(cell), C.byref(opt), C.byref(h)))
        self.h = h

    def _set_meta(self, tensors, pattern, chi):
        self.Ly, self.Lx = len(pattern), len(pattern[0])
        self.d, self.D, self.chi = tensors[0].shape[0], _bond_dim(tensors), chi
        self.n_tensors = len(tensors)

    @classmethod
    def _borrow(cls, lib, h, tensors, pattern, chi, dtype):
        """A view of a handle owned elsewhere (a batch instance)."""
        self = cls.__new__(cls)
        self.lib, self.h, self._borrowed = lib, h, True
        self._set_meta(tensors, pattern, chi)
        self._dtype = dtype
        return self

    @staticmethod
    def workspace_bytes(tensors, pattern, chi, **kw) -> int:
        lib = load_library()
        Ly, Lx = len(pattern), len(pattern[0])
        cell = Cell()
        cell.Lx, cell.Ly = Lx, Ly
        for y in range(Ly):
            for x in range(Lx):
                cell.pattern[y * Lx + x] = pattern[y][x]
        cell.n_tensors = len(tensors)
        cell.d, cell.D = tensors[0].shape[0], _bond_dim(tensors)
        cell.dtype = 1
        dummy = (C.c_void_p * len(tensors))(*([1] * len(tensors)))
        cell.tensors = C.cast(dummy, C.POINTER(C.c_void_p))
        opt = Options()
        lib.ipeps_default_options(C.byref(opt))
        opt.chi = chi
        opt.rsvd_oversample = kw.get("oversample", 16)
        n = C.c_size_t()
        _check(lib.ipeps_ctm_workspace_size(C.byref(cell), C.byref(opt), C.byref(n)))
        return n.value

    def close(self):
        if getattr(self, "h", None):
            if not getattr(self, "_borrowed", False):
                self.lib.ipeps_ctm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rebuild(self):
        """Rebuild the double layers from the device-resident tensors."""
        _check(self.lib.ipeps_ctm_set_tensors(self.h, None, None))

    def set_tensors(self, tensors, bra=None):
        self._keep = [np.ascontiguousarray(t, dtype=self._dtype) for t in tensors]
        self._ptrs = (C.c_void_p * len(tensors))(*[t.ctypes.data for t in self._keep])
        bp = None
        if bra is not None:
            self._keep_bra = [np.ascontiguousarray(t, dtype=self._dtype) for t in bra]
            self._bptrs = (C.c_void_p * len(bra))(*[t.ctypes.data for t in self._keep_bra])
            bp = C.cast(self._bptrs, C.POINTER(C.c_void_p))
        _check(self.lib.ipeps_ctm_set_tensors(self.h, C.cast(self._ptrs, C.POINTER(C.c_void_p)), bp))

    def reset_env(self):
        _check(self.lib.ipeps_ctm_reset_env(self.h))

    def move(self, direction="sweep", count=1):
        _check(self.lib.ipeps_ctm_move(self.h, DIRS[direction], count))

    def sweep(self, count=1):
        self.move("sweep", count)

    def autotune(self) -> int:
        """Tile choices of the tensor-core products measured once; returns the number of shapes."""
        _check(self.lib.ipeps_ctm_autotune(self.h))
        return int(self.lib.ipeps_ctm_tuning_size(self.h))

    def spectra(self) -> np.ndarray:
        out = np.zeros((4, self.Ly, self.Lx, self.chi))
        _check(self.lib.ipeps_ctm_spectra(self.h, _dptr(out)))
        return out

    def converge(self, tol, max_sweeps):
        n, dl = C.c_int(), C.c_double()
        st = self.lib.ipeps_ctm_converge(self.h, tol, max_sweeps, C.byref(n), C.byref(dl))
        if st not in (0, 4):
            _check(st)
        return n.value, dl.value, st == 0

    def rdms(self):
        n = self.d * self.d
        rh = np.zeros((self.Ly, self.Lx, n, n), dtype=np.complex128)
        rv = np.zeros_like(rh)
        _check(self.lib.ipeps_rdm(self.h, _dptr(rh.view(np.float64)), _dptr(rv.view(np.float64))))
        return {"h": rh, "v": rv}

    def site_rdms(self) -> np.ndarray:
        """One-site RDMs [Ly, Lx, d, d] (rows ket), trace one."""
        out = np.zeros((self.Ly, self.Lx, self.d, self.d), dtype=np.complex128)
        _check(self.lib.ipeps_rdm_site(self.h, _dptr(out.view(np.float64))))
        return out

    def energy(self, J) -> float:
        Jv = np.asarray(J, dtype=np.float64)
        e = C.c_double()
        _check(self.lib.ipeps_energy(self.h, _dptr(Jv), C.byref(e)))
        return e.value

    def energy_star(self, J) -> float:
        """Star-lattice Heisenberg energy per spin, J = (J_t, J_e) (ipeps_energy_star)."""
        Jv = np.asarray(J, dtype=np.float64)
        e = C.c_double()
        _check(self.lib.ipeps_energy_star(self.h, _dptr(Jv), C.byref(e)))
        return e.value

    def kappa(self) -> complex:
        k = np.zeros(2)
        _check(self.lib.ipeps_kappa(self.h, _dptr(k)))
        return complex(k[0], k[1])

    @staticmethod
    def fidelity(h12: "CTM", h11: "CTM", h22: "CTM"):
        lib = load_library()
        db, ds = C.c_double(), C.c_double()
        _check(lib.ipeps_fidelity(h12.h, h11.h, h22.h, C.byref(db), C.byref(ds)))
        return db.value, ds.value

    def boundary_rho(self, x, Nv):
        n = self.D ** Nv
        eig = np.zeros(n)
        nout, S = C.c_int(), C.c_double()
        _check(self.lib.ipeps_boundary_rho(self.h, x, Nv, _dptr(eig), C.byref(nout), C.byref(S)))
        return eig[: nout.value], S.value

    def boundary_rho_refined(self, x, Nv, iters=200, tol=1e-12):
        """Boundary spectrum of the rings refined by the exact column transfer
        matrix; returns (lam, S, iterations, last change)."""
        n = self.D ** Nv
        eig = np.zeros(n)
        nout, S, it, ch = C.c_int(), C.c_double(), C.c_int(), C.c_double()
        _check(self.lib.ipeps_boundary_rho_refined(self.h, x, Nv, iters, tol, _dptr(eig), C.byref(nout),
                                                   C.byref(S), C.byref(it), C.byref(ch)))
        return eig[: nout.value], S.value, it.value, ch.value

    def boundary_renyi2(self, x, Nv):
        """Second Renyi entropy of the boundary operator from traces; returns (S2, purity)."""
        S2, p = C.c_double(), C.c_double()
        _check(self.lib.ipeps_boundary_renyi2(self.h, x, Nv, C.byref(S2), C.byref(p)))
        return S2.value, p.value

    def boundary_rho_topk(self, x, Nv, k, max_iter=300, tol=1e-10):
        """Leading k boundary-spectrum values (Lanczos); returns (lam, S, rest, n_conv)."""
        lam = np.zeros(k)
        nc, S, rest = C.c_int(), C.c_double(), C.c_double()
        _check(self.lib.ipeps_boundary_rho_topk(self.h, x, Nv, k, max_iter, tol, _dptr(lam), C.byref(nc),
                                                C.byref(S), C.byref(rest)))
        return lam, S.value, rest.value, nc.value

    def env(self, role, x, y) -> np.ndarray:
        n = self.chi * self.chi if role < 4 else self.chi * self.D * self.D * self.chi
        out = np.zeros(n, dtype=np.complex128)
        _check(self.lib.ipeps_ctm_env_get(self.h, role, x, y, _dptr(out.view(np.float64))))
        if role < 4:
            return out.reshape(self.chi, self.chi)
        return out.reshape(self.chi, self.D * self.D, self.chi)

    def set_env(self, role, x, y, t: np.ndarray):
        """Overwrite one environment tensor (layout of ``env``): a user-supplied start."""
        n = self.chi * self.chi if role < 4 else self.chi * self.D * self.D * self.chi
        buf = np.ascontiguousarray(t, dtype=np.complex128).reshape(-1)
        if buf.size != n:
            raise ValueError(f"role {role} needs {n} complex elements, got {buf.size}")
        _check(self.lib.ipeps_ctm_env_set(self.h, role, x, y, _dptr(buf.view(np.float64))))

    def copy_env_from(self, other: "CTM"):
        """Take other's whole environment (same cell, D and chi), on the device."""
        _check(self.lib.ipeps_ctm_env_copy(self.h, other.h))

    def save(self, path):
        """Write the environment to a checkpoint file."""
        _check(self.lib.ipeps_ctm_save(self.h, os.fsencode(path)))

    def load(self, path):
        """Replace the environment by a checkpoint of the same Lx, Ly, D and chi."""
        _check(self.lib.ipeps_ctm_load(self.h, os.fsencode(path)))

    def sync(self):
        _check(self.lib.ipeps_ctm_sync(self.h))

    def profile(self, enable=True):
        _check(self.lib.ipeps_ctm_profile(self.h, 1 if enable else 0))

    def profile_read(self, kind=0):
        ms, n, fl = C.c_double(), C.c_uint64(), C.c_double()
        _check(self.lib.ipeps_ctm_profile_read(self.h, kind, C.byref(ms), C.byref(n), C.byref(fl)))
        return {"ms": ms.value, "launches": int(n.value), "flops": fl.value}

    def launch_count(self) -> int:
        return int(self.lib.ipeps_ctm_launch_count(self.h))


class Batch:
    """Independent CTM instances advanced together (ipeps_batch_*): one CUDA
    graph launch per move over all instances, tensor-core tiles from the
    library's autotuner.

    instances: list of dicts with keys tensors, pattern, chi (and optionally
    bra); every option of CTM (prec, oversample, ...) applies to all of them.
    """

    def __init__(self, instances, tune=True, **kw):
        lib = load_library()
        self.lib = lib
        n = len(instances)
        cells = (Cell * n)()
        opts = (Options * n)()
        self._keep = []
        for i, inst in enumerate(instances):
            cell, keep = _make_cell(inst["tensors"], inst["pattern"], inst.get("bra"))
            cells[i] = cell
            self._keep.append(keep)
            opts[i] = _make_options(lib, inst["chi"], **kw)
        h = C.c_void_p()
        _check(lib.ipeps_batch_create(n, cells, opts, 1 if tune else 0, C.byref(h)))
        self.h = h
        self.n = n
        self._views = [CTM._borrow(lib, C.c_void_p(lib.ipeps_batch_instance(h, i)), inst["tensors"],
                                   inst["pattern"], inst["chi"], self._keep[i][4])
                       for i, inst in enumerate(instances)]

    def move(self, direction="sweep", count=1):
        _check(self.lib.ipeps_batch_move(self.h, DIRS[direction], count))

    def sweep(self, count=1):
        self.move("sweep", count)

    def energies(self, J) -> np.ndarray:
        Jv = np.ascontiguousarray(np.broadcast_to(np.asarray(J, dtype=np.float64), (self.n, 3)))
        e = np.zeros(self.n)
        _check(self.lib.ipeps_batch_energy(self.h, _dptr(Jv), _dptr(e)))
        return e

    def instance(self, i) -> CTM:
        return self._views[i]

    def fidelity(self, pairs):
        """Fidelity per site of each (i12, i11, i22) triple of instance indices:
        returns (d_block, d_spin) arrays (ipeps_batch_fidelity)."""
        n = len(pairs)
        idx = [np.ascontiguousarray([p[q] for p in pairs], dtype=np.int32) for q in range(3)]
        db, ds = np.zeros(n), np.zeros(n)
        ptr = [a.ctypes.data_as(C.POINTER(C.c_int)) for a in idx]
        _check(self.lib.ipeps_batch_fidelity(self.h, n, ptr[0], ptr[1], ptr[2], _dptr(db), _dptr(ds)))
        return db, ds

    def tuning(self):
        out = []
        f = (C.c_int * 6)()
        us = (C.c_double * 2)()
        for i in range(self.lib.ipeps_batch_tuning_size(self.h)):
            _check(self.lib.ipeps_batch_tuning_entry(self.h, i, f, us))
            out.append({"prec": f[0], "M": f[1], "N": f[2], "K": f[3], "bn": f[4], "splits": f[5],
                        "us": us[0], "default_us": us[1]})
        return out

    def sync(self):
        _check(self.lib.ipeps_batch_sync(self.h))

    def launch_count(self) -> int:
        return int(self.lib.ipeps_batch_launch_count(self.h))

    def stream(self) -> int:
        """cudaStream_t the batch launches its graphs on."""
        return int(self.lib.ipeps_batch_stream(self.h) or 0)

    def close(self):
        if getattr(self, "h", None):
            for v in self._views:
                v.h = None
            self.lib.ipeps_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
