"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA library tests.

This module holds no CTM arithmetic: it only draws numbers.  Every value comes
from SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) used as a counter-based generator:

    z  = seed + (n + 1) * 0x9E3779B97F4A7C15          (mod 2^64)
    z  = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z  = (z ^ (z >> 27)) * 0x94D049BB133111EB
    out = z ^ (z >> 31)

`uniform53(seed, n)` = (out >> 11) * 2^-53 in [0, 1), an exact double.  Normal
deviates use the Box-Muller transform on two consecutive uniforms.

Workloads (the PEPS tensors of the paper's Sec. II.A, A[p,u,l,d,r], d = 2^3 = 8
for a three-spin block site of the ruby lattice, Sec. II.B):

* ``random_real``: iid N(0,1) entries, then divided by max |A| (per tensor).
* ``product_plus_noise``: the all-spins-up product state (A[0,0,0,0,0] = 1,
  p = 0 meaning sigma^z = +1 on all three spins) plus ``eps`` times iid complex
  normal noise with Re, Im ~ N(0, 1/2) on every entry.

Tensor ``t`` of a workload with seed ``s`` draws from stream ``s * 16 + t``.

The randomized range finder of the projector step needs a test matrix Omega;
``omega`` draws it with uniform [-1, 1) real and imaginary parts (exact
doubles, so the CUDA library's own SplitMix64 copy reproduces it bit for bit).
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: np.ndarray) -> np.ndarray:
    """SplitMix64 output for counters ``n`` (uint64 array) of stream ``seed``."""
    n = np.asarray(n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed % (1 << 64)) + (n + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform53(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` exact doubles in [0, 1) from counters offset .. offset+count-1."""
    n = np.arange(offset, offset + count, dtype=np.uint64)
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, count: int) -> np.ndarray:
    """``count`` iid N(0,1) deviates (Box-Muller on uniform pairs)."""
    u = uniform53(seed, 2 * count)
    u1 = 1.0 - u[0::2]  # in (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def random_real(seed: int, tid: int, d: int, D: int) -> np.ndarray:
    """A[p,u,l,d,r] real, iid N(0,1), normalised to max-abs 1."""
    A = normal(seed * 16 + tid, d * D ** 4).reshape(d, D, D, D, D)
    return A / np.max(np.abs(A))


def product_plus_noise(seed: int, tid: int, d: int, D: int, eps: float = 0.1) -> np.ndarray:
    """All-up product state plus eps * complex normal noise (E|z|^2 = 1)."""
    n = d * D ** 4
    g = normal(seed * 16 + tid, 2 * n)
    noise = (g[:n] + 1j * g[n:]) * np.sqrt(0.5)
    A = eps * noise.reshape(d, D, D, D, D)
    A[0, 0, 0, 0, 0] += 1.0
    return A


def omega(seed: int, rows: int, cols: int) -> np.ndarray:
    """Range-finder test matrix, rows x cols complex, Re/Im uniform in [-1, 1).

    Entry (i, j) uses counters 2*(i*cols + j) (real) and 2*(i*cols + j) + 1
    (imaginary) of stream ``seed``.
    """
    u = uniform53(seed, 2 * rows * cols)
    re = 2.0 * u[0::2] - 1.0
    im = 2.0 * u[1::2] - 1.0
    return (re + 1j * im).reshape(rows, cols)


# ---------------------------------------------------------------------------
# Named workloads.  Each returns (tensors, pattern, Lx, Ly, d, D, chi, J).
# pattern[y][x] is the tensor id at cell position (x, y).
# ---------------------------------------------------------------------------

def workload(name: str, seed: int = 0, D: int | None = None, chi: int | None = None):
    """Return a dict describing one of the paper-shaped synthetic workloads.

    ``real``           4 real iid-normal tensors, d=8, J=(1,1,1); D=2, chi=16
                       unless given
    ``product_noise``  4 complex all-up product + 0.1 noise tensors, d=8,
                       J=(1,1,0.5); D and chi must be given (the paper's runs
                       use D = 4, 5, 6 with chi = 64, 100, 144)
    """
    d = 8
    if name == "real":
        D = D or 2
        chi = chi or 16
        tensors = [random_real(seed, t, d, D) for t in range(4)]
        J = (1.0, 1.0, 1.0)
    elif name == "product_noise":
        if D is None or chi is None:
            raise ValueError("product_noise needs D and chi")
        tensors = [product_plus_noise(seed, t, d, D) for t in range(4)]
        J = (1.0, 1.0, 0.5)
    else:
        raise ValueError(f"unknown workload {name}")
    return {
        "tensors": tensors,
        "pattern": [[0, 1], [2, 3]],
        "Lx": 2,
        "Ly": 2,
        "d": d,
        "D": D,
        "chi": chi,
        "J": J,
        "seed": seed,
    }


def scan(seed: int = 0, n: int = 64, Ds=(3, 4, 5), chis=(32, 48, 64, 100)):
    """The batched phase-diagram scan: ``n`` independent instances.

    Instance k sits at Jz = 2k/(n-1) on the line Jx = Jy = (2 - Jz)/2 (the
    paper's Jx = Jy scan, Sec. VI), with bond dimension Ds[(k + r) mod len(Ds)]
    and environment dimension chis[(k + r) mod len(chis)], r = seed mod 12.
    Its four tensors follow the product-plus-noise recipe with workload seed
    seed * 64 + k.  Returns a list of dicts (tensors, pattern, D, chi, J).
    """
    r = seed % 12
    out = []
    for k in range(n):
        Jz = 2.0 * k / max(n - 1, 1)
        D = Ds[(k + r) % len(Ds)]
        chi = chis[(k + r) % len(chis)]
        tensors = [product_plus_noise(seed * 64 + k, t, 8, D) for t in range(4)]
        out.append({"tensors": tensors, "pattern": [[0, 1], [2, 3]], "D": D, "chi": chi,
                    "J": ((2.0 - Jz) / 2.0, (2.0 - Jz) / 2.0, Jz), "k": k})
    return out


def fidelity_line(seed: int = 0, n: int = 5, D: int = 2, d: int = 8, eps: float = 0.1):
    """States at n points of a synthetic coupling line, for fidelity surfaces
    (the paper scans the fidelity per site of ground states at pairs of
    couplings J1, J2 on a line, Sec. VI; its optimised states are not
    available, so a smooth one-parameter family stands in for them).

    Point k has angle theta_k = (pi/2) k/(n-1) and four tensors
    A_t = all-up product + eps * (cos theta_k N1_t + sin theta_k N2_t), where
    N1_t and N2_t are fixed complex normal draws (Re, Im ~ N(0, 1/2)) from
    streams (seed*16 + t) and ((seed+1)*16 + t).  Returns a list of n tensor
    lists (2x2 cell, pattern [[0, 1], [2, 3]])."""
    size = d * D ** 4
    base = []
    for t in range(4):
        g1 = normal(seed * 16 + t, 2 * size)
        g2 = normal((seed + 1) * 16 + t, 2 * size)
        n1 = ((g1[:size] + 1j * g1[size:]) * np.sqrt(0.5)).reshape(d, D, D, D, D)
        n2 = ((g2[:size] + 1j * g2[size:]) * np.sqrt(0.5)).reshape(d, D, D, D, D)
        base.append((n1, n2))
    out = []
    for k in range(n):
        th = 0.5 * np.pi * k / max(n - 1, 1)
        ts = []
        for n1, n2 in base:
            A = eps * (np.cos(th) * n1 + np.sin(th) * n2)
            A[0, 0, 0, 0, 0] += 1.0
            ts.append(A)
        out.append(ts)
    return out


def star_tensors(seed: int = 0, D: int = 2, d: int = 8, eps: float = 0.1):
    """Block tensors of a star-lattice state on the 2x2 cell (App. B): the
    all-up product state plus eps times complex normal noise, on the three
    real legs of each triangle block site; the fourth leg is the trivial
    (dimension 1) edge of the brick wall: u for A sites (pattern ids 0 and 3,
    x + y even), d for B sites (ids 1 and 2).  Tensor t draws from stream
    seed*16 + t.  Shapes (d, 1, D, D, D) for A, (d, D, D, 1, D) for B."""
    out = []
    for t in range(4):
        shape = (d, 1, D, D, D) if t in (0, 3) else (d, D, D, 1, D)
        size = int(np.prod(shape))
        g = normal(seed * 16 + t, 2 * size)
        A = eps * ((g[:size] + 1j * g[size:]) * np.sqrt(0.5)).reshape(shape)
        A[0, 0, 0, 0, 0] += 1.0
        out.append(A)
    return out
