"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module draws random numbers and nothing else: it holds none of the
eigensolver's arithmetic.  Every routine is a pure function of its seed, so the
CPU oracle and the CUDA path read the very same bytes.

* Philox4x32-10 is the counter-based generator of Salmon, Moraes, Dror and Shaw,
  "Parallel random numbers: as easy as 1, 2, 3" (SC'11), written out from its
  published definition (ten rounds of the multiply-xor bijection with a Weyl key
  schedule).  The CUDA library carries its own implementation of the same
  definition for the random test vectors of the multigrid setup; both must
  produce identical bits for the uniforms defined in :func:`uniform_vectors`.
* Gauge links are U = exp(i eps H) with H = sum_a h_a lambda_a / 2 (Gell-Mann
  matrices, h_a standard normal via Box-Muller), i.e. random SU(3) matrices at
  distance O(eps) from the identity.  The exponential is taken through the
  eigen-decomposition of the Hermitian 3x3 matrix and the result is projected
  back onto SU(3) (Gram-Schmidt on two rows, third row = conj cross product).
* Z2 + iZ2 noise (entries (+-1 +- i)/sqrt 2) for right-hand sides, as in Sec. 3
  of the paper (the noise choice stated after Eq. 3.6).

Field layouts (host order, complex128):
  gauge  U[t, z, y, x, mu, a, b]      mu = 0..3 for the x, y, z, t directions
  spinor psi[t, z, y, x, spin, colour]
"""
from __future__ import annotations

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint32(0x9E3779B9)
_W1 = np.uint32(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)

# Stream tags: the fourth counter word keeps the uses of the generator apart.
TAG_GAUGE = 0x6A09E667
TAG_TESTVEC = 0x5EED0001
TAG_RHS = 0x5EED0002
TAG_EXTRA = 0x5EED0003


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on uint32 arrays (broadcasting).

    One round maps (c0, c1, c2, c3) with key (k0, k1) to
    (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0));
    the key is bumped by the Weyl constants (W0, W1) between rounds.
    """
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint32) for v in (c0, c1, c2, c3))
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    c0, c1, c2, c3 = (v.copy() for v in (c0, c1, c2, c3))
    k0 = np.uint32(k0)
    k1 = np.uint32(k1)
    with np.errstate(over="ignore"):
        for rnd in range(10):
            p0 = _M0 * c0.astype(np.uint64)
            p1 = _M1 * c2.astype(np.uint64)
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & _MASK32).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & _MASK32).astype(np.uint32)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
            if rnd != 9:
                k0 = np.uint32((int(k0) + int(_W0)) & 0xFFFFFFFF)
                k1 = np.uint32((int(k1) + int(_W1)) & 0xFFFFFFFF)
    return c0, c1, c2, c3


def _key(seed: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


def volume(dims) -> int:
    lx, ly, lz, lt = dims
    return lx * ly * lz * lt


def _gell_mann() -> np.ndarray:
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1] = -1j
    lam[1][1, 0] = 1j
    lam[2][0, 0] = 1
    lam[2][1, 1] = -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2] = -1j
    lam[4][2, 0] = 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2] = -1j
    lam[6][2, 1] = 1j
    lam[7][0, 0] = lam[7][1, 1] = 1 / np.sqrt(3)
    lam[7][2, 2] = -2 / np.sqrt(3)
    return lam


def _u01(bits: np.ndarray) -> np.ndarray:
    """uint32 -> uniform in the open interval (0, 1)."""
    return (bits.astype(np.float64) + 0.5) * 2.0 ** -32


def gauge_field(dims, eps: float, seed: int) -> np.ndarray:
    """Random SU(3) links U = exp(i eps H), H = sum_a h_a lambda_a/2, h_a ~ N(0,1).

    Link l = ((t*Lz + z)*Ly + y)*Lx + x)*4 + mu draws its 8 normals from two
    Philox blocks with counters (l, 0, b, TAG_GAUGE), b = 0, 1.
    """
    lx, ly, lz, lt = dims
    nlink = volume(dims) * 4
    k0, k1 = _key(seed)
    link = np.arange(nlink, dtype=np.uint64)
    normals = np.empty((nlink, 8), dtype=np.float64)
    for b in range(2):
        r = philox4x32_10(link.astype(np.uint32), 0, b, TAG_GAUGE, k0, k1)
        u1 = _u01(r[0]), _u01(r[2])
        u2 = _u01(r[1]), _u01(r[3])
        for q in range(2):
            rad = np.sqrt(-2.0 * np.log(u1[q]))
            normals[:, 4 * b + 2 * q] = rad * np.cos(2.0 * np.pi * u2[q])
            normals[:, 4 * b + 2 * q + 1] = rad * np.sin(2.0 * np.pi * u2[q])
    H = np.einsum("la,aij->lij", normals, _gell_mann() / 2.0)
    w, v = np.linalg.eigh(H)
    ph = np.exp(1j * eps * w)
    U = np.einsum("lia,la,lja->lij", v, ph, v.conj())
    U = _project_su3(U)
    return U.reshape(lt, lz, ly, lx, 4, 3, 3)


def _project_su3(U: np.ndarray) -> np.ndarray:
    r0 = U[:, 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=1, keepdims=True)
    r1 = U[:, 1, :]
    r1 = r1 - np.sum(r0.conj() * r1, axis=1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=1, keepdims=True)
    r2 = np.cross(r0, r1).conj()
    return np.stack([r0, r1, r2], axis=1)


def unit_gauge(dims) -> np.ndarray:
    lx, ly, lz, lt = dims
    U = np.zeros((lt, lz, ly, lx, 4, 3, 3), dtype=np.complex128)
    U[..., :, :] = np.eye(3)
    return U


def uniform_vectors(dims, n: int, seed: int, tag: int = TAG_TESTVEC) -> np.ndarray:
    """n spinor fields with re, im uniform in [-1, 1), exactly representable.

    Vector j, site s, component pair q (components 2q, 2q+1 of the 12 spin-colour
    components, index = spin*3 + colour) uses the Philox block with counter
    (s, q, j, tag); its four words w give re/im of the two components as
    int32(w) * 2^-31.  The CUDA setup reproduces these bits.
    """
    V = volume(dims)
    lx, ly, lz, lt = dims
    k0, k1 = _key(seed)
    out = np.empty((n, V, 12), dtype=np.complex128)
    site = np.arange(V, dtype=np.uint32)[:, None]
    q = np.arange(6, dtype=np.uint32)[None, :]
    for j in range(n):
        r = philox4x32_10(site, q, j, tag, k0, k1)
        f = [w.astype(np.uint32).view(np.int32).astype(np.float64) * 2.0 ** -31 for w in r]
        out[j, :, 0::2] = f[0] + 1j * f[1]
        out[j, :, 1::2] = f[2] + 1j * f[3]
    return out.reshape(n, lt, lz, ly, lx, 4, 3)


def z2_noise(dims, n: int, seed: int) -> np.ndarray:
    """n Z2+iZ2 noise spinors, entries (+-1 +- i)/sqrt(2) from Philox sign bits."""
    V = volume(dims)
    lx, ly, lz, lt = dims
    k0, k1 = _key(seed)
    out = np.empty((n, V, 12), dtype=np.complex128)
    site = np.arange(V, dtype=np.uint32)[:, None]
    q = np.arange(6, dtype=np.uint32)[None, :]
    s = 1.0 / np.sqrt(2.0)
    for j in range(n):
        r = philox4x32_10(site, q, j, TAG_RHS, k0, k1)
        sg = [np.where((w >> np.uint32(31)) & np.uint32(1), -s, s) for w in r]
        out[j, :, 0::2] = sg[0] + 1j * sg[1]
        out[j, :, 1::2] = sg[2] + 1j * sg[3]
    return out.reshape(n, lt, lz, ly, lx, 4, 3)


def gaussian_vectors(dims, n: int, seed: int) -> np.ndarray:
    """n spinors with independent standard-normal re/im parts (numpy PCG64)."""
    lx, ly, lz, lt = dims
    rng = np.random.default_rng(seed)
    shape = (n, lt, lz, ly, lx, 4, 3)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
