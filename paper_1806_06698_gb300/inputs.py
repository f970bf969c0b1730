"""Seeded synthetic workloads for the batched 3x3 symmetric eigensolver.

This module holds none of the eigensolver's arithmetic: only random-matrix
recipes.  It is the one module that both the CPU oracle's tests and the CUDA
path's tests and benchmark use.  Every recipe returns packed upper triangles
``(n, 6)`` in the order (a11, a22, a33, a12, a13, a23) as a float64 master
copy; FP32 workloads are rounded from it.

Recipes (all from ``numpy.random.default_rng(seed)``):

* ``gaussian``      -- six iid N(0,1) entries (the paper's N(0,1) test set,
                        Sec. 1.5, and the small parity workload).
* ``mixed``         -- the mixed-difficulty batch: 60 % iid N(0,1); 20 %
                        Q diag(1, 1+10^-k, -1) Q^T with Haar Q and k ~ U[2,14];
                        10 % near-diagonal (diagonal N(0,1), off-diagonal
                        N(0,1)*1e-12); 10 % exact diagonals with a repeated
                        entry; every matrix scaled by 10^U(-s, s) (s = 50 for
                        FP64, 6 for FP32).  Subsets are interleaved by a seeded
                        permutation and their ids returned.
* ``structure_tensors`` -- sums of 27 outer products g g^T, g ~ N(0,1)^3,
                        scaled by 10^U(-3,3).  Sampled through the Bartlett
                        decomposition W = L L^T, L lower triangular with
                        L_ii^2 ~ chi^2(27 - i) (i = 0,1,2) and L_ij ~ N(0,1)
                        below the diagonal, which has exactly the Wishart(I, 27)
                        law of the sum of 27 outer products.
* ``spectral``      -- Q diag(d) Q^T with d ~ N(0,1)^3 and relative eigengaps
                        >= 1e-3 (rejection), plus a near-degenerate share whose
                        two closest eigenvalues differ by 1e-9 ||d||_2
                        (the differentiation workload).
* ``paper_set``     -- symmetric matrices with iid U(0,1), N(0,1) or chi^2_1
                        entries (the three distributions of Sec. 1.5).
"""

from __future__ import annotations

import numpy as np

SEED_BASE = 1806066980

SUBSET_GAUSSIAN = 0
SUBSET_CLUSTERED = 1
SUBSET_NEAR_DIAGONAL = 2
SUBSET_DIAGONAL_REPEATED = 3
SUBSET_NAMES = {
    SUBSET_GAUSSIAN: "gaussian",
    SUBSET_CLUSTERED: "clustered",
    SUBSET_NEAR_DIAGONAL: "near_diagonal",
    SUBSET_DIAGONAL_REPEATED: "diagonal_repeated",
}


def pack(M: np.ndarray) -> np.ndarray:
    """(n,3,3) symmetric -> (n,6) packed (a11,a22,a33,a12,a13,a23)."""
    M = np.asarray(M)
    return np.stack([M[:, 0, 0], M[:, 1, 1], M[:, 2, 2], M[:, 0, 1], M[:, 0, 2], M[:, 1, 2]], axis=1)


def unpack(A6: np.ndarray) -> np.ndarray:
    """(n,6) packed -> (n,3,3) symmetric."""
    A6 = np.asarray(A6)
    n = A6.shape[0]
    M = np.empty((n, 3, 3), dtype=A6.dtype)
    M[:, 0, 0], M[:, 1, 1], M[:, 2, 2] = A6[:, 0], A6[:, 1], A6[:, 2]
    M[:, 0, 1] = M[:, 1, 0] = A6[:, 3]
    M[:, 0, 2] = M[:, 2, 0] = A6[:, 4]
    M[:, 1, 2] = M[:, 2, 1] = A6[:, 5]
    return M


def haar(rng: np.random.Generator, n: int) -> np.ndarray:
    """n Haar-distributed 3x3 orthogonal matrices: QR of a Gaussian matrix with
    the signs of R's diagonal moved into Q (Mezzadri, Notices AMS 54, 2007)."""
    Z = rng.standard_normal((n, 3, 3))
    Q, R = np.linalg.qr(Z)
    d = np.sign(np.diagonal(R, axis1=1, axis2=2))
    d[d == 0] = 1.0
    return Q * d[:, None, :]


def conj_diag(Q: np.ndarray, d: np.ndarray) -> np.ndarray:
    """Packed Q diag(d) Q^T."""
    M = np.einsum("nik,nk,njk->nij", Q, d, Q)
    M = 0.5 * (M + np.swapaxes(M, 1, 2))
    return pack(M)


def gaussian(n: int, seed: int = SEED_BASE) -> np.ndarray:
    """Six iid N(0,1) entries per matrix."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, 6))


def _clustered(rng, n):
    k = rng.uniform(2.0, 14.0, n)
    d = np.stack([np.ones(n), 1.0 + 10.0 ** (-k), -np.ones(n)], axis=1)
    return conj_diag(haar(rng, n), d)


def _near_diagonal(rng, n):
    A = np.empty((n, 6))
    A[:, :3] = rng.standard_normal((n, 3))
    A[:, 3:] = rng.standard_normal((n, 3)) * 1e-12
    return A


def _diagonal_repeated(rng, n):
    # Patterns (v,v,w), (v,w,v), (w,v,v), (v,v,v), chosen uniformly.
    v = rng.standard_normal(n)
    w = rng.standard_normal(n)
    pat = rng.integers(0, 4, n)
    A = np.zeros((n, 6))
    A[:, 0] = np.where(pat == 2, w, v)
    A[:, 1] = np.where(pat == 1, w, v)
    A[:, 2] = np.where(pat == 0, w, v)
    return A


def mixed(n: int, seed: int = SEED_BASE + 1, log10_scale: float = 50.0):
    """Mixed-difficulty batch; returns (A6 float64 (n,6), subset ids int8 (n,))."""
    rng = np.random.default_rng(seed)
    n_cl = int(round(0.2 * n))
    n_nd = int(round(0.1 * n))
    n_dr = int(round(0.1 * n))
    n_g = n - n_cl - n_nd - n_dr
    parts = [rng.standard_normal((n_g, 6)), _clustered(rng, n_cl), _near_diagonal(rng, n_nd),
             _diagonal_repeated(rng, n_dr)]
    ids = np.concatenate([np.full(n_g, SUBSET_GAUSSIAN, np.int8), np.full(n_cl, SUBSET_CLUSTERED, np.int8),
                          np.full(n_nd, SUBSET_NEAR_DIAGONAL, np.int8),
                          np.full(n_dr, SUBSET_DIAGONAL_REPEATED, np.int8)])
    A = np.concatenate(parts, axis=0)
    A *= 10.0 ** rng.uniform(-log10_scale, log10_scale, n)[:, None]
    perm = rng.permutation(n)
    return np.ascontiguousarray(A[perm]), ids[perm]


def mixed_fp32(n: int, seed: int = SEED_BASE + 2):
    """The mixed batch at scale 10^U(-6,6), rounded to float32; returns
    (A6 float32, subset ids)."""
    A, ids = mixed(n, seed, log10_scale=6.0)
    return A.astype(np.float32), ids


def structure_tensors(n: int, seed: int = SEED_BASE + 3, dof: int = 27) -> np.ndarray:
    """Sums of ``dof`` outer products g g^T (Wishart(I, dof)) scaled by
    10^U(-3,3), float64 master copy (see the module docstring)."""
    rng = np.random.default_rng(seed)
    l00 = np.sqrt(rng.chisquare(dof, n))
    l11 = np.sqrt(rng.chisquare(dof - 1, n))
    l22 = np.sqrt(rng.chisquare(dof - 2, n))
    l10, l20, l21 = rng.standard_normal((3, n))
    # W = L L^T for L = [[l00,0,0],[l10,l11,0],[l20,l21,l22]].
    A = np.empty((n, 6))
    A[:, 0] = l00 * l00
    A[:, 1] = l10 * l10 + l11 * l11
    A[:, 2] = l20 * l20 + l21 * l21 + l22 * l22
    A[:, 3] = l00 * l10
    A[:, 4] = l00 * l20
    A[:, 5] = l10 * l20 + l11 * l21
    A *= 10.0 ** rng.uniform(-3.0, 3.0, n)[:, None]
    return A


def spectral(n: int, seed: int = SEED_BASE + 4, near_degenerate: float = 0.05,
             min_gap: float = 1e-3, degenerate_gap: float = 1e-9):
    """Q diag(d) Q^T with known d (ascending).  A share ``near_degenerate`` has
    two eigenvalues within ``degenerate_gap * ||d||_2``; the rest have every
    gap >= ``min_gap * ||d||_2``.  Returns (A6, d ascending (n,3), is_degenerate)."""
    rng = np.random.default_rng(seed)
    n_deg = int(round(near_degenerate * n))
    n_ok = n - n_deg
    d_ok = np.empty((0, 3))
    while d_ok.shape[0] < n_ok:
        d = np.sort(rng.standard_normal((2 * (n_ok - d_ok.shape[0]) + 16, 3)), axis=1)
        nrm = np.linalg.norm(d, axis=1)
        good = np.min(np.diff(d, axis=1), axis=1) >= min_gap * nrm
        d_ok = np.concatenate([d_ok, d[good]], axis=0)
    d_ok = d_ok[:n_ok]
    d_deg = np.sort(rng.standard_normal((n_deg, 3)), axis=1)
    pair = rng.integers(0, 2, n_deg)  # which adjacent pair is pinched
    nrm = np.linalg.norm(d_deg, axis=1)
    idx = np.arange(n_deg)
    d_deg[idx, pair + 1] = d_deg[idx, pair] + degenerate_gap * nrm
    d_deg = np.sort(d_deg, axis=1)
    d = np.concatenate([d_ok, d_deg], axis=0)
    deg = np.concatenate([np.zeros(n_ok, bool), np.ones(n_deg, bool)])
    perm = rng.permutation(n)
    d, deg = d[perm], deg[perm]
    A = conj_diag(haar(rng, n), d)
    return np.ascontiguousarray(A), d, deg


def paper_set(n: int, dist: str, seed: int = SEED_BASE + 5) -> np.ndarray:
    """Symmetric test matrices with iid entries from 'uniform' U(0,1), 'normal'
    N(0,1) or 'chisq' chi^2 with one degree of freedom (Sec. 1.5)."""
    rng = np.random.default_rng(seed)
    if dist == "uniform":
        return rng.uniform(0.0, 1.0, (n, 6))
    if dist == "normal":
        return rng.standard_normal((n, 6))
    if dist == "chisq":
        return rng.chisquare(1.0, (n, 6))
    raise ValueError(f"unknown distribution {dist!r}")


def trace_free_spiked(n: int, seed: int = SEED_BASE + 7) -> np.ndarray:
    """Matrices whose leading 2x2 block has zero trace (alpha1 + alpha2 = 0:
    the rotation maps the pair (p, -p) to (l, -l) exactly) and whose spikes
    differ by 10^k in size, k ~ U(4, 20):
    the case where the simplified deflation test of Sec. 1.1 (right side
    ~ |alpha1 + alpha2|) and the EISPACK-style test it comes from disagree.
    Block diag(t, -t), t ~ U(0.5, 2), rotated by a uniform angle in the
    (1,2)-plane; spikes (10^-k z1, z2) rotated with it; a33 ~ N(0,1)."""
    rng = np.random.default_rng(seed)
    t = rng.uniform(0.5, 2.0, n)
    th = rng.uniform(0.0, np.pi, n)
    k = rng.uniform(4.0, 20.0, n)
    z1 = rng.standard_normal(n) * 10.0 ** (-k)
    z2 = rng.standard_normal(n)
    c, s = np.cos(th), np.sin(th)
    A = np.empty((n, 6))
    A[:, 0] = t * (c * c - s * s)   # R diag(t, -t) R^T
    A[:, 1] = -A[:, 0]
    A[:, 3] = 2.0 * t * c * s
    A[:, 4] = c * z1 - s * z2       # R (z1, z2)
    A[:, 5] = s * z1 + c * z2
    A[:, 2] = rng.standard_normal(n)
    return A
