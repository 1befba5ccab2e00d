"""Local Fourier analysis of the ILU(0) smoother and the choice of vertex order
(arXiv 2210.15280, Sec. 3, the paragraphs after the stencil equations).

TEST INFRASTRUCTURE ONLY: imported by tests/; never by the library, with
which it shares no code.

Steps, in the paper's order:
  1. the constant operator stencil A_d of the tet with kappa = 1 (the
     coefficient is assumed to be the identity inside the macro-tet);
  2. the asymptotic ILU stencil L_d (d in D_l), D_c: the stencil equations
     with coordinate-independent values, iterated Gauss-Seidel fashion from
     L_c = D_c = 1, L_d = 0;
  3. the symbols D(t) = D_c, L(t) = 1 + sum_{d in D_l} L_d e^{i d.t},
     A(t) = sum_{d in D} A_d e^{i d.t};
  4. the smoothing factor: the largest |(L D conj(L) - A) / (L D conj(L))| over
     the high frequencies (-pi, pi)^3 minus (-pi/2, pi/2)^3, sampled on a
     uniform grid of 16 points per axis;
  5. over the 24 vertex orders of the tet, the order with the smallest
     smoothing factor.
"""
import itertools

import numpy as np

from . import oracle as orc

# direction vectors in the order of D (Sec. 2.1)
DVEC = np.array([(-1, 0, 0), (0, -1, 0), (1, -1, 0), (-1, 1, -1), (0, 1, -1), (0, 0, -1), (1, 0, -1), (0, 0, 0),
                 (1, 0, 0), (0, 1, 0), (-1, 1, 0), (1, -1, 1), (0, -1, 1), (0, 0, 1), (-1, 0, 1)])
W, S, SE, BNW, BN, BC, BE, C = range(8)


def constant_stencil(P, level=6):
    """The 15 stencil values A_d of the tet with kappa = 1 at a point deep in
    the interior (all interior points of an affine tet share them)."""
    N = 2 ** level
    return orc.local_stencil(P, N, (N // 4, N // 4, N // 4))


def asymptotic_stencil(A, iters=2000, tol=1e-15):
    """Fixed point of the stencil equations of Sec. 3 with the same values at
    every point:
        A_bc  = L_bc D
        A_s   = L_bc D L_bn + L_s D
        A_bnw = L_bc D L_se + L_bnw D
        A_be  = L_bc D L_w + L_be D
        A_w   = L_bc D L_be + L_bnw D L_bn + L_s D L_se + L_w D
        A_bn  = L_bc D L_s + L_be D L_se + L_bnw D L_w + L_bn D
        A_se  = L_bc D L_bnw + L_be D L_bn + L_se D + L_s D L_w
        A_c   = D + sum_{d in D_l} L_d^2 D
    solved in that order for L_bc, L_s, ..., D with the latest values.  The
    iteration runs on A / A_c: L is scale-free and D scales with A (remark
    of Sec. 3), and from D = 1 the iteration converges on that scale for any
    level A was assembled on.
    Returns (L[7] in the order w s se bnw bn bc be, D)."""
    scale = A[C]
    A = np.asarray(A, dtype=np.float64) / scale
    L = np.zeros(7)
    D = 1.0
    for _ in range(iters):
        old = np.append(L, D)
        L[BC] = A[BC] / D
        L[S] = (A[S] - L[BC] * D * L[BN]) / D
        L[BNW] = (A[BNW] - L[BC] * D * L[SE]) / D
        L[BE] = (A[BE] - L[BC] * D * L[W]) / D
        L[W] = (A[W] - L[BC] * D * L[BE] - L[BNW] * D * L[BN] - L[S] * D * L[SE]) / D
        L[BN] = (A[BN] - L[BC] * D * L[S] - L[BE] * D * L[SE] - L[BNW] * D * L[W]) / D
        L[SE] = (A[SE] - L[BC] * D * L[BNW] - L[BE] * D * L[BN] - L[S] * D * L[W]) / D
        D = A[C] / (1.0 + np.sum(L ** 2))
        if np.abs(np.append(L, D) - old).max() <= tol:
            break
    return L, D * scale


def theta_grid(n=16):
    """Uniform samples of (-pi, pi)^3 (k = 0..n-1 at -pi + 2 pi k / n) that
    lie in the high-frequency set: some component outside (-pi/2, pi/2)."""
    t = -np.pi + 2.0 * np.pi * np.arange(n) / n
    T = np.stack(np.meshgrid(t, t, t, indexing="ij"), axis=-1).reshape(-1, 3)
    high = np.any(np.abs(T) >= np.pi / 2, axis=1)
    return T[high]


def smoothing_factor(A, n=16):
    """mu = max over the sampled high frequencies of |1 - A / (L D conj L)|."""
    L, D = asymptotic_stencil(A)
    T = theta_grid(n)
    ph = np.exp(1j * (T @ DVEC.T))  # (samples, 15)
    Ls = 1.0 + ph[:, :7] @ L
    As = ph @ A
    M = Ls * D * np.conj(Ls)
    return float(np.max(np.abs((M - As) / M)))


def best_order(P, n=16):
    """(perm, mu, mus): the vertex order (perm[i] = index of the original
    vertex placed at position i) with the smallest smoothing factor, the
    factor, and the factors of all 24 orders in itertools order."""
    P = np.asarray(P, dtype=np.float64).reshape(4, 3)
    mus = []
    perms = list(itertools.permutations(range(4)))
    for p in perms:
        mus.append(smoothing_factor(constant_stencil(P[list(p)]), n))
    k = int(np.argmin(mus))
    return list(perms[k]), mus[k], mus
