"""TEST INFRASTRUCTURE ONLY (the CPU oracle): the spectral p step, the
nonlinear alternative to K-means that Sec. 4.2 names for the labels, in FP64.

Sec. 4.2 allows any clustering of the columns of L in place of K-means and
names spectral clustering without fixing its form.  This oracle takes the
normalised spectral clustering of Ng, Jordan and Weiss (2001):
  1. A_ij = exp(-||y_i - y_j||^2 / (2 sigma^2)) for i != j, A_ii = 0, with
     sigma^2 = scale * (mean squared distance over the pairs i != j);
  2. M = D^{-1/2} A D^{-1/2},  D = diag(row sums of A);
  3. U = an orthonormal basis of the eigenvectors of M's c largest eigenvalues
     (numpy.linalg.eigh);
  4. e_i = U_i / ||U_i|| (rows of U normalised);
  5. K-means on the e_i with c groups: the same k-means++ seeding (seed) and
     Lloyd iteration as the initial labels (oracle.init_labels).
Steps 4-5 depend on U only through the distances between its rows, which do
not change when U is rotated within the eigenspace, so any basis gives the
same labels.
"""
from __future__ import annotations

import numpy as np

from . import State, init_labels, l_step, s_step, theta_step


def sq_distances(Y):
    """||y_i - y_j||^2 for every pair, summed coordinate by coordinate."""
    Y = np.asarray(Y, dtype=np.float64)
    n = Y.shape[1]
    D2 = np.zeros((n, n))
    for row in Y:
        D2 += (row[:, None] - row[None, :]) ** 2
    return D2


def mean_sq_distance(Y) -> float:
    """Mean of ||y_i - y_j||^2 over the ordered pairs i != j."""
    n = np.asarray(Y).shape[1]
    return float(sq_distances(Y).sum() / (n * (n - 1)))


def affinity(Y, scale):
    """(A, degrees, sigma^2) of step 1-2."""
    n = np.asarray(Y).shape[1]
    D2 = sq_distances(Y)
    sigma2 = scale * D2.sum() / (n * (n - 1))
    A = np.exp(-D2 / (2.0 * sigma2))
    np.fill_diagonal(A, 0.0)
    return A, A.sum(axis=1), sigma2


def embedding(Y, c, scale):
    """(U, eigenvalues, E): the top-c eigenvectors of M (n x c), their
    eigenvalues, and the row-normalised embedding as a c x n matrix."""
    A, deg, _ = affinity(Y, scale)
    s = 1.0 / np.sqrt(deg)
    M = s[:, None] * A * s[None, :]
    w, V = np.linalg.eigh(M)
    U = V[:, -c:]
    E = (U / np.linalg.norm(U, axis=1, keepdims=True)).T
    return U, w[-c:], np.asfortranarray(E)


def labels(Y, c, scale, seed, km_max=100):
    """Spectral p step: labels of the columns of Y."""
    _, _, E = embedding(Y, c, scale)
    p, _ = init_labels(E, c, seed, km_max)
    return p


def iteration(X, state: State, c, lam, scale, seed, kappa=1.5, km_max=100):
    """One iteration of Sec. 4 with the spectral p step: L (Eq. (18), labels
    p_t), p from L_{t+1}, S (Eq. (24)), Theta (Eq. (25)), rho <- kappa rho.
    Returns (state, (||X-L-S||, ||dL||, ||dS||))."""
    X = np.asarray(X, dtype=np.float64)
    s = state.copy()
    L, _, _ = l_step(X, s.S, s.Theta, s.rho, lam, s.labels, c)
    p = labels(L, c, scale, seed, km_max)
    S = s_step(X, L, s.Theta, s.rho)
    T = theta_step(X, L, S, s.Theta, s.rho)
    norms = (np.linalg.norm(X - L - S), np.linalg.norm(L - s.L), np.linalg.norm(S - s.S))
    return State(np.asfortranarray(L), np.asfortranarray(S), np.asfortranarray(T), p.astype(np.int32),
                 s.rho * kappa), norms
