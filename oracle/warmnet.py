"""TEST INFRASTRUCTURE ONLY (the CPU oracle): the unrolled warm-start
network in FP64, written from its definition, for checking the GPU kernels'
forward values and gradients.

The network continues the iteration of Sec. 4 from a state (S, Theta) with
the labels p held fixed, for K layers.  Layer k has its own step rho_k and
soft threshold tau_k:
    D = X - S + Theta/rho_k,   mu_i = mean of D over cluster i        (Eq. (18))
    L = a_k D + (1 - a_k) mu_p,  a_k = rho_k / (2 lambda + rho_k)
    B = X - L + Theta/rho_k,   S' = sign(B) max(|B| - tau_k, 0)       (Eq. (24) with tau_k)
    Theta' = Theta + rho_k (X - L - S')                               (Eq. (25))
With rho_k = rho * kappa^k and tau_k = 1 / rho_k these are the plain
iterations with the labels fixed.  The learned parameters are log
multipliers on that schedule: rho_k = rho kappa^k exp(theta_k),
tau_k = exp(phi_k) / rho_k.
"""
from __future__ import annotations

import numpy as np

from . import cluster_means


def schedule(rho: float, kappa: float, theta, phi):
    """Per-layer (rho_k, tau_k) from the log multipliers."""
    theta = np.asarray(theta, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    K = theta.size
    rho_k = rho * kappa ** np.arange(K) * np.exp(theta)
    tau_k = np.exp(phi) / rho_k
    return rho_k, tau_k


def forward(X, labels, c, lam, S0, T0, rho_k, tau_k):
    """K layers from (S0, Theta0); returns (L, S, Theta) after the last one."""
    X = np.asarray(X, dtype=np.float64)
    S = np.array(S0, dtype=np.float64)
    T = np.array(T0, dtype=np.float64)
    p = np.asarray(labels, dtype=np.int32)
    L = None
    for rho, tau in zip(rho_k, tau_k):
        D = X - S + T / rho
        mu, _ = cluster_means(np.asfortranarray(D), p, c)
        a = rho / (2.0 * lam + rho)
        L = a * D + (1.0 - a) * mu[:, p]
        B = X - L + T / rho
        Sn = np.sign(B) * np.maximum(np.abs(B) - tau, 0.0)
        T = T + rho * (X - L - Sn)
        S = Sn
    return L, S, T


def loss(L, S, Lt, St, scale):
    """scale (||L - Lt||^2 + ||S - St||^2)."""
    return scale * (np.sum((L - Lt) ** 2) + np.sum((S - St) ** 2))


def mlp_unpack(P, nz, H, nout):
    """Packed parameters [W1 (H x nz) | b1 | W2 (nout x H) | b2] as arrays."""
    P = np.asarray(P, dtype=np.float64)
    o = 0
    W1 = P[o:o + H * nz].reshape(H, nz); o += H * nz
    b1 = P[o:o + H]; o += H
    W2 = P[o:o + nout * H].reshape(nout, H); o += nout * H
    b2 = P[o:o + nout]
    return W1, b1, W2, b2


def mlp_forward(P, z, nz, H, nout):
    """out = W2 tanh(W1 z + b1) + b2; returns (out, hidden)."""
    W1, b1, W2, b2 = mlp_unpack(P, nz, H, nout)
    h = np.tanh(W1 @ np.asarray(z, dtype=np.float64) + b1)
    return W2 @ h + b2, h


def mlp_grad(P, z, gout, nz, H, nout):
    """Gradient of <gout, out> with respect to the packed parameters (chain
    rule through the two affine maps and tanh' = 1 - tanh^2)."""
    W1, b1, W2, b2 = mlp_unpack(P, nz, H, nout)
    z = np.asarray(z, dtype=np.float64)
    gout = np.asarray(gout, dtype=np.float64)
    _, h = mlp_forward(P, z, nz, H, nout)
    gh = (W2.T @ gout) * (1.0 - h * h)
    return np.concatenate([np.outer(gh, z).ravel(), gh, np.outer(gout, h).ravel(), gout])


def adam_step(P, G, M, V, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba, Algorithm 1); returns (P, M, V)."""
    M = b1 * M + (1.0 - b1) * G
    V = b2 * V + (1.0 - b2) * G * G
    mh = M / (1.0 - b1 ** t)
    vh = V / (1.0 - b2 ** t)
    return P - lr * mh / (np.sqrt(vh) + eps), M, V
