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
