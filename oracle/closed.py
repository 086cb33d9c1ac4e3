"""Closed-form spectra used to pin the oracle (Sec. III.A).

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import itertools

import numpy as np


def uncoupled_levels(omega, dims, n):
    """Lowest n eigenvalues of sum_i omega_i (n_i + 1/2) with 0 <= n_i < d_i, by brute-force
    enumeration of every occupation vector (tiny systems only)."""
    omega = np.asarray(omega, dtype=np.float64)
    E = [float(np.dot(omega, np.asarray(v) + 0.5))
         for v in itertools.product(*[range(d) for d in dims])]
    return np.sort(E)[:n]


def normal_mode_frequencies(omega, coupling):
    """Frequencies of H = sum_i omega_i/2 (p_i^2 + q_i^2) + sum_{i<j} alpha_ij q_i q_j
    (Eq. coupled_harmonic_oscillator): nu_k = sqrt(eig(Omega^1/2 A Omega^1/2)) with
    A_ii = omega_i and A_ij = alpha_ij (symmetric, i != j)."""
    omega = np.asarray(omega, dtype=np.float64)
    A = np.array(coupling, dtype=np.float64)
    A = 0.5 * (A + A.T)
    np.fill_diagonal(A, omega)
    s = np.sqrt(omega)
    ev = np.linalg.eigvalsh(s[:, None] * A * s[None, :])
    return np.sqrt(ev)


def normal_mode_levels(nu, n, n_max=12):
    """Lowest n values of sum_k nu_k (n_k + 1/2)."""
    nu = np.asarray(nu)
    E = [float(np.dot(nu, np.asarray(v) + 0.5))
         for v in itertools.product(range(n_max), repeat=len(nu))]
    return np.sort(E)[:n]
