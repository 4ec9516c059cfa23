"""The recurrences behind the level-2 contribution blocks of the strip factor (Section 2.3,
the separator system of Algorithm 1 solved in groups), checked on the CPU against a dense
inverse.

A group's separators form a block-tridiagonal system T y = bhat, factored twisted at
tq = (n-1)/2: R_i, E_i = Rinv_i L_i (i < tq) or Rinv_i U_i (i > tq), F_i the inner coupling,
and solved from a_i = Rinv_i bhat_i.  The factor kernel stores K_i with y(last) = sum K_i a_i
and K'_i with y(first) = sum K'_i a_i, from the solve's recurrences run backwards; this file
restates those recurrences (as the kernel runs them) and compares K_i with
(T^-1)[last, i] R_i for every group size up to 9.
"""
import numpy as np
import pytest


def twisted_lu(Tb, Lb, Ub):
    n = len(Tb)
    W = Tb[0].shape[0]
    tq = (n - 1) // 2
    E, F, Rinv = [None] * n, [None] * n, [None] * n
    Z = np.zeros((W, W))
    for i in range(tq):
        R = Tb[i] - (Lb[i] @ F[i - 1] if i >= 1 else 0)
        Rinv[i] = np.linalg.inv(R)
        E[i] = Rinv[i] @ Lb[i] if i >= 1 else Z
        F[i] = Rinv[i] @ Ub[i]
    for i in range(n - 1, tq, -1):
        R = Tb[i] - (Ub[i] @ F[i + 1] if i <= n - 2 else 0)
        Rinv[i] = np.linalg.inv(R)
        E[i] = Rinv[i] @ Ub[i] if i <= n - 2 else Z
        F[i] = Rinv[i] @ Lb[i]
    i = tq
    R = Tb[i] - (Lb[i] @ F[i - 1] if i >= 1 else 0) - (Ub[i] @ F[i + 1] if i <= n - 2 else 0)
    Rinv[i] = np.linalg.inv(R)
    E[i] = Rinv[i] @ Lb[i] if i >= 1 else Z
    F[i] = Rinv[i] @ Ub[i] if i <= n - 2 else Z
    return E, F, Rinv


def k_last(E, F, W):
    n = len(E)
    tq = (n - 1) // 2
    K = [None] * n
    G = [None] * n
    G[n - 1] = np.eye(W)
    for j in range(n - 1, tq, -1):
        G[j - 1] = -G[j] @ F[j]
    K[tq] = G[tq]
    Z = G[tq]
    for j in range(tq, 0, -1):
        Z = -Z @ E[j]
        K[j - 1] = Z
    if n - 1 > tq:
        Z = G[tq + 1] - G[tq] @ F[tq]
        K[tq + 1] = Z
        for j in range(tq + 2, n):
            Z = G[j] - Z @ E[j - 1]
            K[j] = Z
    return K


def k_first(E, F, W):
    n = len(E)
    tq = (n - 1) // 2
    K = [None] * n
    G = [None] * n
    G[0] = np.eye(W)
    for j in range(tq):
        G[j + 1] = -G[j] @ F[j]
    K[tq] = G[tq]
    if n - 1 > tq:
        Z = -G[tq] @ F[tq]
        K[tq + 1] = Z
        for j in range(tq + 1, n - 1):
            Z = -Z @ E[j]
            K[j + 1] = Z
    if tq >= 1:
        Z = G[tq - 1] - G[tq] @ E[tq]
        K[tq - 1] = Z
        for j in range(tq - 1, 0, -1):
            Z = G[j - 1] - Z @ E[j]
            K[j - 1] = Z
    return K


@pytest.mark.parametrize("n", range(1, 10))
def test_end_value_blocks_match_dense_inverse(n):
    rng = np.random.default_rng(100 + n)
    W = 4
    # complex symmetric diagonal blocks, U_i = L_{i+1}^T (the Schur complements of a complex
    # symmetric strip operator)
    Tb = []
    for _ in range(n):
        a = rng.standard_normal((W, W)) + 1j * rng.standard_normal((W, W))
        Tb.append((a + a.T) / 2 + 5 * np.eye(W))
    Ub = [0.4 * (rng.standard_normal((W, W)) + 1j * rng.standard_normal((W, W))) for _ in range(n)]
    Lb = [None] + [Ub[i - 1].T for i in range(1, n)]
    E, F, Rinv = twisted_lu(Tb, Lb, Ub)
    T = np.zeros((n * W, n * W), dtype=complex)
    for i in range(n):
        T[i * W:(i + 1) * W, i * W:(i + 1) * W] = Tb[i]
        if i >= 1:
            T[i * W:(i + 1) * W, (i - 1) * W:i * W] = Lb[i]
        if i <= n - 2:
            T[i * W:(i + 1) * W, (i + 1) * W:(i + 2) * W] = Ub[i]
    Ti = np.linalg.inv(T)
    K, K0 = k_last(E, F, W), k_first(E, F, W)
    for i in range(n):
        R = np.linalg.inv(Rinv[i])
        assert np.allclose(K[i], Ti[(n - 1) * W:, i * W:(i + 1) * W] @ R, atol=1e-12)
        assert np.allclose(K0[i], Ti[:W, i * W:(i + 1) * W] @ R, atol=1e-12)
    # and the end values of a solve through the twisted factors agree with T^-1 bhat
    bhat = rng.standard_normal(n * W) + 1j * rng.standard_normal(n * W)
    a = [Rinv[i] @ bhat[i * W:(i + 1) * W] for i in range(n)]
    y = Ti @ bhat
    assert np.allclose(sum(K[i] @ a[i] for i in range(n)), y[(n - 1) * W:], atol=1e-12)
    assert np.allclose(sum(K0[i] @ a[i] for i in range(n)), y[:W], atol=1e-12)
