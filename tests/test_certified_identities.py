"""The algebra of the certified Gram path, checked in numpy (no GPU, no
library code): the identities that let the CUDA path replace the QR and SVD
of Sections 4 and 5 by Gram matrices when no rank is dropped.

For an orthonormal V_t and new directions A|_t, with C_t = V_t^* A|_t and
N_t = A|_t^* A|_t:
  * G_t = (V_t, A|_t)^* (V_t, A|_t) = L L^* with L = [[I, 0], [C_t^*, L_S]],
    L_S L_S^* = N_t - C_t^* C_t;
  * Q_t = (V_t, A|_t) L^{-*} = (V_t, (A|_t - V_t C_t) L_S^{-*}) is orthonormal
    and keeps V_t as its leading block;
  * the squared singular values of (V_t, A|_t) B~_t^* are the eigenvalues of
    L^* W_t L with W_t = B~_t^* B~_t, so the rank rule of the truncation keeps
    every column iff the smallest is above (eps/2)^2;
  * nested bases: with V_p|_{t_i} = V_{t_i} E_{t_i} and C_p = sum E^* C_i, the
    new father basis restricted to a son is Q_{t_i} F_{t_i},
    F = [[E, (C_i - E C_p) L_Sp^{-*}], [0, L_Si^* L_Sp^{-*}]];
  * a one-sided coupling: R_t [S_b; 0] = [S_b; 0] for R_t = L^*.
"""
import numpy as np
import pytest

from oracle.update import rank_rule


def _orth(rng, m, k):
    q, _ = np.linalg.qr(rng.standard_normal((m, k)))
    return q


def _block_factor(C, N):
    k, u = C.shape
    LS = np.linalg.cholesky(N - C.T @ C)
    L = np.zeros((k + u, k + u))
    L[:k, :k] = np.eye(k)
    L[k:, :k] = C.T
    L[k:, k:] = LS
    return L, LS


@pytest.mark.parametrize("m,k,u,seed", [(32, 16, 8, 1), (20, 5, 3, 2), (64, 24, 8, 3)])
def test_block_factor_and_new_basis(m, k, u, seed):
    rng = np.random.default_rng(seed)
    V = _orth(rng, m, k)
    A = rng.standard_normal((m, u))
    Vx = np.hstack([V, A])
    C, N = V.T @ A, A.T @ A
    L, LS = _block_factor(C, N)
    G = Vx.T @ Vx
    np.testing.assert_allclose(L @ L.T, G, rtol=0, atol=1e-12 * np.abs(G).max())
    Q = np.linalg.solve(L, Vx.T).T                      # Vx L^{-*}
    np.testing.assert_allclose(Q.T @ Q, np.eye(k + u), rtol=0, atol=1e-12)
    np.testing.assert_allclose(Q[:, :k], V, rtol=0, atol=1e-13)
    np.testing.assert_allclose(Q[:, k:], np.linalg.solve(LS, (A - V @ C).T).T, rtol=0, atol=1e-12)
    # one-sided coupling kept: L^* [S; 0] = [S; 0]
    S = rng.standard_normal((k, 7))
    Sx = np.vstack([S, np.zeros((u, 7))])
    np.testing.assert_array_equal(L.T @ Sx, Sx)


@pytest.mark.parametrize("seed", [4, 5])
def test_truncation_spectrum_from_grams(seed):
    m, k, u, n = 32, 16, 8, 90
    rng = np.random.default_rng(seed)
    V = _orth(rng, m, k)
    A = rng.standard_normal((m, u))
    Vx = np.hstack([V, A])
    Bt = rng.standard_normal((n, k + u)) * np.logspace(0, -6, k + u)   # graded weights
    L, _ = _block_factor(V.T @ A, A.T @ A)
    sv = np.linalg.svd(Vx @ Bt.T, compute_uv=False)
    ev = np.linalg.eigvalsh(L.T @ (Bt.T @ Bt) @ L)[::-1]
    np.testing.assert_allclose(ev, sv[:k + u] ** 2, rtol=1e-9, atol=1e-14 * sv[0] ** 2)
    # the oracle's rank rule keeps all K columns iff (eps/2)^2 is below the
    # smallest eigenvalue: the certificate's criterion
    for f, keep in ((0.99, True), (1.01, False)):
        eps = 2.0 * np.sqrt(ev[-1]) * f
        assert (rank_rule(sv, eps) == k + u) == keep


def test_nested_transfer_block_form():
    rng = np.random.default_rng(6)
    m1, m2, k1, k2, kp, u = 20, 24, 6, 7, 8, 3
    V1, V2 = _orth(rng, m1, k1), _orth(rng, m2, k2)
    E = _orth(rng, k1 + k2, kp)                       # [E_1; E_2] orthonormal columns
    E1, E2 = E[:k1], E[k1:]
    Vp = np.vstack([V1 @ E1, V2 @ E2])
    A1, A2 = rng.standard_normal((m1, u)), rng.standard_normal((m2, u))
    C1, C2 = V1.T @ A1, V2.T @ A2
    N1, N2 = A1.T @ A1, A2.T @ A2
    Cp = E1.T @ C1 + E2.T @ C2
    np.testing.assert_allclose(Cp, Vp.T @ np.vstack([A1, A2]), rtol=0, atol=1e-12)
    _, LS1 = _block_factor(C1, N1)
    _, LS2 = _block_factor(C2, N2)
    _, LSp = _block_factor(Cp, N1 + N2)
    Q1 = np.hstack([V1, np.linalg.solve(LS1, (A1 - V1 @ C1).T).T])
    Q2 = np.hstack([V2, np.linalg.solve(LS2, (A2 - V2 @ C2).T).T])
    Qp = np.hstack([Vp, np.linalg.solve(LSp, (np.vstack([A1, A2]) - Vp @ Cp).T).T])
    for Qi, Ei, Ci, LSi, rows in ((Q1, E1, C1, LS1, slice(0, m1)), (Q2, E2, C2, LS2, slice(m1, m1 + m2))):
        ki = Ei.shape[0]
        F = np.zeros((ki + u, kp + u))
        F[:ki, :kp] = Ei
        F[:ki, kp:] = np.linalg.solve(LSp, (Ci - Ei @ Cp).T).T
        F[ki:, kp:] = np.linalg.solve(LSp, LSi).T          # L_Si^* L_Sp^{-*}
        np.testing.assert_allclose(Qi @ F, Qp[rows], rtol=0, atol=1e-12)


def _f32_certificate(A, shift):
    """Float32 first try of the certificate, emulated: A 2^-e truncated
    toward zero to float32 (2^e ~ tr A), the diagonal shifted by
    (shift + 4 (n + 2) 2^-24 tr A) 2^-e rounded up, then an LDL^* in float32
    with every pivot required positive and finite."""
    n = A.shape[0]
    trA = float(np.trace(A))
    _, ex = np.frexp(trA)
    X = A * 2.0 ** (-int(ex))
    F = X.astype(np.float32)
    over = np.abs(F.astype(np.float64)) > np.abs(X)
    F[over] = np.nextafter(F[over], np.float32(0))          # truncation toward zero
    c = (shift + 4.0 * (n + 2) * 2.0 ** -24 * trA) * 2.0 ** (-int(ex))
    cf = np.float32(c)
    if float(cf) < c:
        cf = np.nextafter(cf, np.float32(np.inf))           # rounded up
    F = F - cf * np.eye(n, dtype=np.float32)
    for j in range(n):
        d = F[j, j]
        if not (np.isfinite(d) and d > np.float32(1e-30)):
            return False
        lv = F[j + 1:, j] / d
        F[j + 1:, j + 1:] -= np.outer(F[j + 1:, j], lv).astype(np.float32)
    return True


def test_float32_certificate_never_certifies_an_indefinite_shift():
    """Success of the float32 try proves A - shift I positive definite
    (Rump, BIT 2006): on matrices whose smallest eigenvalue lies just below
    the shift it must fail; well above the margin it succeeds."""
    rng = np.random.default_rng(12)
    fails_below = succeeds_above = 0
    for trial in range(120):
        n = int(rng.integers(4, 25))
        Q = _orth(rng, n, n)
        lam = np.sort(10.0 ** rng.uniform(-3, 0, n))[::-1] * float(rng.uniform(0.5, 4.0))
        trA = lam.sum()
        margin = 4.0 * (n + 2) * 2.0 ** -24 * trA
        shift = float(rng.uniform(0.0, 50.0)) * margin
        below = lam.copy()
        below[-1] = shift * (1.0 - 10.0 ** rng.uniform(-8, -1)) if shift > 0 else -1e-3 * margin
        A = (Q * below) @ Q.T
        A = 0.5 * (A + A.T)
        if np.linalg.eigvalsh(A)[0] - shift < 0:
            assert not _f32_certificate(A, shift), trial
            fails_below += 1
        above = lam.copy()
        above[-1] = shift + 100.0 * margin
        A = (Q * above) @ Q.T
        A = 0.5 * (A + A.T)
        succeeds_above += _f32_certificate(A, shift)
    assert fails_below > 100 and succeeds_above > 100
