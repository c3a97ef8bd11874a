"""Proximal operators of Table 2 and the dual updates of Algorithm 2, float64."""
from __future__ import annotations

import numpy as np


def soft_threshold(z: np.ndarray, alpha) -> np.ndarray:
    """prox_{alpha ||.||_1}(z) = sgn(z) max(|z| - alpha, 0) (Table 2, row 1)."""
    return np.sign(z) * np.maximum(np.abs(z) - alpha, 0.0)


def prox_l21_rows(Z: np.ndarray, alpha) -> np.ndarray:
    """prox_{alpha ||.||_{2,1}} on rows of Z [rows][channels] (Table 2, row 3):
    row_n -> max(||row_n|| - alpha_n, 0) row_n / ||row_n||."""
    nrm = np.linalg.norm(Z, axis=1)
    alpha = np.broadcast_to(np.asarray(alpha, dtype=np.float64), nrm.shape)
    scale = np.where(nrm > 0, np.maximum(nrm - alpha, 0.0) / np.where(nrm > 0, nrm, 1.0), 0.0)
    return Z * scale[:, None]


def proj_l2ball(z: np.ndarray, y: np.ndarray, eps: float) -> np.ndarray:
    """prox of the indicator of B(y, eps) (Table 2, row 4):
    (z - y) / max(||z - y|| / eps, 1) + y."""
    d = z - y
    return d / max(np.linalg.norm(d) / eps, 1.0) + y


def proj_nonneg_real(Z: np.ndarray) -> np.ndarray:
    """prox of the indicator of R_+ (Table 2, row 5): max(0, Re Z)."""
    return np.maximum(0.0, np.real(Z))


def jacobi_svd(A: np.ndarray, tol: float = 1e-15, max_sweeps: int = 60):
    """One-sided (Hestenes) Jacobi SVD of a tall matrix A [m][n], m >= n.

    Cyclic sweeps of plane rotations orthogonalising column pairs of A V,
    stopping when every pair satisfies |a_p . a_q| <= tol sqrt(|a_p|^2 |a_q|^2).
    Returns U [m][n], s [n] (descending), V [n][n] with A = U diag(s) V^T;
    columns of U with s = 0 are zero.
    """
    B = np.array(A, dtype=np.float64, copy=True)
    m, n = B.shape
    V = np.eye(n)
    for _ in range(max_sweeps):
        rotated = False
        for p in range(n - 1):
            for q in range(p + 1, n):
                alpha = B[:, p] @ B[:, p]
                beta = B[:, q] @ B[:, q]
                gamma = B[:, p] @ B[:, q]
                if abs(gamma) <= tol * np.sqrt(alpha * beta) or gamma == 0.0:
                    continue
                rotated = True
                zeta = (beta - alpha) / (2.0 * gamma)
                t = np.sign(zeta) / (abs(zeta) + np.hypot(1.0, zeta)) if zeta != 0 else 1.0
                c = 1.0 / np.sqrt(1.0 + t * t)
                s = c * t
                bp, bq = B[:, p].copy(), B[:, q].copy()
                B[:, p] = c * bp - s * bq
                B[:, q] = s * bp + c * bq
                vp, vq = V[:, p].copy(), V[:, q].copy()
                V[:, p] = c * vp - s * vq
                V[:, q] = s * vp + c * vq
        if not rotated:
            break
    sv = np.linalg.norm(B, axis=0)
    order = np.argsort(-sv, kind="stable")
    sv = sv[order]
    B = B[:, order]
    V = V[:, order]
    U = np.where(sv > 0, B / np.where(sv > 0, sv, 1.0), 0.0)
    return U, sv, V


def prox_weighted_nuclear(Z: np.ndarray, alpha: np.ndarray) -> np.ndarray:
    """prox of sum_j alpha_j s_j(.) (Table 2, row 2 with index-paired thresholds on
    the descending singular values): U diag(max(s_j - alpha_j, 0)) V^T."""
    U, s, V = jacobi_svd(Z)
    return (U * np.maximum(s - alpha, 0.0)) @ V.T


def dual_nuclear(Pq: np.ndarray, DXq: np.ndarray, alpha: np.ndarray) -> np.ndarray:
    """Algorithm 2 nuclear dual: P <- (I - prox_{zeta^-1 mu_bar ||.||_{*,theta_bar}})(P + D_q S~_q X),
    matrices [pixels][channels], alpha_j = zeta^-1 mu_bar theta_bar_j."""
    Z = Pq + DXq
    return Z - prox_weighted_nuclear(Z, alpha)


def dual_l21(Wq: np.ndarray, PsiXq: np.ndarray, alpha: np.ndarray) -> np.ndarray:
    """Algorithm 2 sparsity dual: W <- (I - prox_{kappa^-1 mu ||.||_{2,1,theta}})(W + Psi_q^dagger S_q X),
    matrices [coefficients][channels], alpha_i = kappa^-1 mu theta_i."""
    Z = Wq + PsiXq
    return Z - prox_l21_rows(Z, alpha)


def dual_l2ball(v: np.ndarray, phix: np.ndarray, y: np.ndarray, eps: float) -> np.ndarray:
    """Algorithm 2 data dual with U = I: v <- (I - P_B(y, eps))(v + Phi x_check)."""
    z = v + phix
    return z - proj_l2ball(z, y, eps)


def proj_l2ball_metric(z: np.ndarray, y: np.ndarray, eps: float, U: np.ndarray, n_sub: int) -> np.ndarray:
    """prox^U of the indicator of B(y, eps) (Eq. prox_definition with a diagonal metric
    U > 0), approximated by n_sub forward-backward steps on 1/2 (x - z)^H U (x - z) over
    the ball (Section 3.2: sub-iterations of Euclidean projections): start from the
    Euclidean projection P_B(z), then x <- P_B(x - gamma U (x - z)), gamma = 1 / max U."""
    U = np.asarray(U, dtype=np.float64)
    gamma = 1.0 / U.max()
    x = proj_l2ball(z, y, eps)
    for _ in range(n_sub):
        x = proj_l2ball(x - gamma * U * (x - z), y, eps)
    return x


def dual_l2ball_precond(v: np.ndarray, phix: np.ndarray, y: np.ndarray, eps: float, U: np.ndarray,
                        n_sub: int) -> np.ndarray:
    """Algorithm 2 data dual with a diagonal preconditioner U:
    v <- U (I - prox^U_B(y, eps))(U^-1 v + Phi x_check)."""
    z = v / U + phix
    return U * (z - proj_l2ball_metric(z, y, eps, U, n_sub))
