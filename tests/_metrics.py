"""Comparison helpers shared by the parity tests (test code only).

Singular vectors are unique only up to sign, and only as a subspace inside a
cluster of (near-)equal singular values (section III of the paper: U equals
the proxy's U up to a block-diagonal unitary W).  So:
  * sigma is compared elementwise: relative error for sigma > 1e-10 sigma_1,
    absolute error (as a fraction of sigma_1) below that;
  * vectors are grouped into clusters whose neighbouring sigma differ by less
    than ``gap`` * sigma_1; a singleton cluster is compared by the sine of its
    principal angle, a larger one by the 2-norm distance of its projectors.
"""
import numpy as np


def sigma_check(s, s_ref, rel_tol, abs_tol):
    s = np.asarray(s, dtype=np.float64)
    s_ref = np.asarray(s_ref, dtype=np.float64)
    assert s.shape == s_ref.shape, (s.shape, s_ref.shape)
    s1 = max(float(s_ref[0]), 1e-300)
    big = s_ref > 1e-10 * s1
    rel = np.abs(s[big] - s_ref[big]) / s_ref[big] if big.any() else np.zeros(0)
    small = np.abs(s[~big]) / s1 if (~big).any() else np.zeros(0)
    worst_rel = float(rel.max()) if rel.size else 0.0
    worst_abs = float(small.max()) if small.size else 0.0
    assert worst_rel <= rel_tol, f"sigma relative error {worst_rel:.3e} > {rel_tol:.1e}"
    assert worst_abs <= abs_tol, f"tiny sigma absolute error {worst_abs:.3e} > {abs_tol:.1e}"
    return worst_rel, worst_abs


def clusters(s_ref, gap=1e-3, floor=1e-8):
    """Index groups of the singular values above floor * sigma_1."""
    s1 = max(float(s_ref[0]), 1e-300)
    idx = [i for i in range(len(s_ref)) if s_ref[i] > floor * s1]
    out, cur = [], []
    for i in idx:
        if cur and (s_ref[cur[-1]] - s_ref[i]) >= gap * s1:
            out.append(cur)
            cur = []
        cur.append(i)
    if cur:
        out.append(cur)
    return out


def subspace_check(X, X_ref, s_ref, tol, gap=1e-3, floor=1e-8):
    """Largest principal-angle sine (singletons) / projector distance
    (clusters) between the columns of X and X_ref, over sigma clusters."""
    X = np.asarray(X, dtype=np.float64)
    X_ref = np.asarray(X_ref, dtype=np.float64)
    worst = 0.0
    for c in clusters(s_ref, gap, floor):
        A = X[:, c]
        B = X_ref[:, c]
        if len(c) == 1:
            a = A[:, 0] / max(np.linalg.norm(A[:, 0]), 1e-300)
            b = B[:, 0] / max(np.linalg.norm(B[:, 0]), 1e-300)
            err = float(np.linalg.norm(a - (a @ b) * b))
        else:
            Qa, _ = np.linalg.qr(A)
            Qb, _ = np.linalg.qr(B)
            # || (I - Qb Qb^T) Qa ||_2 = sine of the largest principal angle
            E = Qa - Qb @ (Qb.T @ Qa)
            err = float(np.linalg.norm(E, 2))
        worst = max(worst, err)
    assert worst <= tol, f"subspace error {worst:.3e} > {tol:.1e}"
    return worst


def orthonormality(X):
    X = np.asarray(X, dtype=np.float64)
    return float(np.abs(X.T @ X - np.eye(X.shape[1])).max())


def sparse_csc(col_ptr, row_idx, vals, M):
    """scipy CSC matrix of the input (test-side products at full size)."""
    import scipy.sparse as sp
    N = len(col_ptr) - 1
    return sp.csc_matrix((np.asarray(vals, dtype=np.float64), np.asarray(row_idx),
                          np.asarray(col_ptr)), shape=(M, N))


def gram_angle_bounds(A, s, U):
    """Davis-Kahan bounds on the angle between each computed u_i and the true
    eigenvector of A A^T: r_i = |A A^T u_i - s_i^2 u_i| (FP64 sparse products),
    every true eigenvalue lies within r_j of some s_j^2, so the separation of
    s_i^2 from the other true eigenvalues is at least
    g_i = min_{j != i} |s_i^2 - s_j^2| - r_i - max_j r_j, and
    sin(angle_i) <= r_i / g_i (inf where g_i <= 0)."""
    U = np.asarray(U, dtype=np.float64)
    lam = np.asarray(s, dtype=np.float64) ** 2
    r = np.zeros(len(lam))
    for c0 in range(0, len(lam), 64):
        Uc = U[:, c0:c0 + 64]
        R = A @ (A.T @ Uc) - Uc * lam[None, c0:c0 + 64]
        r[c0:c0 + 64] = np.linalg.norm(R, axis=0)
    out = np.full(len(lam), np.inf)
    rmax = float(r.max())
    for i in range(len(lam)):
        d = np.abs(lam - lam[i])
        d[i] = np.inf
        g = float(d.min()) - r[i] - rmax
        if g > 0:
            out[i] = r[i] / g
    return out, r


def separated(s, gap=1e-3):
    """Indices whose sigma is at least gap * sigma_1 from both neighbours."""
    s = np.asarray(s, dtype=np.float64)
    s1 = float(s[0])
    keep = []
    for i in range(len(s)):
        if i > 0 and s[i - 1] - s[i] < gap * s1:
            continue
        if i + 1 < len(s) and s[i] - s[i + 1] < gap * s1:
            continue
        keep.append(i)
    return np.asarray(keep, dtype=np.int64)
