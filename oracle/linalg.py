"""Ridge least squares pieces of the method, in float64.

Problem (Eq. 1):  x* = argmin f(x),  f(x) = 1/2 ||Ax - b||^2 + nu^2/2 ||x||^2,
A in R^{n x d}, n >= d.  Abar = [A; nu I_d] (Sec. 1.1), so
H = Abar^T Abar = A^T A + nu^2 I and grad f(x) = Abar^T (Abar x - bbar)
= A^T (A x - b) + nu^2 x (the stacked form of Eq. 2 in App. B.1).
"""
import numpy as np


def _f64(a):
    return np.asarray(a, dtype=np.float64)


def objective(A, b, nu, x):
    """f(x) of Eq. 1."""
    A, b, x = _f64(A), _f64(b), _f64(x)
    r = A @ x - b
    return 0.5 * r @ r + 0.5 * nu * nu * x @ x


def gradient(A, b, nu, x):
    """grad f(x) = A^T (A x - b) + nu^2 x.  (App. A.2 writes A^T(Ax_t - b) and
    drops the nu^2 x term; the stacked form of App. B.1 keeps it.)"""
    A, b, x = _f64(A), _f64(b), _f64(x)
    return A.T @ (A @ x - b) + nu * nu * x


def gradient_blocked(A, b, nu, x, block=16384):
    """Same as `gradient`, streaming FP32 rows of a large A in float64 blocks.
    Also returns ||A x||^2."""
    x = _f64(x)
    b = np.asarray(b)
    g = np.zeros(A.shape[1], dtype=np.float64)
    ax2 = 0.0
    for i0 in range(0, A.shape[0], block):
        Ab = _f64(A[i0:i0 + block])
        ax = Ab @ x
        ax2 += ax @ ax
        g += Ab.T @ (ax - _f64(b[i0:i0 + block]))
    return g + nu * nu * x, ax2


def gram_blocked(A, block=16384):
    """A^T A in float64, accumulated over row blocks of A."""
    d = A.shape[1]
    G = np.zeros((d, d), dtype=np.float64)
    for i0 in range(0, A.shape[0], block):
        Ab = _f64(A[i0:i0 + block])
        G += Ab.T @ Ab
    return G


def atb_blocked(A, b, block=16384):
    """A^T b in float64."""
    out = np.zeros(A.shape[1], dtype=np.float64)
    for i0 in range(0, A.shape[0], block):
        out += _f64(A[i0:i0 + block]).T @ _f64(b[i0:i0 + block])
    return out


def direct_solve_dual(A, b, nu):
    """x* = A^T (A A^T + nu^2 I)^{-1} b for n <= d (App. A.2's map x* = A^T z* of
    the dual optimum; equal to Eq. 1's solution by the push-through identity),
    by a float64 Cholesky of the n x n matrix and one step of refinement."""
    A = _f64(A)
    b = _f64(b)
    K = A @ A.T + nu * nu * np.eye(A.shape[0])
    L = np.linalg.cholesky(K)
    z = _chol_solve(L, b)
    z = z + _chol_solve(L, b - K @ z)
    return A.T @ z


def direct_solve(A, b, nu):
    """x* = (A^T A + nu^2 I)^{-1} A^T b (Eq. 1's normal equations) by a float64
    Cholesky factorisation, followed by one step of iterative refinement of the
    normal-equation residual in float64."""
    d = A.shape[1]
    H = gram_blocked(A) + nu * nu * np.eye(d)
    rhs = atb_blocked(A, b)
    L = np.linalg.cholesky(H)
    x = _chol_solve(L, rhs)
    resid = rhs - H @ x
    x = x + _chol_solve(L, resid)
    return x


def direct_solve_path(A, bs, nus):
    """x*_k = (A^T A + nu_k^2 I)^{-1} A^T b_k for a regularisation path on one A
    (Sec. 5's nu-paths): the float64 Gram A^T A is formed once, then each point
    is the Cholesky solve of Eq. 1's normal equations with one refinement step,
    exactly as `direct_solve` does for a single point."""
    d = A.shape[1]
    G = gram_blocked(A)
    out = []
    for b, nu in zip(bs, nus):
        H = G + nu * nu * np.eye(d)
        rhs = atb_blocked(A, b)
        L = np.linalg.cholesky(H)
        x = _chol_solve(L, rhs)
        x = x + _chol_solve(L, rhs - H @ x)
        out.append(x)
    return out


def _chol_solve(L, v):
    import scipy.linalg as sla

    y = sla.solve_triangular(L, v, lower=True)
    return sla.solve_triangular(L.T, y, lower=False)


def svd_solve(U, sigma, V, b, nu):
    """Closed form x* = V diag(sigma / (sigma^2 + nu^2)) U^T b for A = U diag(sigma)
    V^T (App. B.1 notation)."""
    U, sigma, V, b = _f64(U), _f64(sigma), _f64(V), _f64(b)
    return V @ ((sigma / (sigma ** 2 + nu ** 2)) * (U.T @ b))


def effective_dimension_trace(sigma, nu):
    """d_e = tr(A (A^T A + nu^2 I)^{-1} A^T) = sum sigma^2 / (sigma^2 + nu^2) (Sec. 1)."""
    s2 = _f64(sigma) ** 2
    return float(np.sum(s2 / (s2 + nu * nu)))


def effective_dimension_ratio(sigma, nu):
    """d_e = ||D||_F^2 / ||D||_2^2 with D = diag(sigma / sqrt(sigma^2 + nu^2))
    (Sec. 1.1, Notations)."""
    s2 = _f64(sigma) ** 2
    diag2 = s2 / (s2 + nu * nu)
    return float(np.sum(diag2) / np.max(diag2))


def prediction_norm(A, nu, v):
    """||Abar v|| = sqrt(||A v||^2 + nu^2 ||v||^2) (Sec. 1, prediction semi-norm)."""
    v = _f64(v)
    Av = _f64(A) @ v if A.shape[0] <= 65536 else _blocked_matvec(A, v)
    return float(np.sqrt(Av @ Av + nu * nu * v @ v))


def _blocked_matvec(A, v, block=16384):
    out = np.empty(A.shape[0], dtype=np.float64)
    for i0 in range(0, A.shape[0], block):
        out[i0:i0 + block] = _f64(A[i0:i0 + block]) @ v
    return out


def relative_error(A, nu, x, x_star):
    """||Abar (x - x*)|| / ||Abar x*||, the accuracy metric of every solution and the
    square root of delta_t / delta_0 for x_0 = 0 (Sec. 1.1)."""
    x, x_star = _f64(x), _f64(x_star)
    return prediction_norm(A, nu, x - x_star) / prediction_norm(A, nu, x_star)


class WoodburyFactor:
    """Cached factorisation for H_S^{-1} = ((SA)^T SA + nu^2 I_d)^{-1} (Eq. 3).

    m < d : Woodbury form of App. B.4,
            H_S^{-1} = nu^-2 (I_d - (SA)^T (nu^2 I_m + SA (SA)^T)^{-1} SA),
            with a Cholesky factor of the m x m matrix nu^2 I_m + SA (SA)^T.
    m >= d: the d x d matrix (SA)^T SA + nu^2 I_d is factored directly (Sec. 1:
            an exact solve costs O(m d min(m, d))).
    """

    def __init__(self, SA, nu):
        self.SA = _f64(SA)
        self.nu = float(nu)
        m, d = self.SA.shape
        self.woodbury = m < d
        if self.woodbury:
            K = self.nu ** 2 * np.eye(m) + self.SA @ self.SA.T
        else:
            K = self.SA.T @ self.SA + self.nu ** 2 * np.eye(d)
        self.L = np.linalg.cholesky(K)

    def apply(self, g):
        """H_S^{-1} g."""
        g = _f64(g)
        if self.woodbury:
            u = _chol_solve(self.L, self.SA @ g)
            return (g - self.SA.T @ u) / self.nu ** 2
        return _chol_solve(self.L, g)


def sketched_hessian(SA, nu):
    """Dense H_S = (SA)^T SA + nu^2 I_d (Eq. 3), small d only."""
    SA = _f64(SA)
    return SA.T @ SA + nu * nu * np.eye(SA.shape[1])


def newton_decrement(g, gt):
    """r = 1/2 g^T H_S^{-1} g given gt = H_S^{-1} g (Lemma 4.1)."""
    return 0.5 * float(_f64(g) @ _f64(gt))


def c_matrix(U, sigma, nu, S):
    """C_S = D (U^T S^T S U - I) D + I (Sec. 1.1), small n only."""
    U, sigma, S = _f64(U), _f64(sigma), _f64(S)
    Dg = sigma / np.sqrt(sigma ** 2 + nu ** 2)
    SU = S @ U
    inner = SU.T @ SU - np.eye(U.shape[1])
    return (Dg[:, None] * inner * Dg[None, :]) + np.eye(U.shape[1])


def ubar(U, sigma, V, nu):
    """Left singular vectors of Abar: Ubar = [U D; V D'] (App. B.1)."""
    U, sigma, V = _f64(U), _f64(sigma), _f64(V)
    Dg = sigma / np.sqrt(sigma ** 2 + nu ** 2)
    Dp = nu / np.sqrt(sigma ** 2 + nu ** 2)
    return np.vstack([U * Dg[None, :], V * Dp[None, :]])
