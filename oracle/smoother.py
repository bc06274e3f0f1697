"""Scaled Chebyshev-Jacobi smoothers and the inexact symmetric Uzawa step (oracle, FP64).

Sec. 3.3.1.  For M x = b with Jacobi preconditioner D the Chebyshev-Jacobi
semi-iteration started from zero gives x = s_k(D^{-1} M) D^{-1} b with
s_k(t) = (1 - T_{k+1}(t))/t and T_{k+1}(t) = C_{k+1}((beta+alpha-2t)/(beta-alpha)) /
C_{k+1}((beta+alpha)/(beta-alpha)), [alpha, beta] = [beta/2, beta].  It is run by the
classical three-term Chebyshev recurrence and uses k applications of M; k = 0 is
damped Jacobi with omega = 2/(alpha+beta).

Lemma 1 and Algorithm 2: A^-1_hat = sigma Cheb(A, D_A, k_A) and
S^-1_hat = tau Cheb(S_tilde, D_S, k_S) with S_tilde = B A^-1_hat B^T (C = 0) and
sigma, tau = C_{k+1}(3) / (1 + C_{k+1}(3)).  beta comes from a Lanczos estimate of
lambda_max times a safety factor (the paper only asks for a close approximation).

Smoother, compact form (Sec. 3.3.1, K_hat): x <- x + K_hat^{-1}(b - K x), run as
    u_hat = u + A^-1_hat (f - A u - B^T p)
    dp    = S^-1_hat (B u_hat - g)
    u     = u_hat - A^-1_hat B^T dp
    p     = p + dp
(the three-line form printed in the introduction uses A u_hat and p^j in its last
line, which does not match K_hat; the compact form is the one the analysis uses).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from .assemble import Tables, element_matrices

MASK64 = (1 << 64) - 1


def splitmix64_uniform(seed, n):
    """Uniform(-1,1) values u_i, i < n, from the SplitMix64 generator (Steele, Lea, Flood 2014).

    z = seed + (i+1) * 0x9E3779B97F4A7C15 (mod 2^64), then the SplitMix64 output
    mix; u = 2 * (z >> 11) * 2^-53 - 1.  Used only to draw Lanczos start vectors.
    numpy uint64 arithmetic wraps modulo 2^64, which is the generator's definition.
    """
    i = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + i * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return 2.0 * ((z >> np.uint64(11)).astype(np.float64) * 2.0**-53) - 1.0


def cheb_C(n, s):
    """Chebyshev polynomial of the first kind C_n(s) by the three-term recurrence."""
    c0, c1 = 1.0, s
    if n == 0:
        return c0
    for _ in range(n - 1):
        c0, c1 = c1, 2.0 * s * c1 - c0
    return c1


def lemma1_scaling(k, s_bar=3.0):
    """sigma (or tau) = C_{k+1}(s_bar) / (1 + C_{k+1}(s_bar)) = c_1 of Lemma 1."""
    c = cheb_C(k + 1, s_bar)
    return c / (1.0 + c)


def chebyshev(apply_M, Dinv, r, k, beta, alpha=None):
    """Cheb(M, D, k) r: the Chebyshev-Jacobi semi-iteration for M x = r from x = 0.

    theta = (beta+alpha)/2, delta = (beta-alpha)/2, s1 = theta/delta, rho_0 = 1/s1;
    d_0 = D^{-1} r / theta, x_1 = d_0; for j = 1..k:
        rho_j = 1/(2 s1 - rho_{j-1}),
        d_j = rho_j rho_{j-1} d_{j-1} + (2 rho_j / delta) D^{-1}(r - M x_j),
        x_{j+1} = x_j + d_j.
    """
    if alpha is None:
        alpha = 0.5 * beta
    theta = 0.5 * (beta + alpha)
    delta = 0.5 * (beta - alpha)
    s1 = theta / delta
    rho = 1.0 / s1
    d = Dinv * r / theta
    x = d.copy()
    for _ in range(k):
        rho_new = 1.0 / (2.0 * s1 - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * (Dinv * (r - apply_M(x)))
        x = x + d
        rho = rho_new
    return x


def lanczos_max(apply_S, v0, steps):
    """Largest Ritz value of `steps` plain Lanczos steps on the symmetric operator apply_S."""
    v = v0 / np.linalg.norm(v0)
    v_prev = np.zeros_like(v)
    b_prev = 0.0
    alphas, betas = [], []
    for j in range(steps):
        w = apply_S(v) - b_prev * v_prev
        a = float(w @ v)
        w = w - a * v
        alphas.append(a)
        b = float(np.linalg.norm(w))
        if j == steps - 1 or b <= 1e-14 * max(abs(a), 1.0):
            break
        betas.append(b)
        v_prev, v, b_prev = v, w / b, b
    T = np.diag(alphas) + np.diag(betas[: len(alphas) - 1], 1) + np.diag(betas[: len(alphas) - 1], -1)
    return float(np.linalg.eigvalsh(T)[-1])


def local_schur_diag(level, mu, gamma_rho, mu_cell=None, chunk=4096, rho_cell=None, sym=False):
    """D_S_loc = sum_tau P_tau^T diag(B_tau diag(A_tau)^{-1} B_tau^T) P_tau  (Eq. diag loc).

    A_tau is the cell's velocity block (the same scalar block per component, or the coupled block
    of the symmetric form); B_tau excludes constrained velocity DoFs (their columns of B are zero
    globally).
    """
    tab = Tables(level.dim, level.k)
    vn = level.cell_velocity_nodes()
    pn = level.cell_pressure_nodes()
    vmask = level.velocity_constrained()
    out = np.zeros(level.n_p)
    for s in range(0, level.n_cells, chunk):
        cells = np.arange(s, min(s + chunk, level.n_cells))
        E = element_matrices(level, tab, mu, gamma_rho, mu_cell, cells, rho_cell, sym)
        free = (~vmask[vn[cells]]).astype(np.float64)           # (nc, nphi)
        B = E["B"]                                              # (nc, npsi, d, nphi)
        if sym:
            diagA = np.einsum("kcici->kci", E["Af"])             # (nc, d, nphi)
            loc = np.einsum("ciaj,caj->ci", B**2, free[:, None, :] / diagA)
        else:
            diagA = np.einsum("cii->ci", E["As"])              # (nc, nphi)
            loc = np.einsum("ciaj,cj->ci", B**2, free / diagA)
        np.add.at(out, pn[cells], loc)
    return out


class LevelSmoother:
    """Algorithm 2 on one level plus the smoother and its building blocks."""

    def __init__(self, level, ops, kA, kS, schur_diag="loc", mu=1.0, gamma_rho=0.0, mu_cell=None,
                 eig_steps=40, eig_safety=1.1, seed=0x5EED, beta_A=None, beta_S=None, rho_cell=None, sym=False):
        self.level, self.ops = level, ops
        self.kA, self.kS = kA, kS
        self.A, self.B = ops["A"], ops["B"]
        self.C = ops.get("C")
        if self.C is None:
            self.C = sp.csr_matrix((level.n_p, level.n_p))
        pker = ops.get("pker", level.has_pressure_kernel())
        self.BT = self.B.T.tocsr()
        self.n_u = level.n_u
        self.DA = self.A.diagonal().copy()
        self.DAinv = 1.0 / self.DA
        free_u = ~ops["umask"]
        # --- velocity part (Algorithm 2, first block) -------------------------------
        if beta_A is None:
            v0 = splitmix64_uniform(seed, self.n_u) * free_u
            sq = np.sqrt(self.DAinv)
            beta_A = eig_safety * lanczos_max(lambda v: sq * (self.A @ (sq * v)), v0, eig_steps)
        self.beta_A = beta_A
        self.sigma = lemma1_scaling(kA)
        # --- pressure part -------------------------------------------------------------
        # D_S~ approximates the diagonal of S~ = B A^-1_hat B^T + C (Sec. 1): each variant of the
        # first term plus diag(C)
        if schur_diag == "loc":
            DS = local_schur_diag(level, mu, gamma_rho, mu_cell, rho_cell=rho_cell, sym=sym)
        elif schur_diag == "p":
            DS = ops["Mp"].diagonal().copy()
        elif schur_diag == "d":
            DS = np.asarray((self.B.multiply(self.B)) @ self.DAinv).reshape(-1)
        elif schur_diag == "exact":
            Ainv_hat = self.dense_Ainv_hat()
            Bd = self.B.toarray()
            DS = np.einsum("ij,jk,ik->i", Bd, Ainv_hat, Bd)
        else:
            raise ValueError(schur_diag)
        DS = DS + self.C.diagonal()
        self.DS = DS
        self.DSinv = 1.0 / DS
        if beta_S is None:
            v0 = splitmix64_uniform(seed + 1, level.n_p)
            sq = np.sqrt(self.DSinv)
            if pker:
                z = np.sqrt(DS)
                v0 = v0 - (v0 @ z) / (z @ z) * z
            beta_S = eig_safety * lanczos_max(lambda v: sq * self.S_tilde(sq * v), v0, eig_steps)
        self.beta_S = beta_S
        self.tau = lemma1_scaling(kS)

    # --- building blocks -----------------------------------------------------------------
    def Ainv_hat(self, r):
        return self.sigma * chebyshev(lambda x: self.A @ x, self.DAinv, r, self.kA, self.beta_A)

    def S_tilde(self, q):
        return self.B @ self.Ainv_hat(self.BT @ q) + self.C @ q

    def Sinv_hat(self, r):
        return self.tau * chebyshev(self.S_tilde, self.DSinv, r, self.kS, self.beta_S)

    def dense_Ainv_hat(self):
        return np.stack([self.Ainv_hat(e) for e in np.eye(self.n_u)], axis=1)

    def dense_Sinv_hat(self):
        return np.stack([self.Sinv_hat(e) for e in np.eye(self.level.n_p)], axis=1)

    # --- smoother (compact form) ------------------------------------------------------
    def step(self, x, b):
        nu = self.n_u
        u, p = x[:nu], x[nu:]
        f, g = b[:nu], b[nu:]
        u_hat = u + self.Ainv_hat(f - self.A @ u - self.BT @ p)
        dp = self.Sinv_hat(self.B @ u_hat - self.C @ p - g)
        u_new = u_hat - self.Ainv_hat(self.BT @ dp)
        return np.concatenate([u_new, p + dp])

    def smooth(self, x, b, m):
        for _ in range(m):
            x = self.step(x, b)
        return x


def schur_diag_options():
    return ("loc", "p", "d", "exact")


def cheb_scalar_error(t, k, beta, alpha=None):
    """Closed-form T_{k+1}(t) for scalar t: the error factor of Cheb(M, D, k)."""
    if alpha is None:
        alpha = 0.5 * beta

    def C(n, s):
        s = np.asarray(s, dtype=np.float64)
        out = np.empty_like(s)
        inside = np.abs(s) <= 1
        out[inside] = np.cos(n * np.arccos(s[inside]))
        so = s[~inside]
        out[~inside] = np.sign(so) ** n * np.cosh(n * np.arccosh(np.abs(so)))
        return out

    s = (beta + alpha - 2.0 * np.asarray(t)) / (beta - alpha)
    return C(k + 1, s) / C(k + 1, np.array([(beta + alpha) / (beta - alpha)]))[0]
