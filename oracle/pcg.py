"""Preconditioned conjugate gradients (oracle; test infrastructure only).

Sec. 2 / Sec. 5: K u = f solved by PCG with preconditioner M^{-1}; stop when the
residual is reduced by `rtol` relative to ||f|| (x0 = 0 makes this the paper's
"relative norm of the initial residual").  The condition number of M^{-1}K is
estimated from the CG coefficients by the Lanczos connection (Sec. 5, Saad
ch. 6).

Energy-error stopping (a reading added here because rtol alone does not bound
the K-norm error when cond(K) is large): with d = 4 the quantity
    sum_{j=k}^{k+d-1} alpha_j r_j^T z_j
estimates ||u* - u_k||_K^2 (Strakos-Tichy); the iteration also requires this
estimate, for the iterate d steps back, to fall below (etol)^2 * f^T u.
"""
from __future__ import annotations

import numpy as np


def lanczos_cond(alphas, betas):
    """Extreme eigenvalues of the CG Lanczos tridiagonal T_k:
    T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1},  T_{j,j+1} = sqrt(beta_j)/alpha_j."""
    k = len(alphas)
    if k == 0:
        return float("nan"), float("nan"), float("nan")
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < k:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(betas[j]) / alphas[j]
    ev = np.linalg.eigvalsh(T)
    return ev[-1] / ev[0], ev[0], ev[-1]


def pcg(Kop, f, Minv=None, rtol=1e-8, etol=None, maxit=10000, x0=None, delay=4, flexible=False):
    """Returns (x, info).  Kop(x) applies K (Dirichlet rows as identity and
    f = 0 there), Minv(r) the preconditioner (None = identity).  etol: relative
    energy-error target (None = 0.1 * rtol; 0 disables the energy test)."""
    if etol is None:
        etol = 0.1 * rtol
    Minv = Minv or (lambda r: r.copy())
    x = np.zeros_like(f) if x0 is None else x0.copy()
    r = f - Kop(x) if x0 is not None else f.copy()
    nf = np.linalg.norm(f)
    z = Minv(r)
    p = z.copy()
    rz = float(r @ z)
    alphas, betas, used, terms, hist = [], [], [], [], [np.linalg.norm(r) / nf if nf > 0 else 0.0]
    it = 0
    converged = nf == 0.0
    energy_est = float("nan")
    while not converged and it < maxit:
        q = Kop(p)
        pq = float(p @ q)
        if not pq > 0.0:
            break
        alpha = rz / pq
        x += alpha * p
        r -= alpha * q
        alphas.append(alpha)
        terms.append(alpha * rz)
        it += 1
        rel = np.linalg.norm(r) / nf
        hist.append(rel)
        ok_e = True
        if etol > 0.0:
            if len(terms) >= delay:
                energy_est = float(sum(terms[-delay:]))
                ok_e = energy_est <= etol * etol * float(f @ x)
            else:
                ok_e = False
        if rel <= rtol and ok_e:
            converged = True
            break
        zn = Minv(r)
        rzn = float(r @ zn)
        if flexible:
            beta = float(r @ (zn - z)) / rz
        else:
            beta = rzn / rz
        # the Lanczos connection is stated for the PCG coefficients, so the
        # condition estimate takes r_{k+1}^T z_{k+1} / r_k^T z_k in both variants
        betas.append(rzn / rz)
        used.append(beta)
        z = zn
        p = zn + beta * p
        rz = rzn
    cond, lmin, lmax = lanczos_cond(alphas, betas)
    return x, dict(iters=it, converged=converged, rel_res=hist[-1], history=hist,
                   cond=cond, lmin=lmin, lmax=lmax, energy_est=energy_est,
                   alphas=alphas, betas=betas, betas_used=used)


def energy_error(K, u, u_ref):
    """Relative K-norm error ||u - u*||_K / ||u*||_K computed from the error
    vector itself (never from compliance differences)."""
    e = u - u_ref
    return float(np.sqrt(max(e @ (K @ e), 0.0) / (u_ref @ (K @ u_ref))))
