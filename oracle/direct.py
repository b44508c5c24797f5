"""Direct sums (oracle ground truth; test infrastructure only).

Eq. (HelmholtzMatrixVector): sigma_i = sum_{j != i} exp(i k |x_i - x_j|) / |x_i - x_j| psi_j,
generalised to targets x_i != sources y_j; a pair is skipped exactly when
|x_i - y_j| == 0 in float64 (this covers j = i when targets alias sources).

Also: the adjoint A^H w (conjugate transpose of the same matrix) and the
gradient of L = sum_i |phi_i - phi*_i|^2 with respect to the source positions,
from d/dy exp(i k R)/R = G (i k - 1/R) (y - x)/R.
"""
import numpy as np


def _pairs(targets, sources):
    d = targets[:, None, :] - sources[None, :, :]
    r = np.sqrt(np.sum(d * d, axis=-1))
    return d, r


def kernel_matrix(targets, sources, kappa):
    """G[i, j] = exp(i k R_ij) / R_ij, 0 where R_ij == 0."""
    _, r = _pairs(targets, sources)
    g = np.zeros(r.shape, dtype=np.complex128)
    nz = r > 0.0
    g[nz] = np.exp(1j * kappa * r[nz]) / r[nz]
    return g


def direct(sources, targets, q, kappa, block=1024):
    """phi = G q, q of shape (ns,) or (ns, R)."""
    sources = np.asarray(sources, dtype=np.float64)
    targets = np.asarray(targets, dtype=np.float64)
    q = np.asarray(q, dtype=np.complex128)
    out = np.zeros((targets.shape[0],) + q.shape[1:], dtype=np.complex128)
    for i0 in range(0, targets.shape[0], block):
        g = kernel_matrix(targets[i0:i0 + block], sources, kappa)
        out[i0:i0 + block] = g @ q
    return out


def direct_adjoint(sources, targets, w, kappa, block=1024):
    """A^H w with A = G (targets x sources): out_j = sum_i conj(G_ij) w_i."""
    sources = np.asarray(sources, dtype=np.float64)
    targets = np.asarray(targets, dtype=np.float64)
    w = np.asarray(w, dtype=np.complex128)
    out = np.zeros((sources.shape[0],) + w.shape[1:], dtype=np.complex128)
    for i0 in range(0, targets.shape[0], block):
        g = kernel_matrix(targets[i0:i0 + block], sources, kappa)
        out += g.conj().T @ w[i0:i0 + block]
    return out


def direct_grad_sources(sources, targets, q, resid, kappa, block=512):
    """dL/dy_j for L = sum_i |phi_i - phi*_i|^2 (single right-hand side).

    resid = phi - phi*.  dL/dy_j = 2 Re[ q_j sum_i conj(resid_i) dG_ij/dy_j ].
    """
    sources = np.asarray(sources, dtype=np.float64)
    targets = np.asarray(targets, dtype=np.float64)
    q = np.asarray(q, dtype=np.complex128)
    resid = np.asarray(resid, dtype=np.complex128)
    grad = np.zeros(sources.shape, dtype=np.float64)
    for i0 in range(0, targets.shape[0], block):
        x = targets[i0:i0 + block]
        d = sources[None, :, :] - x[:, None, :]            # y - x
        r = np.sqrt(np.sum(d * d, axis=-1))
        nz = r > 0.0
        fac = np.zeros(r.shape, dtype=np.complex128)
        rr = r[nz]
        fac[nz] = np.exp(1j * kappa * rr) / rr * (1j * kappa - 1.0 / rr) / rr
        s = np.conj(resid[i0:i0 + block])[:, None] * fac   # [i, j]
        grad += 2.0 * np.real(q[:, None] * np.einsum('ij,ijc->jc', s, d))
    return grad
