"""Independent FP64 Ewald summation (oracle; test infrastructure).

Sec. 4 compares the method with an Ewald sum taken as exact.  This one is
converged far below the paper's settings (a^2 = 6.25, two images, four modes):
the split parameter, real-space cutoff and k-space cutoff are chosen so both
truncated tails are below ~1e-16 of the terms kept.

    Phi_i = sum_j sum_n' Q_j erfc(alpha |r_ij + nL|) / |r_ij + nL|
          + (4 pi / V) sum_{k != 0} exp(-k^2 / 4 alpha^2) / k^2 Re[S(k) exp(-i k.x_i)]
          - 2 alpha / sqrt(pi) Q_i  -  pi (sum Q) / (alpha^2 V),
    S(k) = sum_j Q_j exp(i k.x_j),
tin-foil boundary, k = 0 omitted, the last term the uniform neutralising background.
Forces are -Q_i grad Phi at x_i (self and background terms have no gradient).
"""
import numpy as np
from scipy.special import erfc


def ewald(pos, Q, L, targets=None, alpha_L=6.5, chunk=256, want_grad=False):
    """Potential (and gradient) at the charges listed in targets (default all)."""
    pos = np.asarray(pos, dtype=np.float64) % L
    Q = np.asarray(Q, dtype=np.float64)
    N = len(Q)
    tg = np.arange(N) if targets is None else np.asarray(targets)
    alpha = alpha_L / L
    rcut = 6.6 / alpha                       # erfc(6.6) ~ 1e-20
    kcut = 2.0 * alpha * np.sqrt(44.0)       # exp(-44) ~ 8e-20
    nk = int(np.ceil(kcut * L / (2 * np.pi)))
    V = L ** 3
    # minimum-image displacements lie in [-L/2, L/2]^3; keep the lattice shifts that can
    # bring such a displacement within rcut
    nimg = int(np.ceil(rcut / L - 0.5))
    cand = np.array([(a, b, c) for a in range(-nimg, nimg + 1)
                     for b in range(-nimg, nimg + 1) for c in range(-nimg, nimg + 1)], float) * L
    gap = np.maximum(np.abs(cand) - 0.5 * L, 0.0)
    shifts = cand[np.sqrt((gap ** 2).sum(axis=1)) < rcut]
    phi = np.zeros(len(tg))
    grad = np.zeros((len(tg), 3))
    # real space: minimum image then the shifts that can fall within rcut
    for s0 in range(0, len(tg), chunk):
        ti = tg[s0:s0 + chunk]
        d0 = pos[None, :, :] - pos[ti, None, :]
        d0 -= L * np.round(d0 / L)
        for sh in shifts:
            d = d0 + sh
            r = np.sqrt(np.einsum('tjk,tjk->tj', d, d))
            keep = (r < rcut) & (r > 0.0)
            rr = np.where(keep, r, 1.0)
            e = np.where(keep, erfc(alpha * rr) / rr, 0.0)
            phi[s0:s0 + chunk] += e @ Q
            if want_grad:
                # d/dx_i of erfc(alpha r)/r with r = |x_j - x_i|: -(d/dr) (x_j - x_i)/r
                dfdr = -erfc(alpha * rr) / rr ** 2 - 2 * alpha / np.sqrt(np.pi) * np.exp(-(alpha * rr) ** 2) / rr
                coef = np.where(keep, -dfdr / rr, 0.0) * Q[None, :]
                grad[s0:s0 + chunk] += np.einsum('tj,tjk->tk', coef, d)
    # reciprocal space with separable exponentials
    m = np.arange(-nk, nk + 1)
    kv = 2 * np.pi * m / L
    E = [np.exp(1j * np.outer(pos[:, a], kv)) for a in range(3)]          # (N, 2nk+1)
    S = np.zeros((len(m),) * 3, dtype=complex)
    for s0 in range(0, N, 4096):
        sl = slice(s0, s0 + 4096)
        A = (Q[sl, None, None] * E[0][sl, :, None] * E[1][sl, None, :]).reshape(E[0][sl].shape[0], -1)
        S += (A.T @ E[2][sl]).reshape(len(m), len(m), len(m))
    KX, KY, KZ = np.meshgrid(kv, kv, kv, indexing='ij')
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    k2[nk, nk, nk] = 1.0
    f = (4 * np.pi / V) * np.exp(-k2 / (4 * alpha ** 2)) / k2
    f[k2 > kcut ** 2] = 0.0
    f[nk, nk, nk] = 0.0
    FS = f * S
    Et = [np.conj(E[a][tg]) for a in range(3)]
    for s0 in range(0, len(tg), chunk):
        sl = slice(s0, s0 + chunk)
        z = np.einsum('abc,tc->tab', FS, Et[2][sl])
        z = np.einsum('tab,tb->ta', z, Et[1][sl])
        val = np.einsum('ta,ta->t', z, Et[0][sl])
        phi[sl] += val.real
        if want_grad:
            for a, K in enumerate((KX, KY, KZ)):
                z = np.einsum('abc,tc->tab', FS * K, Et[2][sl])
                z = np.einsum('tab,tb->ta', z, Et[1][sl])
                grad[sl, a] += np.einsum('ta,ta->t', z, Et[0][sl]).imag
    phi += -2 * alpha / np.sqrt(np.pi) * Q[tg] - np.pi * Q.sum() / (alpha ** 2 * V)
    if want_grad:
        return phi, grad
    return phi


def ewald_energy(pos, Q, L, **kw):
    """U = 1/2 sum Q_i Phi_i (Eq. potentialenergy) with the Ewald potentials."""
    return 0.5 * float(np.dot(Q, ewald(pos, Q, L, **kw)))
