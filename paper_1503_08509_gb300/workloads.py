"""Seeded synthetic particle sets shaped like the paper's tests.

This module only draws random numbers and lays out geometry; it holds none of
the method's arithmetic, so both the CUDA path and the CPU oracle can be fed
from it.  All generators use numpy's PCG64 (``default_rng(seed)``) and return
float64 positions (N, 3) in [0, L) and float64 charges (N,).

The paper's own accuracy workload (Sec. 4) is ``two_biased_cubes``; the others
are the standard test shapes the method is benchmarked on: uniform random
charges, a jittered rock-salt lattice (closed-form Madelung energy), neutral
water-like triplets and Gaussian clusters over a uniform background.
"""
import numpy as np


def uniform_pm(N, L=1.0, seed=1):
    """N uniform-random charges in [0, L)^3, exactly N/2 of +1 and N/2 of -1 in random order."""
    rng = np.random.default_rng(seed)
    pos = rng.random((N, 3)) * L
    Q = np.ones(N)
    Q[N // 2:] = -1.0
    rng.shuffle(Q)
    return pos, Q


def rock_salt(m, L=1.0, jitter=1e-3, seed=2, offset=0.0):
    """m^3 ions on a simple-cubic grid of spacing L/m, charge (-1)^(i+j+k), each coordinate
    jittered by U[-jitter, jitter] * L, plus a common offset (in units of L/m)."""
    rng = np.random.default_rng(seed)
    a = L / m
    I, J, K = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing='ij')
    idx = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1)
    pos = (idx + offset) * a
    if jitter:
        pos = pos + rng.uniform(-jitter, jitter, size=pos.shape) * L
    Q = np.where(idx.sum(axis=1) % 2 == 0, 1.0, -1.0)
    return np.mod(pos, L), Q


def water_triplets(n_mol, density=33.4, r_oh=0.1, angle_deg=109.47, seed=3):
    """n_mol neutral triplets (O -0.8476 at the centre, two H +0.4238 at r_oh, H-O-H angle),
    uniformly random centres at `density` molecules per unit volume and random orientations
    (uniform random unit quaternions).  Returns pos, Q, L."""
    rng = np.random.default_rng(seed)
    L = (n_mol / density) ** (1.0 / 3.0)
    cen = rng.random((n_mol, 3)) * L
    th = np.deg2rad(angle_deg) / 2
    body = np.array([[np.sin(th), 0.0, np.cos(th)], [-np.sin(th), 0.0, np.cos(th)]]) * r_oh
    q = rng.normal(size=(n_mol, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], 1)
    h1 = cen + np.einsum('nij,j->ni', R, body[0])
    h2 = cen + np.einsum('nij,j->ni', R, body[1])
    pos = np.empty((3 * n_mol, 3))
    pos[0::3], pos[1::3], pos[2::3] = cen, h1, h2
    Q = np.tile([-0.8476, 0.4238, 0.4238], n_mol)
    return np.mod(pos, L), Q, L


def gaussian_blobs(N, n_blobs=64, sigma=0.02, background=0.2, L=1.0, seed=5):
    """N charges (+1/-1, exactly half each, randomly assigned): a fraction `background`
    uniform, the rest split evenly over n_blobs Gaussian clusters of width sigma*L at
    uniform-random centres, wrapped periodically."""
    rng = np.random.default_rng(seed)
    n_bg = int(round(background * N))
    n_bl = N - n_bg
    cen = rng.random((n_blobs, 3)) * L
    which = np.repeat(np.arange(n_blobs), int(np.ceil(n_bl / n_blobs)))[:n_bl]
    blob = cen[which] + rng.normal(scale=sigma * L, size=(n_bl, 3))
    pos = np.concatenate([blob, rng.random((n_bg, 3)) * L])
    Q = np.ones(N)
    Q[N // 2:] = -1.0
    rng.shuffle(Q)
    return np.mod(pos, L), Q


def two_biased_cubes(N, seed=6):
    """Sec. 4 workload: half the charges uniform in [0,1/2]^3 with 55% +1 / 45% -1, half in
    [1/2,1]^3 with 45% +1 / 55% -1 (neutral overall for N divisible by 40), L = 1."""
    rng = np.random.default_rng(seed)
    h = N // 2
    a = rng.random((h, 3)) * 0.5
    b = 0.5 + rng.random((N - h, 3)) * 0.5
    na = int(round(0.55 * h))
    qa = np.r_[np.ones(na), -np.ones(h - na)]
    nb = int(round(0.45 * (N - h)))
    qb = np.r_[np.ones(nb), -np.ones(N - h - nb)]
    rng.shuffle(qa)
    rng.shuffle(qb)
    return np.concatenate([a, b]), np.concatenate([qa, qb])


# Named workloads: (generator, mesh elements per axis, description)
def box_charges(N, L=1.0, seed=7, on_faces=6):
    """N charges in the closed box [0, L]^3 for the Dirichlet problem: uniform positions,
    charges +1 / -1 drawn independently (not neutral), and the first on_faces charges moved
    onto the faces, one per face in turn (coordinate 0 or exactly L)."""
    rng = np.random.default_rng(seed)
    pos = rng.random((N, 3)) * L
    Q = rng.choice([-1.0, 1.0], size=N)
    for k in range(min(on_faces, N)):
        pos[k, k % 3] = 0.0 if (k // 3) % 2 == 0 else L
    return pos, Q


def workload(name):
    """Return dict(pos, Q, L, n_el, label) for a named workload."""
    if name == 'uniform1k':
        pos, Q = uniform_pm(1000, seed=1)
        return dict(pos=pos, Q=Q, L=1.0, n_el=16, label='N=1000 uniform +/-1, L=1, 16^3 mesh')
    if name == 'nacl32':
        pos, Q = rock_salt(32, jitter=1e-3, seed=2)
        return dict(pos=pos, Q=Q, L=1.0, n_el=32, label='rock-salt 32^3 ions, jitter 1e-3 L, 32^3 mesh')
    if name == 'water1m':
        pos, Q, L = water_triplets(333333, seed=3)
        return dict(pos=pos, Q=Q, L=L, n_el=128, label='333333 water triplets (999999 atoms), 128^3 mesh')
    if name == 'uniform262k':
        pos, Q = uniform_pm(262144, seed=4)
        return dict(pos=pos, Q=Q, L=1.0, n_el=64, label='N=262144 uniform +/-1, 64^3 mesh')
    if name == 'blobs4m':
        pos, Q = gaussian_blobs(4_000_000, seed=5)
        return dict(pos=pos, Q=Q, L=1.0, n_el=256, label='N=4e6 in 64 Gaussian blobs + 20% background, 256^3 mesh')
    raise KeyError(name)
