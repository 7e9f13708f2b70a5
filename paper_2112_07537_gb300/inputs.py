"""Seeded synthetic inputs: octree leaf sets and analytic fields.

This module only builds inputs.  It holds none of the multiresolution
arithmetic (no filters, no ghosts, no stencils) and is shared by the tests,
the benchmark and the oracle checks.  Leaves are returned as (lev[n],
anc[n,3]) with the anchor in block units of the leaf's own level, in no
particular order.  Every domain is a periodic forest of nt[0] x nt[1] x nt[2]
trees of edge ``tree_len``; point i of a level-L block with anchor a sits at
x = (a*nb + i) * tree_len / (nb * 2^L).
"""
from __future__ import annotations

import numpy as np


# ---------------------------------------------------------------- leaf sets
def uniform_leaves(nt, level):
    n = [t << level for t in nt]
    z, y, x = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    anc = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).astype(np.int32)
    return np.full(len(anc), level, np.int32), anc


def refine_leaves(lev, anc, mask):
    """Replace every leaf with mask=True by its 8 children."""
    out_l, out_a = [], []
    for L, a, m in zip(lev, anc, mask):
        if m:
            for c in range(8):
                out_l.append(L + 1)
                out_a.append([2 * a[0] + (c & 1), 2 * a[1] + ((c >> 1) & 1), 2 * a[2] + (c >> 2)])
        else:
            out_l.append(L)
            out_a.append(list(a))
    return np.asarray(out_l, np.int32), np.asarray(out_a, np.int32).reshape(-1, 3)


def _boxes(lev, anc, finest):
    s = (1 << (finest - lev)).astype(np.int64)[:, None]
    lo = anc.astype(np.int64) * s
    return lo, lo + s


def balance(nt, lev, anc, max_iter=64):
    """Refine until adjacent leaves (face, edge or corner, periodic) differ by
    at most one level.  Brute force over leaf pairs: for input building only."""
    for _ in range(max_iter):
        finest = int(lev.max())
        lo, hi = _boxes(lev, anc, finest)
        P = np.asarray([t << finest for t in nt], np.int64)
        need = np.zeros(len(lev), bool)
        for i in range(len(lev)):
            # leaves touching leaf i (closed boxes, periodic images)
            touch = np.ones(len(lev), bool)
            for d in range(3):
                dl = lo[:, d] - hi[i, d]
                dh = lo[i, d] - hi[:, d]
                ok = np.zeros(len(lev), bool)
                for sh in (-P[d], 0, P[d]):
                    ok |= (lo[:, d] + sh <= hi[i, d]) & (lo[i, d] <= hi[:, d] + sh)
                touch &= ok
                del dl, dh
            touch[i] = False
            if np.any(lev[touch] > lev[i] + 1):
                need[i] = True
        if not need.any():
            return lev, anc
        lev, anc = refine_leaves(lev, anc, need)
    raise RuntimeError("balance did not converge")


def bounded_test_tree(nt=(4, 4, 4)):
    """A 3-level 2:1 tree whose refinement reaches the domain faces: level 1
    in the trees with x-index <= 1 and y-index 1..2 (a slab on the x = 0
    face), level 2 in the level-1 leaf at (0, 2, 0) (on the x = 0, z = 0
    edge), then balanced."""
    lev, anc = uniform_leaves(nt, 0)
    lev, anc = refine_leaves(lev, anc, (anc[:, 0] <= 1) & (anc[:, 1] >= 1) & (anc[:, 1] <= 2))
    lev, anc = refine_leaves(lev, anc, (lev == 1) & np.all(anc == (0, 2, 0), axis=1))
    return balance(nt, lev, anc)


def block_centres(nt, tree_len, lev, anc):
    size = tree_len / (1 << lev.astype(np.int64))
    return (anc + 0.5) * size[:, None], size


def refine_in_ball(nt, tree_len, lev, anc, centre, radius, level):
    """Refine leaves at `level` whose box intersects the periodic ball."""
    c, size = block_centres(nt, tree_len, lev, anc)
    ext = np.asarray(nt, float) * tree_len
    d = np.abs(c - np.asarray(centre))
    d = np.minimum(d, ext - d)
    d = np.maximum(d - 0.5 * size[:, None], 0.0)
    hit = (np.sqrt((d ** 2).sum(1)) <= radius) & (lev == level)
    return refine_leaves(lev, anc, hit)


def tree_config1():
    """Unit cube of 2x2x2 trees (edge 0.5), nb=16; tree (0,0,0) refined once:
    7 root leaves + 8 level-1 leaves."""
    lev, anc = uniform_leaves((2, 2, 2), 0)
    mask = np.all(anc == 0, axis=1)
    return refine_leaves(lev, anc, mask)


def tree_sphere(nt, tree_len, base, radii, centre=(0.5, 0.5, 0.5)):
    """Uniform at `base`, then refine every block meeting the ball of radius
    radii[k] at level base+k; 2:1 balanced."""
    lev, anc = uniform_leaves(nt, base)
    for k, r in enumerate(radii):
        lev, anc = refine_in_ball(nt, tree_len, lev, anc, centre, r, base + k)
        lev, anc = balance_fast(nt, lev, anc)
    return lev, anc


def random_tree(nt, base, nref, rng, max_level):
    """Seeded random balanced tree: `nref` rounds of refining a random leaf."""
    lev, anc = uniform_leaves(nt, base)
    for _ in range(nref):
        cand = np.nonzero(lev < max_level)[0]
        if len(cand) == 0:
            break
        mask = np.zeros(len(lev), bool)
        mask[rng.choice(cand)] = True
        lev, anc = refine_leaves(lev, anc, mask)
        lev, anc = balance(nt, lev, anc)
    return lev, anc


# ------------------------------------------------------------------ fields
def point_coords(nt, tree_len, nb, lev, anc):
    """x, y, z arrays of shape (n, nb, nb, nb) laid out [leaf, z, y, x]."""
    h = tree_len / (nb * (1 << lev.astype(np.int64)))
    i = np.arange(nb)
    out = []
    for d in range(3):
        g = (anc[:, d, None] * nb + i[None, :]) * h[:, None]
        shape = [len(lev), 1, 1, 1]
        shape[3 - d] = nb
        out.append(np.broadcast_to(g.reshape(shape), (len(lev), nb, nb, nb)))
    return out


def periodic_delta(x, c, ext):
    d = x - c
    return d - ext * np.round(d / ext)


def gaussian(xyz, centre, sigma, ext=(1.0, 1.0, 1.0)):
    """exp(-|x-c|^2/sigma^2) on the nearest periodic image."""
    r2 = sum(periodic_delta(xyz[d], centre[d], ext[d]) ** 2 for d in range(3))
    return np.exp(-r2 / sigma ** 2)


def gaussian_images(xyz, centre, sigma, ext=(1.0, 1.0, 1.0), nimg=2):
    """Sum over periodic images (exact periodic Gaussian train)."""
    tot = np.zeros_like(xyz[0])
    rng = range(-nimg, nimg + 1)
    for ix in rng:
        for iy in rng:
            for iz in rng:
                sh = (ix * ext[0], iy * ext[1], iz * ext[2])
                r2 = sum((xyz[d] - centre[d] - sh[d]) ** 2 for d in range(3))
                tot = tot + np.exp(-r2 / sigma ** 2)
    return tot


def fourier_front(xyz, seed, nmodes=16, kmax=8, width=0.02, radius=0.25,
                  centre=(0.5, 0.5, 0.5)):
    """Sum of seeded Fourier modes (|k|_inf in 1..kmax, amplitude ~|k|^-2) plus
    a tanh front on a sphere."""
    rng = np.random.default_rng(seed)
    f = np.zeros_like(xyz[0])
    for _ in range(nmodes):
        while True:
            k = rng.integers(-kmax, kmax + 1, size=3)
            if np.abs(k).max() >= 1:
                break
        th = rng.uniform(0, 2 * np.pi)
        a = 1.0 / float((k ** 2).sum())
        f = f + a * np.cos(2 * np.pi * (k[0] * xyz[0] + k[1] * xyz[1] + k[2] * xyz[2]) + th)
    r = np.sqrt(sum(periodic_delta(xyz[d], centre[d], 1.0) ** 2 for d in range(3)))
    return f + 0.5 * np.tanh((radius - r) / width)


def compact_gaussian(xyz, centre=(0.35, 0.35, 0.35), sigma=0.1, beta=0.2, ext=(1.0, 1.0, 1.0)):
    """exp(-(r^2/sigma^2) / (1 - r^2/beta^2)) for r < beta, else 0 (nearest
    periodic image); the initial field of the deformation test."""
    d = [periodic_delta(xyz[i], centre[i], ext[i]) for i in range(3)]
    r2 = d[0] ** 2 + d[1] ** 2 + d[2] ** 2
    out = np.zeros_like(r2)
    m = r2 < beta * beta
    out[m] = np.exp(-(r2[m] / sigma ** 2) / (1.0 - r2[m] / beta ** 2))
    return out


def deformation_velocity(xyz, comp, scale=1.0):
    """Component comp of the incompressible deformation field (published
    divergence-free form): (2 sin^2(pi x) sin(2 pi y) sin(2 pi z),
    -sin(2 pi x) sin^2(pi y) sin(2 pi z), -sin(2 pi x) sin(2 pi y) sin^2(pi z))."""
    x, y, z = xyz
    p = np.pi
    if comp == 0:
        return 2 * scale * np.sin(p * x) ** 2 * np.sin(2 * p * y) * np.sin(2 * p * z)
    if comp == 1:
        return -scale * np.sin(2 * p * x) * np.sin(p * y) ** 2 * np.sin(2 * p * z)
    return -scale * np.sin(2 * p * x) * np.sin(2 * p * y) * np.sin(p * z) ** 2


def tanh_sphere(xyz, radius=0.3, width=0.01, centre=(0.5, 0.5, 0.5)):
    r = np.sqrt(sum(periodic_delta(xyz[d], centre[d], 1.0) ** 2 for d in range(3)))
    return 0.5 * (1.0 - np.tanh((r - radius) / width))


def polynomial(xyz, coeffs, degree, x0=(0.5, 0.5, 0.5)):
    """Seeded-coefficient polynomial of total degree <= degree (not periodic:
    used away from the periodic seam)."""
    f = np.zeros_like(xyz[0])
    m = 0
    for p in range(degree + 1):
        for q in range(degree + 1 - p):
            for r in range(degree + 1 - p - q):
                f = f + coeffs[m % len(coeffs)] * ((xyz[0] - x0[0]) ** p) * \
                    ((xyz[1] - x0[1]) ** q) * ((xyz[2] - x0[2]) ** r)
                m += 1
    return f


def dyadic_random(shape, rng, bits=10):
    """Random values on a dyadic grid k/2^bits (exact in FP32 and FP64)."""
    return rng.integers(-(1 << bits), 1 << bits, size=shape).astype(np.float64) / (1 << bits)


# ------------------------------------------------------ large-tree helpers
def _level_map(nt, lev, anc, M):
    """Dense map at level M of the level of the leaf covering each cell."""
    D = np.zeros((nt[2] << M, nt[1] << M, nt[0] << M), np.int8)
    for L in np.unique(lev):
        s = 1 << (M - L)
        a = anc[lev == L]
        V = np.zeros((nt[2] << L, nt[1] << L, nt[0] << L), np.int8)
        V[a[:, 2], a[:, 1], a[:, 0]] = L + 1
        D = np.maximum(D, np.repeat(np.repeat(np.repeat(V, s, 0), s, 1), s, 2))
    return D - 1


def balance_fast(nt, lev, anc, max_iter=32):
    """2:1 balance (face, edge, corner; periodic) with a dense level map:
    refine every leaf that touches a leaf two or more levels finer."""
    from scipy.ndimage import maximum_filter
    for _ in range(max_iter):
        M = int(lev.max())
        D = _level_map(nt, lev, anc, M)
        Dn = maximum_filter(D, size=3, mode="wrap")
        need = np.zeros(len(lev), bool)
        for L in np.unique(lev):
            s = 1 << (M - L)
            Z, Y, X = Dn.shape
            B = Dn.reshape(Z // s, s, Y // s, s, X // s, s).max(axis=(1, 3, 5))
            idx = np.nonzero(lev == L)[0]
            a = anc[idx]
            need[idx] = B[a[:, 2], a[:, 1], a[:, 0]] > L + 1
        if not need.any():
            return lev, anc
        lev, anc = refine_leaves(lev, anc, need)
    raise RuntimeError("balance did not converge")


def tree_shell(nt, tree_len, base, top, radius, widths, centre=(0.5, 0.5, 0.5)):
    """Uniform at `base`; then at each level L < top refine the leaves whose
    box comes within widths[L-base] of the sphere |x - c| = radius
    (periodic); 2:1 balanced."""
    lev, anc = uniform_leaves(nt, base)
    ext = np.asarray(nt, float) * tree_len
    for k, L in enumerate(range(base, top)):
        c, size = block_centres(nt, tree_len, lev, anc)
        d = np.abs(c - np.asarray(centre))
        d = np.minimum(d, ext - d)
        half = 0.5 * size[:, None]
        near = np.sqrt((np.maximum(d - half, 0.0) ** 2).sum(1))
        far = np.sqrt(((d + half) ** 2).sum(1))
        hit = (near <= radius + widths[k]) & (far >= radius - widths[k]) & (lev == L)
        lev, anc = refine_leaves(lev, anc, hit)
        lev, anc = balance_fast(nt, lev, anc)
    return lev, anc


# --------------------------------------------------- independent-tree batch
def batch_leaves(per_tree, nt):
    """Leaves of a batch of independent one-tree grids laid out as the trees
    of an nt[0] x nt[1] x nt[2] forest: per_tree[k] = (lev, anc) of grid k
    (anchors within its own tree), tree k at (k % nt0, (k // nt0) % nt1,
    k // (nt0 nt1)).  Returns (lev, anc, tree index of every leaf)."""
    ls, as_, ts = [], [], []
    for k, (lev, anc) in enumerate(per_tree):
        t = np.array([k % nt[0], (k // nt[0]) % nt[1], k // (nt[0] * nt[1])], np.int64)
        ls.append(np.asarray(lev, np.int32))
        as_.append((np.asarray(anc, np.int64) + t[None, :] * (1 << np.asarray(lev, np.int64))[:, None]).astype(np.int32))
        ts.append(np.full(len(lev), k, np.int32))
    return np.concatenate(ls), np.concatenate(as_), np.concatenate(ts)
