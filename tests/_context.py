"""Oracle reference values for a sample of particles of a large set, with the
full neighbour context, and the per-particle edge allowance of the count
rule. Used by the full-size parity tests.

The force on a sampled particle i needs h, rho and Omega of every j with
r_ij < max(h_i, h_j). Those come from the oracle's own density solve, on a
region C that provably contains every such j: each particle's root h is
bounded from above by geometry alone. If K particles (itself included) lie
within h/2 of particle j, each adds w(q) >= w(1/2) = 1/4 to the weighted
neighbour number, so N_j(h) >= (32/3)(K/4) = (8/3) K; with K = 18 that is
48, and N is non-decreasing in h, so the root satisfies h_j <= 2 d18(j),
d18 = the distance to the 18th-nearest particle counting j itself (this
holds for a target of 48; the helper scales K with n_ngb). C = every j
within max(b_i, b_j) (1 + 1e-5) of some sampled i, b = 2 d_K. Outside C, h
is taken as 1e-30 with rho = Omega = 1: such j satisfy r_ij >= h_j
(1 + 1e-5) and r_ij >= h_i (1 + 1e-5) for every sampled i, so they enter the
oracle's force sums only through the target's own kernel term, exactly as
with their true values, and lie off every kernel edge of the count rule.
Nothing here comes from the CUDA path except which particles are sampled.
"""
import math

import numpy as np
from scipy.spatial import cKDTree

import oracle

EDGE = 1e-6
CHUNK = 1 << 21


def _tree(x, box):
    return cKDTree(x, boxsize=np.asarray(box, dtype=np.float64))


def h_upper_bound(tree, x, n_ngb):
    """2 d_K per particle, K = ceil(3 n_ngb / 8) (the 18th-nearest for 48)."""
    K = int(math.ceil(3.0 * n_ngb / 8.0))
    out = np.empty(x.shape[0])
    for a in range(0, x.shape[0], CHUNK):
        d, _ = tree.query(x[a:a + CHUNK], k=K, workers=-1)
        out[a:a + CHUNK] = 2.0 * d[:, -1]
    return out


def context_region(tree, x, box, S, b):
    """Indices of every particle within max(b_i, b_j) (1 + 1e-5) of some i in S."""
    near = set()
    for i, pts in zip(S, tree.query_ball_point(x[S], b[S] * (1 + 1e-5), workers=-1)):
        near.update(pts)
    ts = _tree(x[S], box)
    far = []
    for a in range(0, x.shape[0], CHUNK):
        d, _ = ts.query(x[a:a + CHUNK], k=1, workers=-1)
        far.append(a + np.nonzero(d < b[a:a + CHUNK] * (1 + 1e-5))[0])
    C = np.union1d(np.fromiter(near, dtype=np.int64), np.concatenate(far))
    return np.union1d(C, S)


def sampled_reference(p, S):
    """Oracle h, rho, Omega, density count, a, du/dt and force count of the
    particles S of a single-box set p (the sampled particles' arrays are
    indexed like S), plus the context (C and its oracle h) for edge counts."""
    x = np.ascontiguousarray(p.x, dtype=np.float64)
    box = p.box[0]
    m = p.m.astype(np.float64)
    tree = _tree(x, box)
    b = h_upper_bound(tree, x, p.n_ngb)
    C = context_region(tree, x, box, S, b)
    d = oracle.density(x, m, box, p.h, p.n_ngb, subset=C)
    h = np.full(p.n, 1e-30)
    rho = np.ones(p.n)
    om = np.ones(p.n)
    h[C], rho[C], om[C] = d["h"][C], d["rho"][C], d["omega"][C]
    assert np.all(h[C] <= b[C] * (1 + 1e-12))  # the bound the region relies on holds
    f = oracle.force(x, p.v.astype(np.float64), m, p.u.astype(np.float64), h, rho, om, box,
                     p.gamma, subset=S)
    return {"h": h[S], "rho": rho[S], "omega": om[S], "nngb": d["count"][S],
            "a": f["a"][S], "dudt": f["dudt"][S], "nforce": f["count"][S],
            "C": C, "h_all": h, "tree": tree, "x": x}


def edge_density(tree, x, h, S, eps=EDGE):
    """Per i in S: #{j : |r_ij - h_i| <= eps h_i} (pairs whose density count
    may legitimately differ)."""
    up = tree.query_ball_point(x[S], h[S] * (1 + eps), return_length=True, workers=-1)
    dn = tree.query_ball_point(x[S], h[S] * (1 - eps), return_length=True, workers=-1)
    return np.asarray(up) - np.asarray(dn)


def edge_force(tree, x, h, S, C, box, eps=EDGE):
    """Per i in S, an upper bound of #{j : |r_ij - max(h_i, h_j)| <= eps
    max(h_i, h_j)}: the pairs on the edge of i's own kernel plus those on the
    edge of j's kernel (j in C, whose h are the oracle's)."""
    amb = edge_density(tree, x, h, S, eps).astype(np.int64)
    ts = _tree(x[S], box)
    pos = {int(i): k for k, i in enumerate(S)}
    up = ts.query_ball_point(x[C], h[C] * (1 + eps), return_length=True, workers=-1)
    dn = ts.query_ball_point(x[C], h[C] * (1 - eps), return_length=True, workers=-1)
    hit = np.nonzero(np.asarray(up) > np.asarray(dn))[0]
    for k in hit:
        j = C[k]
        inner = set(ts.query_ball_point(x[j], h[j] * (1 - eps)))
        for s in ts.query_ball_point(x[j], h[j] * (1 + eps)):
            if s not in inner and int(S[s]) != int(j):
                amb[s] += 1
    return amb
