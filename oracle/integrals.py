"""Panel integrals of the modified RWG functions.

Eq. (RWG): on a triangle T with area A_T the modified RWG function of the edge
opposite vertex v_k is f(r) = s (r - v_k) / (2 A_T), s = +1 on T+ and -1 on T-,
with no edge-length factor, so the coefficient is the branch current.

Eq. (Zb), read as in Sec. II-D (R_b is the sparse surface-impedance term, L_b
the full one; the Gram term is the same-point dot product):
  R_b = Z_s G,   G_ij = int_S f_i(r) . f_j(r) dS
  L_b = (j w mu0 / 4 pi) Lt,   Lt_ij = int int f_i(r) . f_j(r') / |r - r'| dS' dS

Per triangle pair (T, T') the 3x3 block
  Blk[k, l] = int_T int_T' (r - v_k)/(2 A_T) . (r' - v'_l)/(2 A_T') / |r - r'| dS' dS
is evaluated with the inner integral over T' in closed form (the standard
potential integrals of 1 and of (rho' - rho) over a plane triangle: a sum over
the triangle's edges of logarithms and, off the plane, arctangents) and an
outer quadrature rule over T.  The exact block is symmetric under exchange of
the two triangles; a block is defined here with the lower-index triangle as
the outer one, the mirrored block is its transpose, and a self block is
replaced by its symmetric part.

Parity: the closed-form inner integrals are pinned against polar-coordinate
brute force; the Gram closed form against an exact quadrature rule; the blocks
against the far-field limit (int f_i).(int f_j)/R and against outer-rule
convergence (tests/test_oracle_integrals.py).
"""
from __future__ import annotations

import numpy as np

from .quadrature import radon7, collapsed_gauss, rule_points

MU0 = 4e-7 * np.pi


def tri_geometry(xyz, tri):
    p0, p1, p2 = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    n = np.cross(p1 - p0, p2 - p0)
    a2 = np.linalg.norm(n, axis=1)
    return dict(p=np.stack([p0, p1, p2], axis=1), area=0.5 * a2, normal=n / a2[:, None],
                centroid=(p0 + p1 + p2) / 3.0,
                diam=np.max(np.stack([np.linalg.norm(p1 - p0, axis=1),
                                      np.linalg.norm(p2 - p1, axis=1),
                                      np.linalg.norm(p0 - p2, axis=1)]), axis=0))


def gram_local(p, area):
    """Per-triangle 3x3 Gram block g[k,l] = int_T (r - v_k).(r - v_l) dS / (4 A^2).

    Closed form: int_T r_a r_b dS = A/12 (sum_i p_i,a p_i,b + (sum_i p_i,a)(sum_i p_i,b)),
    so int_T (r-a).(r-b) dS = A [ (sum|p_i|^2 + |sum p_i|^2)/12 - (a+b).c + a.b ]."""
    s = p.sum(axis=1)
    c = s / 3.0
    quad = (np.einsum("tij,tij->t", p, p) + np.einsum("ti,ti->t", s, s)) / 12.0
    pc = np.einsum("tki,ti->tk", p, c)                       # v_k . c
    pp = np.einsum("tki,tli->tkl", p, p)                     # v_k . v_l
    I = quad[:, None, None] - pc[:, :, None] - pc[:, None, :] + pp
    return I / (4.0 * area[:, None, None])


def gram_matrix(mesh, loops, sigma_weight=None):
    """Sparse branch Gram matrix G [nb, nb] (optionally each triangle's block
    scaled by sigma_weight[cond]), assembled from the per-triangle blocks."""
    import scipy.sparse as sp
    g = tri_geometry(mesh.xyz, mesh.tri)
    gl = gram_local(g["p"], g["area"])
    tb, ts = tri_branches(mesh.nt, loops)
    rows, cols, vals = [], [], []
    for t in range(mesh.nt):
        wt = 1.0 if sigma_weight is None else sigma_weight[mesh.cond[t]]
        for k in range(3):
            if tb[t, k] < 0:
                continue
            for l in range(3):
                if tb[t, l] < 0:
                    continue
                rows.append(tb[t, k])
                cols.append(tb[t, l])
                vals.append(wt * ts[t, k] * ts[t, l] * gl[t, k, l])
    nb = loops.nb
    return sp.csr_matrix((vals, (rows, cols)), shape=(nb, nb))


def tri_branches(nt, loops):
    """tb[t,k]: branch id of the edge opposite local vertex k of triangle t (-1 if
    none); ts[t,k]: +1 if t is the branch's T+, -1 if T-."""
    tb = np.full((nt, 3), -1, dtype=np.int64)
    ts = np.zeros((nt, 3))
    for b in range(loops.nb):
        tp, tm = loops.br_tri[b]
        kp, km = loops.br_local[b]
        tb[tp, kp] = b
        ts[tp, kp] = 1.0
        tb[tm, km] = b
        ts[tm, km] = -1.0
    return tb, ts


def potential_integrals(r, a0, a1, a2):
    """K0 = int_T 1/|r-r'| dS',  K1 = int_T (rho' - rho)/|r-r'| dS' over the plane
    triangle (a0, a1, a2), rho the projection of r onto its plane.

    Edge sum form: for edge i from p- to p+ with unit tangent l, outward in-plane
    normal u = l x n, distances l+- = (p+- - rho).l, P0 = (p- - rho).u, h = n.(r - a0),
    R0^2 = P0^2 + h^2, R+- = |r - p+-|, f = ln((R+ + l+)/(R- + l-)):
       K1 = 1/2 sum_i u_i (R0^2 f + l+ R+ - l- R-)    (divergence theorem on the plane)
       K0 = sum_i P0 f - |h| sum_i [atan(P0 l+/(R0^2+|h|R+)) - atan(P0 l-/(R0^2+|h|R-))]
    Broadcasts over leading dimensions."""
    n = np.cross(a1 - a0, a2 - a0)
    n = n / np.linalg.norm(n, axis=-1, keepdims=True)
    h = np.einsum("...i,...i->...", r - a0, n)
    rho = r - h[..., None] * n
    ah = np.abs(h)
    K0 = np.zeros(h.shape)
    K1 = np.zeros(rho.shape)
    for pm, pp in ((a0, a1), (a1, a2), (a2, a0)):
        L = pp - pm
        lt = L / np.linalg.norm(L, axis=-1, keepdims=True)
        u = np.cross(lt, n)
        lp = np.einsum("...i,...i->...", pp - rho, lt)
        lm = np.einsum("...i,...i->...", pm - rho, lt)
        P0 = np.einsum("...i,...i->...", pm - rho, u)
        R0s = P0 * P0 + h * h
        Rp = np.linalg.norm(r - pp, axis=-1)
        Rm = np.linalg.norm(r - pm, axis=-1)
        with np.errstate(divide="ignore", invalid="ignore"):
            num = np.where(lp >= 0, Rp + lp, R0s / (Rp - lp))
            den = np.where(lm >= 0, Rm + lm, R0s / (Rm - lm))
            f = np.log(num / den)
        f = np.where(R0s > 0, f, 0.0)
        beta = (np.arctan2(P0 * lp, R0s + ah * Rp) - np.arctan2(P0 * lm, R0s + ah * Rm))
        K0 += P0 * f - ah * beta
        K1 += 0.5 * u * (R0s * f + lp * Rp - lm * Rm)[..., None]
    return K0, K1


def pair_blocks(pT, aT, pS, aS, rule):
    """3x3 blocks Blk[k,l] for triangle pairs (T outer, S inner), inner integral in
    closed form, outer `rule` on T.  pT, pS: [m, 3, 3] vertices; aT, aS: [m]."""
    bary, w = rule
    rq = rule_points(rule, pT[:, 0], pT[:, 1], pT[:, 2])           # [m, Q, 3]
    s0, s1, s2 = (pS[:, None, i, :] for i in range(3))
    K0, K1 = potential_integrals(rq, s0, s1, s2)                    # [m,Q], [m,Q,3]
    n = np.cross(pS[:, 1] - pS[:, 0], pS[:, 2] - pS[:, 0])
    n = n / np.linalg.norm(n, axis=1, keepdims=True)
    h = np.einsum("mqi,mi->mq", rq - pS[:, None, 0], n)
    rho = rq - h[..., None] * n[:, None, :]
    # inner vector for each l: K1 + (rho - v'_l) K0
    inner = K1[:, :, None, :] + (rho[:, :, None, :] - pS[:, None, :, :]) * K0[:, :, None, None]
    outer = rq[:, :, None, :] - pT[:, None, :, :]                   # (r - v_k)
    blk = np.einsum("q,mqki,mqli->mkl", w, outer, inner)
    return blk * (aT / (4.0 * aT * aS))[:, None, None]
    # (outer weight A_T, normalisation 1/(2A_T) 1/(2A_S))


def pair_blocks_quadrature(pT, aT, pS, aS, rule_o, rule_i):
    """Same blocks with both integrals by product quadrature (regular pairs only)."""
    ro = rule_points(rule_o, pT[:, 0], pT[:, 1], pT[:, 2])
    ri = rule_points(rule_i, pS[:, 0], pS[:, 1], pS[:, 2])
    d = np.linalg.norm(ro[:, :, None, :] - ri[:, None, :, :], axis=-1)
    fo = ro[:, :, None, :] - pT[:, None, :, :]
    fi = ri[:, :, None, :] - pS[:, None, :, :]
    blk = np.einsum("p,q,mpki,mqli,mpq->mkl", rule_o[1], rule_i[1], fo, fi, 1.0 / d)
    return blk * (aT * aS / (4.0 * aT * aS))[:, None, None]


def touching(tri, i, j):
    """Boolean per pair: triangles i and j share at least one vertex (or are equal)."""
    a = tri[i]
    b = tri[j]
    return (a[:, :, None] == b[:, None, :]).any(axis=(1, 2))


def symmetric_blocks(mesh, pairs_i, pairs_j, rule_touch, rule_far, far_ratio=None, rule_mid=None,
                     chunk=20000, native=True):
    """Blocks for ordered pairs (i, j), defined symmetrically: each unordered pair is
    evaluated with the lower index outer; (j, i) is the transpose; i == j blocks
    are symmetrised.  Touching pairs use `rule_touch` for the outer integral,
    others `rule_far` (or `rule_mid` when the centroid distance is below
    far_ratio times the larger diameter).  native=True evaluates the blocks with
    the plain C loop (oracle/c), otherwise with numpy."""
    g = tri_geometry(mesh.xyz, mesh.tri)
    i = np.asarray(pairs_i, dtype=np.int64)
    j = np.asarray(pairs_j, dtype=np.int64)
    lo, hi = np.minimum(i, j), np.maximum(i, j)
    out = np.empty((i.shape[0], 3, 3))
    tch = touching(mesh.tri, lo, hi)
    if far_ratio is not None and rule_mid is not None:
        dist = np.linalg.norm(g["centroid"][lo] - g["centroid"][hi], axis=1)
        mid = (~tch) & (dist < far_ratio * np.maximum(g["diam"][lo], g["diam"][hi]))
    else:
        mid = np.zeros_like(tch)
    groups = [(tch, rule_touch), (mid, rule_mid), (~tch & ~mid, rule_far)]
    for mask, rule in groups:
        idx = np.nonzero(mask)[0]
        if rule is None:
            continue
        step = chunk if native else max(1, 2000000 // (len(rule[1]) * 40))
        fn = pair_blocks
        if native:
            from .native import pair_blocks as fn
        for c0 in range(0, idx.shape[0], step):
            s = idx[c0:c0 + step]
            blk = fn(g["p"][lo[s]], g["area"][lo[s]], g["p"][hi[s]], g["area"][hi[s]], rule)
            swap = i[s] > j[s]
            blk[swap] = np.transpose(blk[swap], (0, 2, 1))
            same = i[s] == j[s]
            blk[same] = 0.5 * (blk[same] + np.transpose(blk[same], (0, 2, 1)))
            out[s] = blk
    return out


# Outer rules used by the dense oracle: accurate enough that the dense L-tilde is
# the reference definition (pinned by outer-rule convergence in the tests).
DENSE_RULE_TOUCH = None
DENSE_RULE_MID = None
DENSE_RULE_FAR = None


def dense_rules():
    global DENSE_RULE_TOUCH, DENSE_RULE_MID, DENSE_RULE_FAR
    if DENSE_RULE_TOUCH is None:
        DENSE_RULE_TOUCH = collapsed_gauss(24)
        DENSE_RULE_MID = collapsed_gauss(8)
        DENSE_RULE_FAR = radon7()
    return DENSE_RULE_TOUCH, DENSE_RULE_MID, DENSE_RULE_FAR
