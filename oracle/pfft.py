"""Plain pre-corrected FFT product of the inductive term (Sec. IV-B), O2.

The four steps of Sec. IV-B in the paper's order and notation, each written
plainly (dense or scipy-sparse matrices, numpy's FFT as the library step):

  1. Projection, Eq. (Projection):   Q_g = B alpha        (alpha = A^T I_l)
  2. Convolution, Eq. (FFTCal):      phi_g = H Q_g        (3-level Toeplitz, via FFT)
  3. Interpolation, Eq. (interpolation): Phi = I phi_g,   I = B^T (Galerkin)
  4. Near field, Eq. (Lb):           L_b ~ L_d + I H B

Readings where the paper is silent or ambiguous:
  * grid: N_x x N_y x N_z nodes spanning the mesh bounding box, spacing
    h_d = extent_d / (N_d - 1); the Toeplitz product is an aperiodic
    convolution evaluated on the zero-padded 2N_d periodic grid;
  * H(d) = 1 / |d o h| for a node offset d != 0 and H(0) = h0 (0 by default;
    every pair whose stencils share a node is in the near list, so the
    result does not depend on h0);
  * the current of each triangle is sampled at the points of a triangle rule
    (Radon 7-point by default); each point carries its own stencil of O_s
    nodes per axis (the O_s nodes nearest the point, clamped inside the grid)
    with tensor-product Lagrange weights;
  * near pairs: centroid distance below r_near, or stencil boxes overlapping;
    L_d = L_direct - (I H B) restricted to near pairs, so near pairs get the
    direct integral and all others the grid product;
  * L_direct: closed-form inner integral, outer rule collapsed Gauss (n_touch^2
    points) for pairs sharing a vertex and Radon 7-point otherwise.
Parity: pinned by the FFT convolution against a direct sum, the all-near case
against the dense product, H(0) independence, polynomial exactness of the
stencils and convergence to the dense MoM (tests/test_oracle_pfft.py).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from .integrals import (MU0, tri_geometry, tri_branches, symmetric_blocks, gram_matrix)
from .quadrature import radon7, collapsed_gauss, rule_points
from .mom import branch_zs


@dataclass
class PfftParams:
    grid: tuple = (16, 8, 8)
    order: int = 3            # O_s
    near_factor: float = 4.0  # r_near = near_factor * max(h)
    near_min_diam: float = 2.0  # r_near >= near_min_diam * max triangle diameter
    n_touch: int = 16         # collapsed-Gauss order for touching near pairs
    h0: float = 0.0           # H at zero offset
    box: tuple = None         # (lo, hi) grid box; default the mesh's bounding box


def grid_of(mesh, N, box=None):
    lo, hi = mesh.bbox() if box is None else (np.asarray(box[0], float), np.asarray(box[1], float))
    N = np.asarray(N, dtype=np.int64)
    h = (hi - lo) / (N - 1)
    return lo, h, N


def stencil_1d(t, order, n):
    """Start node and Lagrange weights of the `order` nodes nearest coordinate t
    (in grid units), clamped inside [0, n)."""
    if order % 2:
        start = np.floor(t + 0.5).astype(np.int64) - (order - 1) // 2
    else:
        start = np.floor(t).astype(np.int64) - (order // 2 - 1)
    start = np.clip(start, 0, n - order)
    w = np.ones(t.shape + (order,))
    for i in range(order):
        for j in range(order):
            if j != i:
                w[..., i] *= (t - (start + j)) / (i - j)
    return start, w


class Pfft:
    """pFFT operator of one mesh and loop basis (plain FP64)."""

    def __init__(self, mesh, loops, params: PfftParams, rule=None, targets=None, lean=False):
        """targets: optional triangle ids; the near list then holds only the pairs
        (t, j) with t in targets, so that rows of the product are exact for the
        branches whose triangles are all targets (sampled rows of a large mesh).
        lean: apply the projection B and the interpolation B^T triangle by
        triangle (project / interpolate) instead of storing B as a sparse matrix
        (meshes of hundreds of thousands of triangles)."""
        self.mesh, self.loops, self.p = mesh, loops, params
        self.lean = lean
        self.targets = None if targets is None else np.unique(np.asarray(targets, dtype=np.int64))
        self.rule = radon7() if rule is None else rule
        self.lo, self.h, self.N = grid_of(mesh, params.grid, params.box)
        g = tri_geometry(mesh.xyz, mesh.tri)
        self.geo = g
        nt = mesh.nt
        rq = rule_points(self.rule, g["p"][:, 0], g["p"][:, 1], g["p"][:, 2])   # [nt,Q,3]
        self.rq = rq
        Q = rq.shape[1]
        O = params.order
        t = (rq - self.lo) / self.h
        starts, wts = [], []
        for d in range(3):
            s, w = stencil_1d(t[..., d], O, self.N[d])
            starts.append(s)
            wts.append(w)
        self.start = np.stack(starts, axis=-1)          # [nt,Q,3]
        self.lw = wts                                   # 3 x [nt,Q,O]
        self.tb, self.ts = tri_branches(nt, loops)
        # point current weights: J_q = sum_k c_k (w_q/2)(r_q - v_k)
        self.mom = 0.5 * self.rule[1][None, :, None, None] * (rq[:, :, None, :] - g["p"][:, None, :, :])
        if not lean:
            self._build_B()
        self._build_H()
        self._build_near()

    # -- step 1: projection matrix B [3 N_g, nb]
    def _build_B(self):
        nt, Q = self.rq.shape[:2]
        O = self.p.order
        Nx, Ny, Nz = self.N
        off = np.arange(O)
        # node index and Lagrange weight of each (triangle, point, stencil node)
        ix = self.start[..., 0][..., None, None, None] + off[:, None, None]
        iy = self.start[..., 1][..., None, None, None] + off[None, :, None]
        iz = self.start[..., 2][..., None, None, None] + off[None, None, :]
        node = ((ix * Ny + iy) * Nz + iz).reshape(nt, Q, -1)              # [nt,Q,O^3]
        lw = (self.lw[0][..., :, None, None] * self.lw[1][..., None, :, None]
              * self.lw[2][..., None, None, :]).reshape(nt, Q, -1)
        rows, cols, vals = [], [], []
        for kk in range(3):
            ok = self.tb[:, kk] >= 0
            for c in range(3):
                # B[(c, n), b] += s_k (w_q/2)(r_q - v_k)_c L_n(r_q)
                m = (self.ts[:, kk, None] * self.mom[:, :, kk, c])[:, :, None] * lw
                rows.append((c * self.ng + node)[ok].ravel())
                cols.append(np.broadcast_to(self.tb[:, kk, None, None], node.shape)[ok].ravel())
                vals.append(m[ok].ravel())
        self.B = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(3 * self.ng, self.loops.nb))

    @property
    def ng(self):
        return int(np.prod(self.N))

    # -- step 2: kernel on the padded grid
    def kernel_value(self, d):
        """H at integer node offsets d [...,3]."""
        r = np.linalg.norm(d * self.h, axis=-1)
        with np.errstate(divide="ignore"):
            v = 1.0 / r
        return np.where(np.all(d == 0, axis=-1), self.p.h0, v)

    def _build_H(self):
        M = 2 * self.N
        ax = [np.where(np.arange(m) < m // 2, np.arange(m), np.arange(m) - m) for m in M]
        ax[0][M[0] // 2] = ax[1][M[1] // 2] = ax[2][M[2] // 2] = 0   # unused wrap offset
        dx, dy, dz = np.meshgrid(*ax, indexing="ij")
        H = self.kernel_value(np.stack([dx, dy, dz], axis=-1))
        for a, m in enumerate(M):
            sl = [slice(None)] * 3
            sl[a] = m // 2
            H[tuple(sl)] = 0.0
        self.Hpad = H
        self.Hhat = np.fft.fftn(H)

    def convolve(self, Qg):
        """phi_g = H Q_g for one component, Q_g [N_x,N_y,N_z] complex (FFT)."""
        M = 2 * self.N
        pad = np.zeros(tuple(M), dtype=complex)
        pad[:self.N[0], :self.N[1], :self.N[2]] = Qg
        out = np.fft.ifftn(np.fft.fftn(pad) * self.Hhat)
        return out[:self.N[0], :self.N[1], :self.N[2]]

    def convolve_direct(self, Qg):
        """Same product by the direct O(N_g^2) sum (tiny grids only)."""
        Nx, Ny, Nz = self.N
        idx = np.stack(np.meshgrid(np.arange(Nx), np.arange(Ny), np.arange(Nz), indexing="ij"),
                       axis=-1).reshape(-1, 3)
        Hm = self.kernel_value(idx[:, None, :] - idx[None, :, :])
        return (Hm @ Qg.reshape(-1)).reshape(Qg.shape)

    def far(self, alpha):
        """Bt H B alpha over all pairs (branch space, no mu0/4pi)."""
        if self.lean:
            Qg = self.project(alpha)
            return self.interpolate(np.stack([self.convolve(Qg[c]) for c in range(3)]))
        Qg = (self.B @ alpha).reshape(3, *self.N)
        phi = np.stack([self.convolve(Qg[c]) for c in range(3)]).reshape(-1)
        return self.B.T @ phi

    # -- steps 1 and 3 without storing B (the same sums, a chunk of triangles at a time)
    def _stencil_chunk(self, t0, t1):
        O = self.p.order
        Nx, Ny, Nz = self.N
        off = np.arange(O)
        st = self.start[t0:t1]
        ix = st[..., 0][..., None, None, None] + off[:, None, None]
        iy = st[..., 1][..., None, None, None] + off[None, :, None]
        iz = st[..., 2][..., None, None, None] + off[None, None, :]
        node = ((ix * Ny + iy) * Nz + iz).reshape(t1 - t0, st.shape[1], -1)
        lw = (self.lw[0][t0:t1][..., :, None, None] * self.lw[1][t0:t1][..., None, :, None]
              * self.lw[2][t0:t1][..., None, None, :]).reshape(t1 - t0, st.shape[1], -1)
        return node, lw

    def project(self, alpha, chunk=20000):
        """Q_g = B alpha [3, N_x, N_y, N_z]: each sample point's current
        J_q = sum_k s_k alpha_k (w_q/2)(r_q - v_k) spread over its stencil with the
        Lagrange weights (Eq. Projection)."""
        alpha = np.asarray(alpha, dtype=complex)
        ng = self.ng
        out = np.zeros((3, ng), dtype=complex)
        a_tri = np.where(self.tb >= 0, self.ts * alpha[np.maximum(self.tb, 0)], 0.0)   # [nt, 3]
        for t0 in range(0, self.mesh.nt, chunk):
            t1 = min(self.mesh.nt, t0 + chunk)
            node, lw = self._stencil_chunk(t0, t1)
            J = np.einsum("tk,tqkc->tqc", a_tri[t0:t1], self.mom[t0:t1])          # [m, Q, 3]
            for c in range(3):
                v = (J[:, :, c, None] * lw).ravel()
                out[c] += (np.bincount(node.ravel(), weights=v.real, minlength=ng)
                           + 1j * np.bincount(node.ravel(), weights=v.imag, minlength=ng))
        return out.reshape(3, *self.N)

    def interpolate(self, phi, chunk=20000):
        """B^T phi [nb] for grid potentials phi [3, N_x, N_y, N_z] (I = B^T, Eq.
        interpolation): each sample point's interpolated potential, tested with
        s_k (w_q/2)(r_q - v_k) and summed into the triangle's branches."""
        ph = np.asarray(phi).reshape(3, -1)
        out = np.zeros(self.loops.nb, dtype=complex)
        for t0 in range(0, self.mesh.nt, chunk):
            t1 = min(self.mesh.nt, t0 + chunk)
            node, lw = self._stencil_chunk(t0, t1)
            P = np.stack([np.einsum("tqn,tqn->tq", lw, ph[c][node]) for c in range(3)], axis=-1)   # [m, Q, 3]
            val = np.einsum("tqkc,tqc->tk", self.mom[t0:t1], P) * self.ts[t0:t1]
            ok = self.tb[t0:t1] >= 0
            np.add.at(out, self.tb[t0:t1][ok], val[ok])
        return out

    # -- step 4: near list and pre-correction
    def _build_near(self):
        g = self.geo
        O = self.p.order
        r_near = max(self.p.near_factor * float(np.max(self.h)),
                     self.p.near_min_diam * float(np.max(g["diam"])))
        self.r_near = r_near
        c = g["centroid"]
        bmin = self.start.min(axis=1)
        bmax = self.start.max(axis=1) + (O - 1)
        nt = self.mesh.nt
        pi, pj = [], []
        for t in (range(nt) if self.targets is None else self.targets):
            d = c - c[t]
            d2 = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]
            box = np.all((bmin <= bmax[t]) & (bmax >= bmin[t]), axis=1)
            nb = np.nonzero((d2 < r_near * r_near) | box)[0]
            pi.append(np.full(nb.shape, t))
            pj.append(nb)
        self.near_i = np.concatenate(pi)
        self.near_j = np.concatenate(pj)
        rule_t = collapsed_gauss(self.p.n_touch)
        self.L_direct = symmetric_blocks(self.mesh, self.near_i, self.near_j, rule_t, radon7())
        self.L_grid = self.grid_blocks(self.near_i, self.near_j)
        self.L_d = self.L_direct - self.L_grid

    def grid_blocks(self, ti, tj, native=True):
        """(I H B) 3x3 blocks for triangle pairs, written out node by node:
        sum_q sum_q' (w_q/2)(w_q'/2) (r_q - v_k).(r_q' - v'_l)
                    sum_{n in S(q)} sum_{n' in S(q')} L_n(q) H(n - n') L_n'(q')."""
        if native:
            from .native import grid_blocks
            return grid_blocks(ti, tj, self.start, self.lw, self.mom, self.Hpad)
        O = self.p.order
        Q = self.rq.shape[1]
        off = np.stack(np.meshgrid(np.arange(O), np.arange(O), np.arange(O), indexing="ij"),
                       axis=-1).reshape(-1, 3)                       # [O^3, 3]
        out = np.zeros((len(ti), 3, 3), dtype=self.Hpad.dtype)   # complex for a complex kernel table
        for s0 in range(0, len(ti), 200):
            a = ti[s0:s0 + 200]
            b = tj[s0:s0 + 200]
            na = self.start[a][:, :, None, :] + off[None, None]       # [m,Q,O^3,3]
            nb_ = self.start[b][:, :, None, :] + off[None, None]
            la = (self.lw[0][a][:, :, :, None, None] * self.lw[1][a][:, :, None, :, None]
                  * self.lw[2][a][:, :, None, None, :]).reshape(len(a), Q, -1)
            lb = (self.lw[0][b][:, :, :, None, None] * self.lw[1][b][:, :, None, :, None]
                  * self.lw[2][b][:, :, None, None, :]).reshape(len(b), Q, -1)
            d = na[:, :, None, :, None, :] - nb_[:, None, :, None, :, :]   # [m,Q,Q,O3,O3,3]
            M = 2 * self.N
            Hv = self.Hpad[d[..., 0] % M[0], d[..., 1] % M[1], d[..., 2] % M[2]]   # H(n - n')
            G = np.einsum("mpu,mpquv,mqv->mpq", la, Hv, lb)
            fa = self.mom[a]                                              # [m,Q,3,3]
            fb = self.mom[b]
            out[s0:s0 + 200] = np.einsum("mpki,mqli,mpq->mkl", fa, fb, G)
        return out

    def near_matrix(self, blocks=None):
        """Sparse branch matrix of the near blocks (default L_d)."""
        blocks = self.L_d if blocks is None else blocks
        tb, ts = self.tb, self.ts
        rows, cols, vals = [], [], []
        for k in range(3):
            for l in range(3):
                bi = tb[self.near_i, k]
                bj = tb[self.near_j, l]
                ok = (bi >= 0) & (bj >= 0)
                rows.append(bi[ok])
                cols.append(bj[ok])
                vals.append(ts[self.near_i[ok], k] * ts[self.near_j[ok], l] * blocks[ok, k, l])
        nb = self.loops.nb
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(nb, nb))

    def Lt_apply(self, alpha, near=None):
        """pFFT approximation of Lt alpha (branch space)."""
        if near is None:
            if not hasattr(self, "_near"):
                self._near = self.near_matrix()
            near = self._near
        return self.far(alpha) + near @ alpha


class PfftSystem:
    """Loop-space product y = A (Z_s G + j w mu0/4pi (L_d + I H B)) A^T x."""

    def __init__(self, mesh, loops, params: PfftParams, t_eff=None, targets=None, lean=False):
        self.mesh, self.loops = mesh, loops
        self.t_eff = t_eff   # effective thickness per conductor: slab surface impedance (mom.py)
        self.op = Pfft(mesh, loops, params, targets=targets, lean=lean)
        self.G = gram_matrix(mesh, loops)
        nb = loops.nb
        self.A = loops.A[:, :nb].tocsr()

    def branch_product(self, alpha, omega):
        zs = branch_zs(self.mesh, self.loops, omega, self.t_eff)
        return zs * (self.G @ alpha) + (1j * omega * MU0 / (4.0 * np.pi)) * self.op.Lt_apply(alpha)

    def matvec(self, x, omega):
        return self.A @ self.branch_product(self.A.T @ x, omega)

    def diag_Zb(self, omega):
        """diag(Z_b): Gram and inductive self terms (the near blocks hold the
        direct self integrals)."""
        zs = branch_zs(self.mesh, self.loops, omega, self.t_eff)
        Ld = self.op.near_matrix(self.op.L_direct)
        return zs * self.G.diagonal() + (1j * omega * MU0 / (4.0 * np.pi)) * Ld.diagonal()
