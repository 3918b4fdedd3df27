"""Seeded synthetic conductor meshes.

These generators produce the inputs of the method only: vertex coordinates,
triangle connectivity (counter-clockwise seen from outside, so the right-hand
normal points out of the conductor), a conductor id per triangle, the
conductivity of each conductor and the port contact sets.  They hold none of
the method's arithmetic and are shared by the oracle, the tests and the bench.

A port is a pair (source triangles, sink triangles) on one conductor, the
electrode faces between which a unit voltage source is applied (Sec. III-C of
the paper: a voltage source between two circuit nodes; a contact face made of
many triangles is one node).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np


@dataclass
class Mesh:
    xyz: np.ndarray          # float64 [nv, 3], metres
    tri: np.ndarray          # int32   [nt, 3], CCW seen from outside
    cond: np.ndarray         # int32   [nt], conductor id
    sigma: np.ndarray        # float64 [ncond], S/m
    ports: list = field(default_factory=list)  # [(src int32[], sink int32[])]
    name: str = ""

    @property
    def nv(self):
        return int(self.xyz.shape[0])

    @property
    def nt(self):
        return int(self.tri.shape[0])

    @property
    def ncond(self):
        return int(self.sigma.shape[0])

    def bbox(self):
        return self.xyz.min(axis=0), self.xyz.max(axis=0)


def _orient(xyz, tris, outward):
    """Flip triangles whose right-hand normal points against `outward`."""
    tris = np.asarray(tris, dtype=np.int64)
    p0, p1, p2 = xyz[tris[:, 0]], xyz[tris[:, 1]], xyz[tris[:, 2]]
    n = np.cross(p1 - p0, p2 - p0)
    flip = np.einsum("ij,ij->i", n, outward) < 0
    tris[flip] = tris[flip][:, [0, 2, 1]]
    return tris


def box_mesh(L, W, T, nx, ny, nz, jitter=0.0, seed=1, sigma=5.8e7, origin=(0.0, 0.0, 0.0),
             with_port=True, name="box"):
    """Closed triangulated surface of the box [0,L]x[0,W]x[0,T] (+origin).

    Each face is a structured grid of quads (nx, ny, nz divisions along x, y,
    z), each quad split into two triangles with alternating diagonals.  Face
    vertices that do not lie on a box edge are moved in-plane by a seeded
    uniform jitter of +-`jitter` times the local spacing.  The port (if
    requested) drives current from the x=0 end face to the x=L end face.
    """
    rng = np.random.default_rng(seed)
    hx, hy, hz = L / nx, W / ny, T / nz
    vid = {}
    verts = []

    def vertex(i, j, k):
        key = (i, j, k)
        if key not in vid:
            vid[key] = len(verts)
            verts.append((i, j, k))
        return vid[key]

    faces = []   # (quad vertex ids, outward normal, face tag)
    # each face: fixed axis a at value v, two running axes (u, w)
    dims = (nx, ny, nz)
    for axis in range(3):
        for side in (0, 1):
            fixed = side * dims[axis]
            ua, wa = [a for a in range(3) if a != axis]
            nrm = np.zeros(3)
            nrm[axis] = 1.0 if side else -1.0
            tag = 2 * axis + side
            for u in range(dims[ua]):
                for w in range(dims[wa]):
                    def lat(du, dw):
                        c = [0, 0, 0]
                        c[axis] = fixed
                        c[ua] = u + du
                        c[wa] = w + dw
                        return vertex(*c)
                    q = (lat(0, 0), lat(1, 0), lat(1, 1), lat(0, 1))
                    faces.append((q, nrm, tag, (u + w) % 2))
    lattice = np.array(verts, dtype=np.float64)
    xyz = lattice * np.array([hx, hy, hz]) + np.asarray(origin, dtype=np.float64)
    if jitter > 0.0:
        for n, (i, j, k) in enumerate(verts):
            on = [i in (0, nx), j in (0, ny), k in (0, nz)]
            if sum(on) != 1:
                continue          # on a box edge or corner: keep
            axis = on.index(True)
            for a, h in zip(range(3), (hx, hy, hz)):
                if a != axis:
                    xyz[n, a] += rng.uniform(-jitter, jitter) * h
    tris, outward, tags = [], [], []
    for (a, b, c, d), nrm, tag, par in faces:
        if par == 0:
            tris += [(a, b, c), (a, c, d)]
        else:
            tris += [(a, b, d), (b, c, d)]
        outward += [nrm, nrm]
        tags += [tag, tag]
    tris = _orient(xyz, tris, np.array(outward))
    tags = np.array(tags)
    mesh = Mesh(xyz=xyz, tri=tris.astype(np.int32), cond=np.zeros(len(tris), np.int32),
                sigma=np.array([sigma], dtype=np.float64), name=name)
    if with_port:
        src = np.nonzero(tags == 0)[0].astype(np.int32)   # x = 0 face
        snk = np.nonzero(tags == 1)[0].astype(np.int32)   # x = L face
        mesh.ports = [(src, snk)]
    return mesh


def wire_array_mesh(n_wires, radius, length, pitch, n_sides=16, seg_len=None, n_seg=None,
                    jitter=0.0, seed=2, sigma=4.1e7, name="wires"):
    """Parallel round wires along x, polygonal cross-section with `n_sides` sides.

    Wire w has its axis on (y, z) = (w * pitch, 0).  The lateral surface is a
    ring-by-ring structured quad mesh split into triangles; each end cap is a
    fan around a centre vertex.  Interior ring positions get a seeded axial
    jitter of +-`jitter` times the segment length.  Port w drives wire w from
    its x=0 cap (source) to its x=length cap (sink).
    """
    rng = np.random.default_rng(seed)
    if n_seg is None:
        n_seg = max(1, int(round(length / seg_len)))
    xyz, tris, outward, cond, ports = [], [], [], [], []
    th = 2.0 * np.pi * np.arange(n_sides) / n_sides
    for w in range(n_wires):
        y0 = w * pitch
        base = len(xyz)
        xs = np.linspace(0.0, length, n_seg + 1)
        if jitter > 0.0 and n_seg > 1:
            xs[1:-1] += rng.uniform(-jitter, jitter, n_seg - 1) * (length / n_seg)
        for s in range(n_seg + 1):
            for k in range(n_sides):
                xyz.append((xs[s], y0 + radius * np.cos(th[k]), radius * np.sin(th[k])))
        c0 = len(xyz)
        xyz.append((0.0, y0, 0.0))
        c1 = len(xyz)
        xyz.append((length, y0, 0.0))

        def rv(s, k):
            return base + s * n_sides + (k % n_sides)
        t_start = len(tris)
        for s in range(n_seg):
            for k in range(n_sides):
                a, b, c, d = rv(s, k), rv(s + 1, k), rv(s + 1, k + 1), rv(s, k + 1)
                mid = 0.5 * (th[k] + th[(k + 1) % n_sides] + (2 * np.pi if k == n_sides - 1 else 0.0))
                nrm = np.array([0.0, np.cos(mid), np.sin(mid)])
                if (s + k) % 2 == 0:
                    tris += [(a, b, c), (a, c, d)]
                else:
                    tris += [(a, b, d), (b, c, d)]
                outward += [nrm, nrm]
        src = []
        for k in range(n_sides):
            src.append(len(tris))
            tris.append((c0, rv(0, k), rv(0, k + 1)))
            outward.append(np.array([-1.0, 0.0, 0.0]))
        snk = []
        for k in range(n_sides):
            snk.append(len(tris))
            tris.append((c1, rv(n_seg, k), rv(n_seg, k + 1)))
            outward.append(np.array([1.0, 0.0, 0.0]))
        cond += [w] * (len(tris) - t_start)
        ports.append((np.array(src, np.int32), np.array(snk, np.int32)))
    xyz = np.array(xyz, dtype=np.float64)
    tris = _orient(xyz, tris, np.array(outward))
    return Mesh(xyz=xyz, tri=tris.astype(np.int32), cond=np.array(cond, np.int32),
                sigma=np.full(n_wires, sigma, dtype=np.float64), ports=ports, name=name)


def merge(meshes, name="merged"):
    """Concatenate meshes into one multi-conductor mesh (ids and ports shifted)."""
    xyz, tri, cond, sigma, ports = [], [], [], [], []
    nv = nt = nc = 0
    for m in meshes:
        xyz.append(m.xyz)
        tri.append(m.tri + nv)
        cond.append(m.cond + nc)
        sigma.append(m.sigma)
        for s, k in m.ports:
            ports.append((s + nt, k + nt))
        nv += m.nv
        nt += m.nt
        nc += m.ncond
    return Mesh(xyz=np.concatenate(xyz), tri=np.concatenate(tri).astype(np.int32),
                cond=np.concatenate(cond).astype(np.int32), sigma=np.concatenate(sigma),
                ports=ports, name=name)


def plane_pair_mesh(L=10e-3, t=35e-6, gap=100e-6, n=250, m_gap=3, n_pairs=200, via_k=2, n_ports=4, pad_k=3,
                    site=10, jitter=0.15, seed=11, sigma=5.8e7, name="plane_pair"):
    """Two square planes (L x L, thickness t) a gap apart, joined by via pairs.

    Both planes sit on one structured lattice of n x n cells (spacing h = L/n);
    every quad is split into two triangles with alternating diagonals.  A via
    is a square prism of via_k x via_k cells spanning the gap (m_gap divisions
    in height); its cells are removed from the two inner faces and its walls
    share their end edges with the hole boundaries, so the surface is
    conformal (one closed conductor with a handle per via).  Via pairs are
    placed at seeded distinct sites of a coarse lattice (site x site cells),
    the two vias of a pair 2 via_k cells apart along x.  Each port drives a
    pad of pad_k x pad_k cells on the top plane's upper face (source) against
    the pad below it on the bottom plane's lower face (sink), at further
    seeded sites.  Vertices inside the two outer faces get an in-plane jitter
    of +-jitter h.
    """
    rng = np.random.default_rng(seed)
    h = L / n
    zlev = np.concatenate([[0.0], t + gap * np.arange(m_gap + 1) / m_gap, [2 * t + gap]])
    top_in, top_out = 1 + m_gap, 2 + m_gap          # z levels of the top plane's faces
    nsite = n // site
    cand = np.array([(I, J) for I in range(1, nsite - 1) for J in range(1, nsite - 1)])
    if site < 3 * via_k + 2 or site < pad_k + 4 or len(cand) < n_pairs + n_ports:
        raise ValueError("plane_pair_mesh: too few via/pad sites for the lattice")
    pick = rng.permutation(len(cand))[:n_pairs + n_ports]
    via_sites, pad_sites = cand[pick[:n_pairs]], cand[pick[n_pairs:]]
    hole = np.zeros((n, n), bool)
    vias = []
    for I, J in via_sites:
        i0, j0 = I * site + 1, J * site + 2
        for dx in (0, 2 * via_k):
            vias.append((i0 + dx, j0))
            hole[i0 + dx:i0 + dx + via_k, j0:j0 + via_k] = True

    def code(lz, i, j):
        return (np.asarray(lz) * (n + 1) + np.asarray(i)) * (n + 1) + np.asarray(j)

    quads, normals, tags = [], [], []   # quads: [k, 4] lattice codes; tag: face id for ports

    def add(q, nrm, tag):
        quads.append(np.stack(q, axis=-1).reshape(-1, 4))
        normals.append(np.broadcast_to(np.asarray(nrm, float), (quads[-1].shape[0], 3)))
        tags.append(np.full(quads[-1].shape[0], tag))

    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    cell_i, cell_j = {}, {}
    for lz, sgn, keep, tag in ((0, -1.0, None, 0), (1, 1.0, ~hole, 1), (top_in, -1.0, ~hole, 2),
                               (top_out, 1.0, None, 3)):
        ci, cj = (ii, jj) if keep is None else (ii[keep], jj[keep])
        ci, cj = ci.ravel(), cj.ravel()
        cell_i[tag], cell_j[tag] = ci, cj
        add((code(lz, ci, cj), code(lz, ci + 1, cj), code(lz, ci + 1, cj + 1), code(lz, ci, cj + 1)),
            (0.0, 0.0, sgn), tag)
    r = np.arange(n)
    for l0, l1 in ((0, 1), (top_in, top_out)):        # plane sides
        for fixed, axis, sgn in ((0, 0, -1.0), (n, 0, 1.0), (0, 1, -1.0), (n, 1, 1.0)):
            nrm = np.zeros(3)
            nrm[axis] = sgn
            if axis == 0:
                q = (code(l0, fixed, r), code(l0, fixed, r + 1), code(l1, fixed, r + 1), code(l1, fixed, r))
            else:
                q = (code(l0, r, fixed), code(l0, r + 1, fixed), code(l1, r + 1, fixed), code(l1, r, fixed))
            add(q, nrm, 4)
    kk = np.arange(via_k)
    lv = np.arange(1, 1 + m_gap)
    for i0, j0 in vias:                               # via walls
        K, Lv = np.meshgrid(kk, lv, indexing="ij")
        for fixed, axis, sgn in ((i0, 0, -1.0), (i0 + via_k, 0, 1.0), (j0, 1, -1.0), (j0 + via_k, 1, 1.0)):
            nrm = np.zeros(3)
            nrm[axis] = sgn
            if axis == 0:
                a = j0 + K
                q = (code(Lv, fixed, a), code(Lv, fixed, a + 1), code(Lv + 1, fixed, a + 1), code(Lv + 1, fixed, a))
            else:
                a = i0 + K
                q = (code(Lv, a, fixed), code(Lv, a + 1, fixed), code(Lv + 1, a + 1, fixed), code(Lv + 1, a, fixed))
            add(q, nrm, 5)
    Q = np.concatenate(quads)
    nrm = np.concatenate(normals)
    tag = np.concatenate(tags)
    used, inv = np.unique(Q.ravel(), return_inverse=True)
    Q = inv.reshape(Q.shape)
    lz = used // ((n + 1) * (n + 1))
    rem = used % ((n + 1) * (n + 1))
    vi, vj = rem // (n + 1), rem % (n + 1)
    xyz = np.stack([vi * h, vj * h, zlev[lz]], axis=1)
    if jitter > 0.0:
        outer = ((lz == 0) | (lz == top_out)) & (vi > 0) & (vi < n) & (vj > 0) & (vj < n)
        xyz[outer, :2] += rng.uniform(-jitter, jitter, (int(outer.sum()), 2)) * h
    par = np.arange(Q.shape[0]) % 2
    t0 = np.where(par[:, None] == 0, Q[:, [0, 1, 2]], Q[:, [0, 1, 3]])
    t1 = np.where(par[:, None] == 0, Q[:, [0, 2, 3]], Q[:, [1, 2, 3]])
    tris = np.empty((2 * Q.shape[0], 3), np.int64)
    tris[0::2], tris[1::2] = t0, t1
    tris = _orient(xyz, tris, np.repeat(nrm, 2, axis=0))
    tri_tag = np.repeat(tag, 2)
    # triangle ids of the two outer faces by cell (both triangles of a quad)
    qid = {f: np.nonzero(tag == f)[0] for f in (0, 3)}
    ports = []
    for I, J in pad_sites:
        a0, b0 = I * site + 3, J * site + 3
        sets = []
        for f in (3, 0):
            inpad = ((cell_i[f] >= a0) & (cell_i[f] < a0 + pad_k) & (cell_j[f] >= b0) & (cell_j[f] < b0 + pad_k))
            qs = qid[f][inpad]
            sets.append(np.sort(np.concatenate([2 * qs, 2 * qs + 1])).astype(np.int32))
        ports.append((sets[0], sets[1]))
    for src, snk in ports:
        assert np.all(tri_tag[src] == 3) and np.all(tri_tag[snk] == 0)
    return Mesh(xyz=xyz, tri=tris.astype(np.int32), cond=np.zeros(tris.shape[0], np.int32),
                sigma=np.array([sigma], dtype=np.float64), ports=ports, name=name)


def extruded_cells_mesh(mask, c, t, nz, src_edges, snk_edges, jitter=0.0, seed=0, sigma=5.8e7, name="extruded"):
    """Closed surface of the region of occupied cells `mask` [nx, ny] (cell size
    c) extruded through thickness t: a top and a bottom quad per cell, and wall
    quads (nz divisions in height) on every lattice edge between an occupied
    and an empty cell.  Port contacts are the wall triangles on the lattice
    edges listed in src_edges / snk_edges, given as (axis, i, j): the edge on
    lattice line x = i between y = j and j + 1 (axis 0) or on y = j between
    x = i and i + 1 (axis 1).  Top and bottom vertices strictly inside the
    region get an in-plane jitter of +-jitter c."""
    rng = np.random.default_rng(seed)
    mask = np.asarray(mask, bool)
    nx, ny = mask.shape
    occ = np.zeros((nx + 2, ny + 2), bool)
    occ[1:-1, 1:-1] = mask

    def code(k, i, j):
        return (np.asarray(k) * (nx + 1) + np.asarray(i)) * (ny + 1) + np.asarray(j)

    quads, normals, edge_key = [], [], []
    ci, cj = np.nonzero(mask)
    for k, sgn in ((0, -1.0), (nz, 1.0)):
        quads.append(np.stack([code(k, ci, cj), code(k, ci + 1, cj), code(k, ci + 1, cj + 1), code(k, ci, cj + 1)],
                              axis=-1))
        normals.append(np.broadcast_to([0.0, 0.0, sgn], (ci.size, 3)))
        edge_key.append(np.full(ci.size, -1, np.int64))
    kz = np.arange(nz)
    # walls on x-lines: between cells (i-1, j) and (i, j)
    a, b = occ[:-1, 1:-1], occ[1:, 1:-1]                 # [nx+1, ny]: left / right cell of line i
    for side, sgn in ((a & ~b, 1.0), (~a & b, -1.0)):
        li, lj = np.nonzero(side)
        I, K = np.broadcast_arrays(li[:, None], kz[None, :])
        J = np.broadcast_to(lj[:, None], I.shape)
        quads.append(np.stack([code(K, I, J), code(K, I, J + 1), code(K + 1, I, J + 1), code(K + 1, I, J)],
                              axis=-1).reshape(-1, 4))
        normals.append(np.broadcast_to([sgn, 0.0, 0.0], (I.size, 3)))
        edge_key.append((0 * (nx + 1) + I.ravel()) * (ny + 1) + J.ravel())
    # walls on y-lines: between cells (i, j-1) and (i, j)
    a, b = occ[1:-1, :-1], occ[1:-1, 1:]                 # [nx, ny+1]
    for side, sgn in ((a & ~b, 1.0), (~a & b, -1.0)):
        li, lj = np.nonzero(side)
        I, K = np.broadcast_arrays(li[:, None], kz[None, :])
        J = np.broadcast_to(lj[:, None], I.shape)
        quads.append(np.stack([code(K, I, J), code(K, I + 1, J), code(K + 1, I + 1, J), code(K + 1, I, J)],
                              axis=-1).reshape(-1, 4))
        normals.append(np.broadcast_to([0.0, sgn, 0.0], (I.size, 3)))
        edge_key.append(((nx + 1) * (ny + 1)) + I.ravel() * (ny + 1) + J.ravel())
    Q = np.concatenate(quads)
    nrm = np.concatenate(normals)
    ekey = np.concatenate(edge_key)
    used, inv = np.unique(Q.ravel(), return_inverse=True)
    Q = inv.reshape(Q.shape)
    k = used // ((nx + 1) * (ny + 1))
    rem = used % ((nx + 1) * (ny + 1))
    vi, vj = rem // (ny + 1), rem % (ny + 1)
    xyz = np.stack([vi * c, vj * c, k * (t / nz)], axis=1).astype(np.float64)
    if jitter > 0.0:
        # a vertex is inside the region when its four surrounding cells are occupied
        inside = occ[vi, vj] & occ[vi + 1, vj] & occ[vi, vj + 1] & occ[vi + 1, vj + 1]
        move = inside & ((k == 0) | (k == nz))
        xyz[move, :2] += rng.uniform(-jitter, jitter, (int(move.sum()), 2)) * c
    par = np.arange(Q.shape[0]) % 2
    tris = np.empty((2 * Q.shape[0], 3), np.int64)
    tris[0::2] = np.where(par[:, None] == 0, Q[:, [0, 1, 2]], Q[:, [0, 1, 3]])
    tris[1::2] = np.where(par[:, None] == 0, Q[:, [0, 2, 3]], Q[:, [1, 2, 3]])
    tris = _orient(xyz, tris, np.repeat(nrm, 2, axis=0))
    tkey = np.repeat(ekey, 2)

    def contact(edges):
        keys = [(ax * (nx + 1) * (ny + 1)) + i * (ny + 1) + j for ax, i, j in edges]
        return np.nonzero(np.isin(tkey, keys))[0].astype(np.int32)

    ports = [(contact(src_edges), contact(snk_edges))]
    return Mesh(xyz=xyz, tri=tris.astype(np.int32), cond=np.zeros(tris.shape[0], np.int32),
                sigma=np.array([sigma], dtype=np.float64), ports=ports, name=name)


def meander_mesh(n_seg, w, t, run, kw=2, gap_w=1.0, jitter=0.1, seed=0, sigma=5.8e7, name="meander"):
    """Serpentine trace of width w and thickness t: n_seg segments alternating
    runs of length `run` along x and jogs along y with right-angle corners
    (the runs 2 gap_w w apart centre line to centre line minus w), on a lattice
    of cell size w / kw, walls divided in height like the cell size.  One port
    from the free end face of the first run (source) to that of the last run."""
    c = w / kw
    nr = max(2, (n_seg + 1) // 2)
    gap = max(1, int(round(gap_w * kw)))
    L = max(3 * kw, int(round(run / c)))
    nx, ny = L, nr * kw + (nr - 1) * gap
    mask = np.zeros((nx, ny), bool)
    for r in range(nr):
        y0 = r * (kw + gap)
        mask[:, y0:y0 + kw] = True
        if r + 1 < nr:                       # jog to the next run: right end after even runs, left after odd
            xs = slice(nx - kw, nx) if r % 2 == 0 else slice(0, kw)
            mask[xs, y0:y0 + 2 * kw + gap] = True
    nz = max(1, int(round(t / c)))
    src = [(0, 0, j) for j in range(kw)]
    y_last = (nr - 1) * (kw + gap)
    i_end = nx if (nr - 1) % 2 == 0 else 0   # the last run's free end
    snk = [(0, i_end, y_last + j) for j in range(kw)]
    return extruded_cells_mesh(mask, c, t, nz, src, snk, jitter=jitter, seed=seed, sigma=sigma, name=name)
