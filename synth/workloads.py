"""Named synthetic workloads (geometry, frequencies, grid sizes) and seeded vectors.

The shapes follow the paper's example classes: a straight rectangular copper
interconnect (Sec. V-A), an array of bond wires (Sec. V-B) a power
distribution structure of two planes joined by vias (Sec. V-D), and batches of
meander traces of uneven sizes (the interconnects of a circuit, Sec. V-C).  All sizes are
in metres, conductivities in S/m, frequencies in Hz.
"""
from __future__ import annotations

import numpy as np

from .meshes import box_mesh, wire_array_mesh, merge, plane_pair_mesh, meander_mesh

UM = 1e-6


def bar_1500():
    """Cu bar 1000 x 20 x 10 um, ~1,500 triangles (8 x 10 x 10 um cells),
    in-plane jitter +-15% (seed 1), one port between the x end faces.
    Frequency 1 GHz; pFFT grid 64 x 16 x 16."""
    m = box_mesh(1000 * UM, 20 * UM, 10 * UM, 125, 2, 1, jitter=0.15, seed=1, sigma=5.8e7,
                 name="bar_1000x20x10um")
    return dict(mesh=m, freqs=np.array([1e9]), grid=(64, 16, 16), name="bar_1000x20x10um_1.5k")


def bondwires_40k():
    """8 Au round wires, r = 12.5 um (16-gon), 2 mm long, pitch 100 um,
    axial segment 12.8 um (156 rings, ~40k triangles), axial jitter +-10%
    (seed 2), 8 ports (one per wire, end cap to end cap), 16 log-spaced
    frequencies 1 MHz - 10 GHz; pFFT grid 128 x 64 x 32."""
    m = wire_array_mesh(8, 12.5 * UM, 2000 * UM, 100 * UM, n_sides=16, n_seg=156,
                        jitter=0.10, seed=2, sigma=4.1e7, name="bondwires_8x2mm")
    return dict(mesh=m, freqs=np.logspace(6, 10, 16), grid=(128, 64, 32),
                name="bondwires_8x2mm_40k")


def pdn_500k():
    """PDN-like plane pair: two Cu planes 10 x 10 mm, 35 um thick, 100 um apart,
    on a 40 um cell lattice (~517k triangles), 200 seeded via pairs (square
    80 um vias, 3 divisions across the gap), 4 ports from a pad on the top
    plane's upper face to the pad below it on the bottom plane's lower face,
    8 log-spaced frequencies 1 MHz - 1 GHz; pFFT grid 256 x 256 x 32."""
    m = plane_pair_mesh(L=10e-3, t=35 * UM, gap=100 * UM, n=250, m_gap=3, n_pairs=200, via_k=2, n_ports=4,
                        pad_k=3, site=10, jitter=0.15, seed=11, sigma=5.8e7, name="pdn_2x10mm")
    return dict(mesh=m, freqs=np.logspace(6, 9, 8), grid=(256, 256, 32), name="pdn_2x10mm_500k")


def grid_for(mesh, cell, lo=4, hi=128):
    """pFFT grid per geometry: per axis the power of two nearest above
    extent / cell, clamped to [lo, hi] (the grid spacing follows the panel
    size until the axis cap)."""
    ext = mesh.xyz.max(axis=0) - mesh.xyz.min(axis=0)
    out = []
    for e in ext:
        n = lo
        while n < hi and (n - 1) * cell < e:
            n *= 2
        out.append(n)
    return tuple(out)


def meander(k, n_tri=None):
    """Meander trace k of the batched workload (seed k): segments U{3..12},
    width U(10, 50) um, thickness U(5, 20) um, triangle count log-uniform in
    [5k, 60k] (or about n_tri), 2 cells across the width; one port between
    the free end faces."""
    rng = np.random.default_rng(1000 + k)
    n_seg = int(rng.integers(3, 13))
    w = rng.uniform(10, 50) * UM
    t = rng.uniform(5, 20) * UM
    target = float(np.exp(rng.uniform(np.log(5e3), np.log(6e4)))) if n_tri is None else float(n_tri)
    nr = max(2, (n_seg + 1) // 2)
    # cells across the width such that the runs are about 25 widths long
    kw = int(np.clip(round(np.sqrt(target / (100.0 * nr))), 2, 16))
    c = w / kw
    nz = max(1, int(round(t / c)))
    # per cell of run length: 4 triangles per cell across (top and bottom) and 2 per wall layer on each side
    per_cell_x = 4 * kw * nr + 4 * nr * nz
    run = max(3 * kw, target / per_cell_x) * c
    m = meander_mesh(n_seg, w, t, run, kw=kw, jitter=0.1, seed=k, sigma=5.8e7, name="meander_%d" % k)
    return dict(mesh=m, grid=grid_for(m, c, hi=256), freqs=np.logspace(7, np.log10(5e9), 32), name=m.name)


def meanders_32(n=32, n_tri=None):
    """The batched uneven workload: meanders 0..n-1 (about 1M triangles for 32)."""
    return [meander(k, n_tri) for k in range(n)]


def learned_geometry(seed):
    """A geometry of the learned-preconditioner study (seed): even seeds a
    meander trace, odd seeds a bond-wire array; triangle count log-uniform in
    [5k, 40k].  Meander: the batched workload's generator with that count.
    Bond wires: U{1..8} Au wires, radius U(10, 30) um (16-gon), pitch U(3, 8)
    radii, axial segments as long as a side of the polygon (axial jitter
    +-10%) and as many as the triangle count asks, one port per wire.  Grid
    from grid_for with two panel sizes as the cell."""
    rng = np.random.default_rng(seed)
    target = float(np.exp(rng.uniform(np.log(5e3), np.log(4e4))))
    if seed % 2 == 0:
        w = meander(seed, n_tri=target)
        return dict(w, name="learned_meander_%d" % seed)
    nw = int(rng.integers(1, 9))
    r = rng.uniform(10, 30) * UM
    pitch = rng.uniform(3, 8) * r
    n_sides = 16
    seg = 2 * np.pi * r / n_sides                      # square-ish panels
    n_seg = max(4, int(round(target / (nw * 2 * n_sides) - 1)))
    m = wire_array_mesh(nw, r, n_seg * seg, pitch, n_sides=n_sides, n_seg=n_seg, jitter=0.10, seed=seed,
                        sigma=4.1e7, name="learned_wires_%d" % seed)
    return dict(mesh=m, freqs=np.array([1e9, 1e10]), grid=grid_for(m, 2 * seg),
                name="learned_wires_%d" % seed)


def tiny_pdn(seed=12):
    """Small plane pair (0.6 x 0.6 mm, 25 um cells, 2 via pairs of one-cell vias,
    2 ports, ~4.8k triangles) for oracle checks of the same structure."""
    return plane_pair_mesh(L=0.6e-3, t=35 * UM, gap=100 * UM, n=24, m_gap=3, n_pairs=2, via_k=1, n_ports=2,
                           pad_k=2, site=6, jitter=0.15, seed=seed, sigma=5.8e7, name="tiny_pdn")


def tiny_bar(nx=10, ny=2, nz=1, L=100 * UM, W=20 * UM, T=10 * UM, jitter=0.15, seed=3):
    """Small Cu bar for dense checks (128 triangles at the default sizes)."""
    return box_mesh(L, W, T, nx, ny, nz, jitter=jitter, seed=seed, sigma=5.8e7, name="tiny_bar")


def tiny_wires(n_wires=2, n_sides=8, n_seg=6, length=120 * UM, radius=10 * UM, pitch=40 * UM,
               seed=4):
    """Two short polygonal wires, two ports (multi-port checks)."""
    return wire_array_mesh(n_wires, radius, length, pitch, n_sides=n_sides, n_seg=n_seg,
                           jitter=0.1, seed=seed, sigma=4.1e7, name="tiny_wires")


def tiny_two_bars():
    """Two parallel bars side by side as separate conductors."""
    a = box_mesh(100 * UM, 10 * UM, 10 * UM, 8, 1, 1, jitter=0.1, seed=5, name="a")
    b = box_mesh(100 * UM, 10 * UM, 10 * UM, 8, 1, 1, jitter=0.1, seed=6, name="b",
                 origin=(0.0, 30 * UM, 0.0))
    return merge([a, b], name="tiny_two_bars")


WORKLOADS = {
    "bar_1000x20x10um_1.5k": bar_1500,
    "bondwires_8x2mm_40k": bondwires_40k,
    "pdn_2x10mm_500k": pdn_500k,
    "meanders_32x_5k-60k": meanders_32,
}


def complex_gaussian(n, nrhs=1, seed=7):
    """Seeded complex Gaussian vectors, shape [nrhs, n], complex128."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((nrhs, n)) + 1j * rng.standard_normal((nrhs, n))) / np.sqrt(2.0)
