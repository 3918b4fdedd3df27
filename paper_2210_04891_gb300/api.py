"""Python binding of libsie: argument marshalling only.

Every step of the method runs in the library (host graph code and CUDA
kernels); this module converts numpy/torch arguments to the C ABI of
include/sie.h and raises SieError on any non-zero return code.  Device
buffers are torch tensors (complex128, CUDA); streams are torch streams.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import native as N
from .native import check, lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


class Mesh:
    def __init__(self, xyz, tri, cond, sigma):
        self._keep = [np.ascontiguousarray(xyz, np.float64), np.ascontiguousarray(tri, np.int32),
                      np.ascontiguousarray(cond, np.int32), np.ascontiguousarray(sigma, np.float64)]
        xyz, tri, cond, sigma = self._keep
        h = ctypes.c_void_p()
        check(lib().sie_mesh_load(_ptr(xyz), xyz.shape[0], _ptr(tri), tri.shape[0], _ptr(cond), _ptr(sigma),
                                  sigma.shape[0], ctypes.byref(h)))
        self.h = h
        self.nt = tri.shape[0]
        self.ncond = sigma.shape[0]

    @classmethod
    def from_synth(cls, m):
        return cls(m.xyz, m.tri, m.cond, m.sigma)

    @classmethod
    def from_file(cls, path, nt=None, ncond=None):
        """Load a mesh file (sie_mesh_load_file); nt and ncond are read from its
        size line when not given."""
        self = cls.__new__(cls)
        self._keep = []
        if nt is None or ncond is None:
            nt, ncond = _mesh_file_sizes(path)
        h = ctypes.c_void_p()
        check(lib().sie_mesh_load_file(os.fsencode(path), ctypes.byref(h)))
        self.h, self.nt, self.ncond = h, nt, ncond
        return self

    def __del__(self):
        if getattr(self, "h", None) and lib is not None:
            lib().sie_mesh_destroy(self.h)
            self.h = None


def sie_mesh_load(xyz, tri, cond, sigma):
    return Mesh(xyz, tri, cond, sigma)


def sie_mesh_load_file(path):
    return Mesh.from_file(path)


def write_mesh_file(path, xyz, tri, cond, sigma):
    """Write the text format sie_mesh_load_file reads (17 significant digits)."""
    xyz = np.asarray(xyz, np.float64).reshape(-1, 3)
    tri = np.asarray(tri, np.int64).reshape(-1, 3)
    cond = np.asarray(cond, np.int64).reshape(-1)
    sigma = np.asarray(sigma, np.float64).reshape(-1)
    with open(path, "w") as f:
        f.write("sie_mesh 1\n# nv nt ncond\n%d %d %d\n" % (xyz.shape[0], tri.shape[0], sigma.shape[0]))
        f.write(" ".join("%.17g" % s for s in sigma) + "\n")
        for x in xyz:
            f.write("%.17g %.17g %.17g\n" % tuple(x))
        for t, c in zip(tri, cond):
            f.write("%d %d %d %d\n" % (t[0], t[1], t[2], c))


def _mesh_file_sizes(path):
    with open(path) as f:
        toks = []
        for line in f:
            toks += line.split("#", 1)[0].split()
            if len(toks) >= 5:
                return int(toks[3]), int(toks[4])
    raise ValueError("%s: no size line" % path)


class Loops:
    def __init__(self, mesh: Mesh, ports):
        self.mesh = mesh
        arrs = []
        P = (N.SiePort * max(1, len(ports)))()
        for i, (src, snk) in enumerate(ports):
            s = np.ascontiguousarray(src, np.int32)
            k = np.ascontiguousarray(snk, np.int32)
            arrs += [s, k]
            P[i].src = s.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            P[i].n_src = s.shape[0]
            P[i].sink = k.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            P[i].n_sink = k.shape[0]
        st = N.SieLoopStats()
        h = ctypes.c_void_p()
        check(lib().loop_basis_build(mesh.h, P, len(ports), ctypes.byref(h), ctypes.byref(st)))
        self.h = h
        self.stats = {f: getattr(st, f) for f, _ in N.SieLoopStats._fields_}
        self.nl = st.n_loops
        self.nb = st.n_branches
        self.np = st.n_ports

    def export(self):
        """(row_ptr, col, val, br_tri) of the loop matrix A and the branch triangles."""
        s = self.stats
        row_ptr = np.zeros(s["n_loops"] + 1, np.int64)
        col = np.zeros(s["nnz_A"], np.int32)
        val = np.zeros(s["nnz_A"], np.int8)
        br = np.zeros((s["n_branches"], 2), np.int32)
        check(lib().sie_loops_export(self.h, _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(br)))
        return row_ptr, col, val, br

    def __del__(self):
        if getattr(self, "h", None):
            lib().sie_loops_destroy(self.h)
            self.h = None


def loop_basis_build(mesh, ports):
    return Loops(mesh, ports)


DEFAULT_PARAMS = dict(grid=(16, 8, 8), order=3, near_factor=4.0, near_min_diam=2.0, n_touch=16, h0=0.0)


def _c_params(p):
    cp = N.PfftParams()
    for i in range(3):
        cp.grid[i] = int(p["grid"][i])
    cp.order = int(p["order"])
    cp.near_factor = float(p["near_factor"])
    cp.near_min_diam = float(p["near_min_diam"])
    cp.n_touch = int(p["n_touch"])
    cp.kernel = int(p.get("kernel", N.KERNEL_STATIC))
    cp.h0 = float(p["h0"])
    return cp


def autotune(mesh, loops, params, nrhs, omega, tol, stream=None):
    """pfft_autotune: (best params dict, report dict) for the geometry."""
    import torch
    p = dict(DEFAULT_PARAMS)
    p.update(params or {})
    torch.cuda.init()
    best = N.PfftParams()
    rep = N.TuneReport()
    check(lib().pfft_autotune(mesh.h, loops.h, ctypes.byref(_c_params(p)), int(nrhs), float(omega), float(tol),
                              _stream(stream), ctypes.byref(best), ctypes.byref(rep)))
    out = dict(p, grid=tuple(best.grid[i] for i in range(3)), near_factor=best.near_factor)
    n = rep.n_tried
    report = dict(best=rep.best, grids=[tuple(rep.grid[c][i] for i in range(3)) for c in range(n)],
                  ms=[rep.ms[c] for c in range(n)], err=[rep.err[c] for c in range(n)])
    return out, report


class Plan:
    def __init__(self, mesh: Mesh, loops: Loops, params=None, stream=None):
        import torch
        p = dict(DEFAULT_PARAMS)
        p.update(params or {})
        self.params = p
        cp = _c_params(p)
        torch.cuda.init()
        h = ctypes.c_void_p()
        check(lib().pfft_plan_create(mesh.h, loops.h, ctypes.byref(cp), _stream(stream), ctypes.byref(h)))
        self.h = h
        self.mesh, self.loops = mesh, loops      # the plan borrows the loop basis
        self.nl, self.nb, self.np = loops.nl, loops.nb, loops.np

    def set_surface_model(self, t_eff=None):
        """Slab surface impedance with effective thickness t_eff[c] per conductor
        (None or 0: the classic form); see pfft_plan_set_surface_model."""
        nc = self.mesh.ncond
        if t_eff is None:
            check(lib().pfft_plan_set_surface_model(self.h, None, nc))
            return
        t = np.ascontiguousarray(np.broadcast_to(np.asarray(t_eff, dtype=np.float64), (nc,)))
        check(lib().pfft_plan_set_surface_model(self.h, t.ctypes.data_as(ctypes.c_void_p), nc))

    def info(self):
        v = [ctypes.c_int64() for _ in range(4)]
        gh = (ctypes.c_double * 3)()
        rn = ctypes.c_double()
        db = ctypes.c_int64()
        check(lib().pfft_plan_info(self.h, *[ctypes.byref(x) for x in v], gh, ctypes.byref(rn), ctypes.byref(db)))
        return dict(n_loops=v[0].value, n_branches=v[1].value, n_tri=v[2].value, n_near_pairs=v[3].value,
                    grid_h=list(gh), r_near=rn.value, device_bytes=db.value)

    def export(self, what):
        """Copy a setup array to the host (see pfft_plan_export in include/sie.h)."""
        info = self.info()
        nt, nn = info["n_tri"], info["n_near_pairs"]
        g = self.params["grid"]
        shapes = {N.EXPORT_NEAR_PTR: ((nt + 1,), np.int64), N.EXPORT_NEAR_COL: ((nn,), np.int32),
                  N.EXPORT_LD: ((nn, 3, 3), np.float64), N.EXPORT_LDIRECT: ((nn, 3, 3), np.float64),
                  N.EXPORT_HHAT: ((g[1] + 1, g[2] + 1, g[0] + 1), np.float64),
                  N.EXPORT_START: ((nt, 7, 3), np.int32)}
        if what in (N.EXPORT_PROJ_NODE, N.EXPORT_PROJ_W):
            npair = int(self.export(N.EXPORT_PROJ_PTR)[-1])
            shapes[N.EXPORT_PROJ_NODE] = ((npair,), np.int32)
            shapes[N.EXPORT_PROJ_W] = ((npair, 3, 3), np.float64)
        shapes[N.EXPORT_PROJ_PTR] = ((nt + 1,), np.int64)
        shape, dt = shapes[what]
        out = np.zeros(shape, dt)
        check(lib().pfft_plan_export(self.h, what, _ptr(out), out.nbytes))
        return out

    def profile(self, on=True):
        check(lib().pfft_profile_enable(self.h, int(on)))

    def profile_read(self):
        """{stage: (ms, launches)} accumulated since profile(True)."""
        ms = np.zeros(len(N.STAGES))
        cnt = np.zeros(len(N.STAGES), np.int64)
        check(lib().pfft_profile_read(self.h, _ptr(ms), _ptr(cnt)))
        return {s: (float(ms[i]), int(cnt[i])) for i, s in enumerate(N.STAGES)}

    def launches(self):
        return int(lib().pfft_plan_launches(self.h))

    def __del__(self):
        if getattr(self, "h", None):
            lib().pfft_plan_destroy(self.h)
            self.h = None


def pfft_plan_create(mesh, loops, params=None, stream=None):
    return Plan(mesh, loops, params, stream)


def _check_vec(x, n, name):
    import torch
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.complex128):
        raise TypeError(f"{name} must be a CUDA complex128 tensor")
    if x.dim() != 2 or x.shape[1] != n or not x.is_contiguous():
        raise ValueError(f"{name} must be contiguous [nrhs, {n}]")


def precond_info(plan: Plan):
    """Band width, unknowns and blocks of the preconditioner's banded LDL^T."""
    w, u, b = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
    check(lib().pfft_precond_info(plan.h, ctypes.byref(w), ctypes.byref(u), ctypes.byref(b)))
    return dict(band_width=w.value, unknowns=u.value, blocks=b.value)


def set_kernel_tuning(plan: Plan, near=0, far_slab=0, proj_slab=0, plane_gpc=0):
    """pfft_plan_set_kernel_tuning (all 0: automatic)."""
    t = N.KernelTuning(near=near, far_slab=far_slab, proj_slab=proj_slab, plane_gpc=plane_gpc)
    check(lib().pfft_plan_set_kernel_tuning(plan.h, ctypes.byref(t)))


def get_kernel_tuning(plan: Plan):
    t = N.KernelTuning()
    check(lib().pfft_plan_get_kernel_tuning(plan.h, ctypes.byref(t)))
    return {f: getattr(t, f) for f, _ in N.KernelTuning._fields_}


def autotune_kernels(plan: Plan, nrhs, omega, stream=None):
    """pfft_autotune_kernels: (chosen tuning, [(candidate, ms)])."""
    best = N.KernelTuning()
    rep = N.KernelTuneReport()
    check(lib().pfft_autotune_kernels(plan.h, int(nrhs), float(omega), _stream(stream), ctypes.byref(best),
                                      ctypes.byref(rep)))
    cands = [({f: getattr(rep.cand[i], f) for f, _ in N.KernelTuning._fields_}, rep.ms[i])
             for i in range(rep.n_tried)]
    return {f: getattr(best, f) for f, _ in N.KernelTuning._fields_}, cands


def precond_set_method(plan: Plan, method):
    """pfft_precond_set_method: N.PC_AUTO, N.PC_BAND or N.PC_ND."""
    check(lib().pfft_precond_set_method(plan.h, int(method)))


def precond_nd_info(plan: Plan):
    """Route of the preconditioner and, for nested dissection, its fronts, factor
    entries per frequency, largest front and complex multiply-adds per factorisation."""
    m, f, mf = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    nz, fl = ctypes.c_int64(), ctypes.c_int64()
    check(lib().pfft_precond_nd_info(plan.h, ctypes.byref(m), ctypes.byref(f), ctypes.byref(nz), ctypes.byref(mf),
                                     ctypes.byref(fl)))
    return dict(method=m.value, fronts=f.value, nnz=nz.value, max_front=mf.value, flops=fl.value)


def pfft_matvec(plan: Plan, x, omega, space=N.SPACE_LOOP, prec=N.PREC_FP64, out=None, stream=None):
    """y = A Z_b(omega) A^T x (space=LOOP) or Z_b(omega) x (space=BRANCH), x [nrhs, n]."""
    import torch
    n = plan.nl if space == N.SPACE_LOOP else plan.nb
    _check_vec(x, n, "x")
    om = np.ascontiguousarray(np.broadcast_to(np.asarray(omega, np.float64), (x.shape[0],)))
    y = torch.empty_like(x) if out is None else out
    _check_vec(y, n, "out")
    check(lib().pfft_matvec(plan.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), x.shape[0],
                            _ptr(om), space, prec, _stream(stream)))
    return y


def postprocess(plan: Plan, x, omega=None, prec=N.PREC_FP64, currents=True, voltages=True, potentials=True,
                stream=None):
    """Branch currents A^T x, branch voltage drops Z_b A^T x and panel potentials
    (conductor reference nodes at 0) of loop currents x [nrhs, n_loops]; returns
    the three (None where not asked for)."""
    import torch
    _check_vec(x, plan.nl, "x")
    R = x.shape[0]
    om = None
    if voltages or potentials:
        if omega is None:
            raise ValueError("omega is needed for voltages and potentials")
        om = np.ascontiguousarray(np.broadcast_to(np.asarray(omega, np.float64), (R,)))
    dev = dict(dtype=torch.complex128, device=x.device)
    a = torch.empty((R, plan.nb), **dev) if currents else None
    v = torch.empty((R, plan.nb), **dev) if voltages else None
    phi = torch.empty((R, plan.mesh.nt), **dev) if potentials else None

    def vp(t):
        return ctypes.c_void_p(t.data_ptr() if t is not None else None)
    check(lib().sie_postprocess(plan.h, ctypes.c_void_p(x.data_ptr()), R, _ptr(om) if om is not None else None,
                                prec, vp(a), vp(v), vp(phi), _stream(stream)))
    return a, v, phi


def pfft_convolve(plan: Plan, grid, prec=N.PREC_FP64, stream=None):
    """phi_g = H Q_g in place for grid [nbatch, N_x, N_y, N_z] (complex128 or complex64)."""
    import torch
    g = plan.params["grid"]
    want = torch.complex128 if prec == N.PREC_FP64 else torch.complex64
    if not (grid.is_cuda and grid.dtype == want and grid.is_contiguous() and tuple(grid.shape[1:]) == tuple(g)):
        raise ValueError("grid must be a contiguous CUDA tensor [nbatch, N_x, N_y, N_z] of the precision's dtype")
    check(lib().pfft_convolve(plan.h, ctypes.c_void_p(grid.data_ptr()), grid.shape[0], prec, _stream(stream)))
    return grid


def pfft_convolve_lossy(plan: Plan, grid, omega, sigma, prec=N.PREC_FP64, stream=None):
    """phi_g = H_k Q_g in place with the lossy kernel exp(-jkR)/R, k = (1 - j)/delta (skin depth
    delta of sigma at omega), grid [nbatch, N_x, N_y, N_z] (complex128 or complex64)."""
    import torch
    g = plan.params["grid"]
    want = torch.complex128 if prec == N.PREC_FP64 else torch.complex64
    if not (grid.is_cuda and grid.dtype == want and grid.is_contiguous() and tuple(grid.shape[1:]) == tuple(g)):
        raise ValueError("grid must be a contiguous CUDA tensor [nbatch, N_x, N_y, N_z] of the precision's dtype")
    check(lib().pfft_convolve_lossy(plan.h, ctypes.c_void_p(grid.data_ptr()), grid.shape[0], float(omega),
                                    float(sigma), prec, _stream(stream)))
    return grid


def pfft_precond_apply(plan: Plan, y, omega, out=None, prec=N.PREC_FP64, stream=None):
    """z = P(omega)^-1 y, P = A diag(Z_b) A^T, for y [nrhs, n_loops]."""
    import torch
    _check_vec(y, plan.nl, "y")
    om = np.ascontiguousarray(np.broadcast_to(np.asarray(omega, np.float64), (y.shape[0],)))
    z = torch.empty_like(y) if out is None else out
    _check_vec(z, plan.nl, "out")
    check(lib().pfft_precond_apply(plan.h, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(z.data_ptr()),
                                   y.shape[0], _ptr(om), prec, _stream(stream)))
    return z


class MLP:
    """The learned preconditioner correction's network (sie_mlp_*): f [6] -> H -> H -> g."""

    def __init__(self, hidden=32, seed=0):
        h = ctypes.c_void_p()
        check(lib().sie_mlp_create(int(hidden), int(seed), ctypes.byref(h)))
        self.h = h
        self.hidden = hidden
        self.n = int(lib().sie_mlp_param_count(h))

    def params(self):
        out = np.zeros(self.n, np.float32)
        check(lib().sie_mlp_get_params(self.h, _ptr(out), self.n))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        check(lib().sie_mlp_set_params(self.h, _ptr(p), p.size))

    def forward(self, feats, stream=None):
        import torch
        g = torch.empty(feats.shape[0], dtype=torch.float32, device=feats.device)
        check(lib().sie_mlp_forward(self.h, ctypes.c_void_p(feats.data_ptr()), feats.shape[0],
                                    ctypes.c_void_p(g.data_ptr()), _stream(stream)))
        return g

    def grad(self, feats, target, stream=None):
        gr = np.zeros(self.n, np.float32)
        loss = np.zeros(1, np.float32)
        check(lib().sie_mlp_grad(self.h, ctypes.c_void_p(feats.data_ptr()), ctypes.c_void_p(target.data_ptr()),
                                 feats.shape[0], _ptr(gr), _ptr(loss), _stream(stream)))
        return float(loss[0]), gr

    def train(self, feats, target, steps, lr=1e-2, stream=None):
        losses = np.zeros(steps, np.float32)
        check(lib().sie_mlp_train(self.h, ctypes.c_void_p(feats.data_ptr()), ctypes.c_void_p(target.data_ptr()),
                                  feats.shape[0], int(steps), float(lr), _ptr(losses), _stream(stream)))
        return losses

    def __del__(self):
        if getattr(self, "h", None):
            lib().sie_mlp_destroy(self.h)
            self.h = None


def branch_features(plan, omega, stream=None):
    """[n_branches, 6] float32 CUDA tensor of the learned correction's features."""
    import torch
    f = torch.empty((plan.nb, 6), dtype=torch.float32, device="cuda")
    check(lib().pfft_branch_features(plan.h, float(omega), ctypes.c_void_p(f.data_ptr()), _stream(stream)))
    return f


def branch_probe_target(plan, alpha, omega, stream=None):
    """Per-branch probing targets (float32 [n_branches]) from probe currents alpha [k, n_branches]."""
    import torch
    _check_vec(alpha, plan.nb, "alpha")
    t = torch.empty(plan.nb, dtype=torch.float32, device=alpha.device)
    check(lib().pfft_branch_probe_target(plan.h, ctypes.c_void_p(alpha.data_ptr()), alpha.shape[0], float(omega),
                                         ctypes.c_void_p(t.data_ptr()), _stream(stream)))
    return t


def selftest_bounded_wait(plan, limit_ms=5.0, stream=None):
    """Run the failure-detection self-test; returns the library's code (SIE_ERR_TIMEOUT expected)."""
    return lib().sie_selftest_bounded_wait(plan.h, float(limit_ms), _stream(stream))


def set_learned(plan, mlp):
    """Use mlp (MLP or None) in the plan's preconditioner; the plan keeps a reference."""
    check(lib().pfft_plan_set_learned(plan.h, mlp.h if mlp is not None else None))
    plan._learned = mlp


class Batch:
    """Plans of uneven geometries driven together (sie_batch_*)."""

    def __init__(self, plans):
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p.h.value for p in self.plans])
        h = ctypes.c_void_p()
        check(lib().sie_batch_create(arr, len(self.plans), ctypes.byref(h)))
        self.h = h

    def matvec(self, xs, omegas, space=N.SPACE_LOOP, prec=N.PREC_FP64, graph=True, outs=None, stream=None):
        """[y_i] for plans i, x_i [nrhs_i, n_i] CUDA complex128, omegas[i] [nrhs_i]."""
        import torch
        n = len(self.plans)
        if len(xs) != n or len(omegas) != n:
            raise ValueError("one input and one omega array per plan")
        ys = []
        oms = []
        for i, (p, x) in enumerate(zip(self.plans, xs)):
            _check_vec(x, p.nl if space == N.SPACE_LOOP else p.nb, "x")
            y = torch.empty_like(x) if outs is None else outs[i]
            ys.append(y)
            oms.append(np.ascontiguousarray(np.broadcast_to(np.asarray(omegas[i], np.float64), (x.shape[0],))))
        xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
        yp = (ctypes.c_void_p * n)(*[y.data_ptr() for y in ys])
        r = np.array([x.shape[0] for x in xs], np.int32)
        op = (ctypes.c_void_p * n)(*[o.ctypes.data for o in oms])
        check(lib().sie_batch_matvec(self.h, xp, yp, _ptr(r), op, space, prec, int(graph), _stream(stream)))
        return ys

    def stats(self):
        c, r = ctypes.c_int64(), ctypes.c_int64()
        check(lib().sie_batch_stats(self.h, ctypes.byref(c), ctypes.byref(r)))
        return dict(captures=c.value, replays=r.value)

    def solve(self, freqs, ports=None, tol=1e-6, restart=200, max_iter=2000, precond=1, prec=N.PREC_FP64,
              refine=False, graph=False):
        """[(Z_i, stats_i)] of sie_solve for every plan at once; freqs[i] per plan.
        graph=True: sie_batch_solve_graph (one graph replay per Arnoldi step of all plans)."""
        n = len(self.plans)
        fs = [np.ascontiguousarray(f, np.float64) for f in freqs]
        prs = [np.arange(p.np, dtype=np.int32) if ports is None or ports[i] is None
               else np.ascontiguousarray(ports[i], np.int32) for i, p in enumerate(self.plans)]
        Zs = [np.zeros((f.shape[0], q.shape[0], q.shape[0]), np.complex128) for f, q in zip(fs, prs)]
        o = N.SolveOpts(tol=tol, restart=restart, max_iter=max_iter, precond=precond, prec=prec, refine=int(refine))
        st = (N.SolveStats * n)()
        fp = (ctypes.c_void_p * n)(*[f.ctypes.data for f in fs])
        nf = np.array([f.shape[0] for f in fs], np.int32)
        pp = (ctypes.c_void_p * n)(*[q.ctypes.data for q in prs])
        npr = np.array([q.shape[0] for q in prs], np.int32)
        zp = (ctypes.c_void_p * n)(*[z.ctypes.data for z in Zs])
        fn = lib().sie_batch_solve_graph if graph else lib().sie_batch_solve
        rc = fn(self.h, fp, _ptr(nf), pp, _ptr(npr), ctypes.byref(o), zp, st)
        if rc not in (N.SIE_OK, -6):
            check(rc)
        out = []
        for i in range(n):
            d = {k: getattr(st[i], k) for k, _ in N.SolveStats._fields_}
            d["converged"] = d["n_not_converged"] == 0
            out.append((Zs[i], d))
        return out

    def __del__(self):
        if getattr(self, "h", None):
            lib().sie_batch_destroy(self.h)
            self.h = None


def sie_solve(plan: Plan, freqs, ports=None, tol=1e-6, restart=200, max_iter=2000, precond=1,
              prec=N.PREC_FP64, refine=False):
    """Port impedances Z[f] by preconditioned loop-basis GMRES (Eq. LoopWithP).
    refine (with prec = PREC_MIXED): False / REFINE_OFF all mixed, True / REFINE_FP64
    iterative refinement with FP64 residual products, REFINE_DF the same with
    double-float residual products."""
    f = np.ascontiguousarray(freqs, np.float64)
    pr = np.arange(plan.np, dtype=np.int32) if ports is None else np.ascontiguousarray(ports, np.int32)
    o = N.SolveOpts(tol=tol, restart=restart, max_iter=max_iter, precond=precond, prec=prec, refine=int(refine))
    Z = np.zeros((f.shape[0], pr.shape[0], pr.shape[0]), np.complex128)
    st = N.SolveStats()
    rc = lib().sie_solve(plan.h, _ptr(f), f.shape[0], _ptr(pr), pr.shape[0], ctypes.byref(o), _ptr(Z),
                         ctypes.byref(st))
    stats = {k: getattr(st, k) for k, _ in N.SolveStats._fields_}
    if rc not in (N.SIE_OK, -6):
        check(rc)
    stats["converged"] = rc == N.SIE_OK
    return Z, stats
