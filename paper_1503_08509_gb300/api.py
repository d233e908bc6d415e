"""Python front end of the FE-P3M library.

Thin marshalling over the C ABI (include/fep3m.h): torch supplies device
memory and the CUDA stream; every step of the method runs in the library's
CUDA kernels.  Inputs may be CUDA tensors (device path, no copies) or numpy
arrays / CPU tensors (host path: the library stages the copies itself).
"""
import ctypes

import numpy as np
import torch

from . import _lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        return ctypes.c_void_p(x.ctypes.data)
    raise TypeError("expected a torch.Tensor or numpy.ndarray, got %r" % type(x))


def _f64(x, shape):
    if isinstance(x, torch.Tensor):
        if x.dtype != torch.float64 or not x.is_contiguous():
            x = x.to(torch.float64).contiguous()
    else:
        x = np.ascontiguousarray(x, dtype=np.float64)
    if tuple(x.shape) != tuple(shape):
        raise ValueError("expected shape %s, got %s" % (shape, tuple(x.shape)))
    return x


class FEP3M:
    """One FE-P3M context: mesh, screen tables and mesh solver for a periodic cube.

    precision: 'fp64' or 'mixed' (FP32 pair sums and inner mesh solve, FP64 refinement).
    tensor_cores: False runs the split-precision contractions (the mixed pair
    kernel's screen field, the fast-diagonalisation transforms) on the FP32
    CUDA cores instead of as bf16 tensor-core MMAs.
    solver: the FP32 inner solve of the mesh system's iterative refinement,
    'fdm' (exact, by fast diagonalisation) or 'multigrid' (multigrid-
    preconditioned CG; q = 1).
    q: screen order 1..4 (mesh order q + 2); q >= 2 computes potentials and
    energy (no forces).  one_element: one-element screens (q >= 2).
    dirichlet / neumann: the box [0, L]^3 with Dirichlet data at the mesh's
    nodes (node_points) or Neumann data at the face quadrature points
    (face_points), given by set_boundary (default 0), instead of the periodic
    cube; q = 1, potentials and energy.
    """

    def __init__(self, L, n_el, n_sr=3, precision="fp64", mg_rtol=0.0, mg_max_cycles=0, neutralize=False,
                 table_pad=0, device=None, stream=None, tensor_cores=True, solver="fdm", q=1, one_element=False,
                 dirichlet=False, neumann=False):
        lib = _lib.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.L, self.n_el, self.n_sr, self.q = float(L), int(n_el), int(n_sr), int(q)
        self.precision = precision
        self.dirichlet, self.neumann = bool(dirichlet), bool(neumann)
        cfg = _lib.Config(L=self.L, n_el=self.n_el, q=self.q, n_sr=self.n_sr,
                          precision=_lib.FEP3M_MIXED if precision == "mixed" else _lib.FEP3M_FP64,
                          mg_rtol=mg_rtol, mg_max_cycles=mg_max_cycles, table_pad=table_pad,
                          flags=(_lib.FEP3M_NEUTRALIZE if neutralize else 0) |
                          (0 if tensor_cores else _lib.FEP3M_CUDA_CORES) |
                          (_lib.FEP3M_MULTIGRID if solver == "multigrid" else 0) |
                          (_lib.FEP3M_ONE_ELEMENT if one_element else 0) |
                          (_lib.FEP3M_DIRICHLET if dirichlet else 0) |
                          (_lib.FEP3M_NEUMANN if neumann else 0))
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            h = ctypes.c_void_p()
            _lib.check(lib.fep3m_create(ctypes.byref(cfg), ctypes.c_void_p(self.stream.cuda_stream),
                                        ctypes.byref(h)), "fep3m_create")
        self._h = h
        self.N = 0
        self.generation = 0   # bumped by set_particles: which charges the context holds

    def close(self):
        if getattr(self, "_h", None):
            _lib.load().fep3m_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nodes(self):
        if self.dirichlet or self.neumann:
            return (3 * self.n_el + 1) ** 3
        return ((self.q + 2) * self.n_el) ** 3

    def face_points(self):
        """Points and outward normals (each (6 n^2 NGL^2) x 3) of the Neumann data, in the order of
        fep3m_set_boundary: [face = 2 axis + side][e1][e2][i][j]."""
        n, h, G = self.n_el, self.L / self.n_el, _lib.FEP3M_NEUMANN_NGL
        t = 0.5 * (np.polynomial.legendre.leggauss(G)[0] + 1.0)
        pts, nrm = [], []
        for ax in range(3):
            a1, a2 = (ax + 1) % 3, (ax + 2) % 3
            for side in (0, 1):
                e1, e2, i, j = np.meshgrid(np.arange(n), np.arange(n), np.arange(G), np.arange(G), indexing="ij")
                p = np.zeros(e1.shape + (3,))
                p[..., ax] = side * self.L
                p[..., a1] = (e1 + t[i]) * h
                p[..., a2] = (e2 + t[j]) * h
                v = np.zeros(3)
                v[ax] = 1.0 if side else -1.0
                pts.append(p.reshape(-1, 3))
                nrm.append(np.tile(v, (p.size // 3, 1)))
        return np.concatenate(pts), np.concatenate(nrm)

    def node_points(self):
        """Coordinates (nodes x 3) of the box mesh's nodes, index ix + (3n+1) iy + (3n+1)^2 iz."""
        m = 3 * self.n_el + 1
        t = np.arange(m) * (self.L / (3 * self.n_el))
        z, y, x = np.meshgrid(t, t, t, indexing="ij")
        return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)

    def set_boundary(self, g):
        """Dirichlet data at the box mesh's nodes (only the boundary nodes are read), or Neumann
        data at the face quadrature points (face_points)."""
        size = 6 * self.n_el ** 2 * _lib.FEP3M_NEUMANN_NGL ** 2 if self.neumann else self.nodes
        g = _f64(g, (size,))
        _lib.check(_lib.load().fep3m_set_boundary(self._h, _ptr(g)), "fep3m_set_boundary")

    def set_particles(self, pos, Q):
        N = int(pos.shape[0])
        pos = _f64(pos, (N, 3))
        Q = _f64(Q, (N,))
        self._keep = (pos, Q)   # the device path reads them on the stream
        self.generation += 1
        _lib.check(_lib.load().fep3m_set_particles(self._h, N, _ptr(pos), _ptr(Q)), "fep3m_set_particles")
        self.N = N

    def compute(self, phi=True, energy=True, forces=False, out=None, allow_noconv=False):
        """Returns dict(phi, U, forces).  Outputs are CUDA tensors unless out= gives buffers."""
        N = self.N
        out = dict(out or {})
        if phi and "phi" not in out:
            out["phi"] = torch.empty(N, dtype=torch.float64, device=self.device)
        if forces and "forces" not in out:
            out["forces"] = torch.empty((N, 3), dtype=torch.float64, device=self.device)
        U = ctypes.c_double(0.0)
        st = _lib.load().fep3m_compute(self._h, _ptr(out.get("phi")), ctypes.byref(U) if energy else None,
                                       _ptr(out.get("forces")))
        _lib.check(st, "fep3m_compute", allow=(_lib.FEP3M_ENOCONV,) if allow_noconv else ())
        if energy:
            out["U"] = U.value
        out["status"] = st
        return out

    def vjp(self, gU=1.0, gphi=None, dpos=None, dQ=None):
        N = self.N
        if gphi is not None:
            gphi = _f64(gphi, (N,))
        if dpos is None:
            dpos = torch.empty((N, 3), dtype=torch.float64, device=self.device)
        if dQ is None:
            dQ = torch.empty(N, dtype=torch.float64, device=self.device)
        _lib.check(_lib.load().fep3m_vjp(self._h, float(gU), _ptr(gphi), _ptr(dpos), _ptr(dQ)), "fep3m_vjp")
        return dpos, dQ

    def binning(self):
        N, ne = self.N, self.n_el ** 3
        d = dict(perm=np.empty(N, np.int32), count=np.empty(ne, np.int32), cell=np.empty(N, np.int32),
                 delta=np.empty((N, 3), np.float64))
        _lib.check(_lib.load().fep3m_get_binning(self._h, _ptr(d["perm"]), _ptr(d["count"]), _ptr(d["cell"]),
                                                 _ptr(d["delta"])), "fep3m_get_binning")
        return d

    def mesh(self):
        ne = self.n_el ** 3
        d = dict(C=np.empty((ne, (self.q + 1) ** 3)), b=np.empty(self.nodes), phi_mesh=np.empty(self.nodes))
        _lib.check(_lib.load().fep3m_get_mesh(self._h, _ptr(d["C"]), _ptr(d["b"]), _ptr(d["phi_mesh"])),
                   "fep3m_get_mesh")
        return d

    def solve_mesh(self, b):
        b = _f64(b, (self.nodes,))
        phi = np.empty(self.nodes) if isinstance(b, np.ndarray) else torch.empty_like(b)
        _lib.check(_lib.load().fep3m_solve_mesh(self._h, _ptr(b), _ptr(phi)), "fep3m_solve_mesh",
                   allow=(_lib.FEP3M_ENOCONV,))
        return phi

    def table(self):
        s = 6 * self.n_sr + 7
        t = np.empty(s ** 3)
        _lib.check(_lib.load().fep3m_get_table(self._h, _ptr(t)), "fep3m_get_table")
        return t.reshape(s, s, s)      # [iz, iy, ix]

    def stats(self):
        s = _lib.Stats()
        _lib.check(_lib.load().fep3m_get_stats(self._h, ctypes.byref(s)), "fep3m_get_stats")
        return {k: getattr(s, k) for k, _ in s._fields_}

    def set_timing(self, on=True):
        _lib.check(_lib.load().fep3m_set_timing(self._h, 1 if on else 0), "fep3m_set_timing")


class FEP3MEnergy(torch.autograd.Function):
    """(U, Phi) = FEP3MEnergy.apply(pos, Q, engine); backward uses the library's adjoint.

    The engine holds one set of charges at a time.  The forward saves its
    inputs and the engine's generation; if the engine was given other charges
    before this backward runs (another apply, set_particles), the backward sets
    the saved ones again, so that the adjoint is that of this forward."""

    @staticmethod
    def forward(ctx, pos, Q, engine):
        pos_d, Q_d = pos.detach(), Q.detach()
        engine.set_particles(pos_d, Q_d)
        out = engine.compute(phi=True, energy=True, forces=False)
        ctx.engine = engine
        ctx.generation = engine.generation
        ctx.save_for_backward(pos_d, Q_d)
        U = torch.tensor(out["U"], dtype=torch.float64, device=pos.device)
        return U, out["phi"]

    @staticmethod
    def backward(ctx, gU, gphi):
        eng = ctx.engine
        if eng.generation != ctx.generation:
            pos, Q = ctx.saved_tensors
            eng.set_particles(pos, Q)
            ctx.generation = eng.generation
        gUv = 0.0 if gU is None else float(gU)
        dpos, dQ = eng.vjp(gUv, None if gphi is None else gphi.contiguous())
        return dpos, dQ, None
