"""Convenience wrapper over the C ABI: one ``Solver`` per lattice.

Marshalling only (see ``binding``): gauge fields, sources and solutions are
complex128 numpy arrays (host) or torch CUDA tensors (device), in the ABI
layouts; every operation runs in libmgclover.
"""
from __future__ import annotations

import numpy as np

from . import binding as B


def solve_batch(solvers, etas, tol: float = 1e-10, outs=None):
    """Solve several lattices together (``mg_solve_batch``): ``etas[i]`` holds the
    right-hand sides of ``solvers[i]`` (shape ``(nrhs_i, Lt, Lz, Ly, Lx, 4, 3)``
    or a single source).  Returns ``(outs, infos)``."""
    if outs is None:
        outs = [e.new_zeros(e.shape) if not isinstance(e, np.ndarray) else np.zeros_like(e) for e in etas]
    nrhs = [1 if e.ndim == 6 else e.shape[0] for e in etas]
    st, infos = B.mg_solve_batch([s.ctx for s in solvers], outs, etas, nrhs, tol)
    return outs, infos


class Solver:
    """``[D(U) + m] psi = eta`` on one lattice ``dims = (Lx, Ly, Lz, Lt)``."""

    def __init__(self, dims, device: int = 0, stream: int | None = None):
        self.dims = tuple(int(d) for d in dims)
        self.ctx = B.mg_create(self.dims, device, stream)
        self.params = B.mg_default_params()
        self.gauge_ref = None
        self.gauge_version = None

    # -- lifecycle
    def close(self):
        if self.ctx is not None:
            B.mg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):  # pragma: no cover - best effort
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- configuration
    def load_gauge(self, U):
        B.mg_load_gauge(self.ctx, U)
        # the field the operator was built from (checked by the autograd Function)
        self.gauge_ref = U
        self.gauge_version = getattr(U, "_version", None)

    def set_clover(self, csw: float, m0: float):
        B.mg_set_clover(self.ctx, csw, m0)

    def set_clover_aniso(self, weights, csw_s: float, csw_t: float, m0: float):
        """Anisotropic operator: hop weights ``(w_x, w_y, w_z, w_t)``, mass term
        ``sum(w) + m0``, clover coefficient ``csw_t`` on the planes containing t."""
        B.mg_set_clover_aniso(self.ctx, weights, csw_s, csw_t, m0)

    def set_params(self, levels=None, blocks=None, nv=None, **kw):
        p = self.params
        if levels is not None:
            p.levels = int(levels)
        if blocks is not None:
            for l, b in enumerate(blocks):
                for m in range(4):
                    p.block[l][m] = int(b[m])
        if nv is not None:
            for l, n in enumerate(nv):
                p.nv[l] = int(n)
        for k, v in kw.items():
            if not hasattr(p, k):
                raise AttributeError(f"mg_params has no field {k}")
            setattr(p, k, v)
        B.mg_set_params(self.ctx, p)

    def set_null_vectors(self, level: int, V):
        B.mg_set_null_vectors(self.ctx, level, V, V.shape[0])

    def get_null_vectors(self, level: int):
        dims, ndof = self.level_info(level)
        out = np.zeros((self.params.nv[level], dims[3], dims[2], dims[1], dims[0], ndof), dtype=np.complex128)
        B.mg_get_null_vectors(self.ctx, level, out, out.shape[0])
        return out

    def coarse_links(self, level: int):
        """Dequantised coarse links ``(Y, X)`` of a coarse level: ``Y`` shaped
        ``(Tc, Zc, Yc, Xc, 8, nc, nc)``, ``X`` shaped ``(Tc, Zc, Yc, Xc, nc, nc)``."""
        dims, nc = self.level_info(level)
        shp = (dims[3], dims[2], dims[1], dims[0])
        Y = np.zeros(shp + (8, nc, nc), dtype=np.complex128)
        X = np.zeros(shp + (nc, nc), dtype=np.complex128)
        B.mg_get_coarse_links(self.ctx, level, Y, X)
        return Y, X

    def save_setup(self, path: str):
        B.mg_save_setup(self.ctx, path)

    def load_setup(self, path: str):
        """Parameters and null vectors from a saved setup; the hierarchy is rebuilt for the current field."""
        info = B.mg_load_setup(self.ctx, path)
        self.params = B.mg_get_params(self.ctx)
        return info

    def update_mass(self, m0: float):
        """New bare mass, hierarchy rebuilt from the current null vectors (no inverse iteration)."""
        return B.mg_update_mass(self.ctx, m0)

    def adapt_setup(self, passes: int = 1, relax: int = 2, transfers: int = 1):
        """Adaptive refinement: relax the null vectors of the `transfers` finest transfers (0: all)
        with the current solver and rebuild."""
        return B.mg_adapt_setup(self.ctx, passes, relax, transfers)

    def setup(self):
        return B.mg_setup(self.ctx)

    def level_info(self, level: int):
        return B.mg_level_info(self.ctx, level)

    # -- work
    def solve(self, eta, tol: float = 1e-10, mode: int = B.MG_MODE_MG, out=None, allow_not_converged=False):
        """Solve for eta of shape ``(Lt, Lz, Ly, Lx, 4, 3)`` or ``(nrhs, ...)``."""
        nrhs = 1 if eta.ndim == 6 else eta.shape[0]
        if out is None:
            out = eta.new_zeros(eta.shape) if not isinstance(eta, np.ndarray) else np.zeros_like(eta)
        st, info = B.mg_solve(self.ctx, out, eta, nrhs, tol, mode, allow_not_converged)
        return out, info

    def solve_dagger(self, eta, tol: float = 1e-10, mode: int = B.MG_MODE_MG, out=None, allow_not_converged=False):
        """Solve ``D^dag psi = eta`` (same shapes as :meth:`solve`)."""
        nrhs = 1 if eta.ndim == 6 else eta.shape[0]
        if out is None:
            out = eta.new_zeros(eta.shape) if not isinstance(eta, np.ndarray) else np.zeros_like(eta)
        st, info = B.mg_solve_dagger(self.ctx, out, eta, nrhs, tol, mode, allow_not_converged)
        return out, info

    def force(self, lam, psi, kind: int = B.MG_FORCE_SU3, out=None):
        """Derivative of ``-Re<lam, D(U) psi>`` with respect to the links, shaped like the gauge field."""
        shape = tuple(psi.shape[:4]) + (4, 3, 3)
        if out is None:
            out = np.zeros(shape, dtype=np.complex128) if isinstance(psi, np.ndarray) else psi.new_zeros(shape)
        B.mg_force(self.ctx, out, lam, psi, kind)
        return out

    def apply(self, op: int, x, level: int = 0, prec: int = B.MG_FP64, out_shape=None, nrhs: int = 1):
        """Apply operator ``op`` of ``level`` to ``nrhs`` consecutive vectors in ``x``."""
        if out_shape is None:
            out = x.new_zeros(x.shape) if not isinstance(x, np.ndarray) else np.zeros_like(x)
        else:
            out = np.zeros(out_shape, dtype=np.complex128) if isinstance(x, np.ndarray) else x.new_zeros(out_shape)
        B.mg_apply(self.ctx, op, level, out, x, nrhs, prec)
        return out
