"""Adaptive multigrid of the oracle: setup, transfer operators, Galerkin coarse
operator, coarse even-odd and the recursive K-cycle MG-GCR solve.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper sections followed:

* "Adaptive multigrid": smoother + coarse solve; R restricts, P prolongs;
  the cycle preconditions an outer GCR.
* "Red-black preconditioning": the coarse operator is ``R D_p P`` (a
  projection of the *full* preconditioned ``D_p``, not of ``D_r``); the coarse
  system is itself solved by its reduced even-odd system; ``P`` comes from
  low modes of ``D_p``; ``R = P^dag gamma_5``; the vectors forming ``P`` are
  split into the two chiralities inside every block.
* "Implementation": the coarse solve is a GCR preconditioned by the next
  level's cycle, down to an unpreconditioned GCR on the coarsest lattice;
  only a residual tolerance (about 0.1) is given per level.  The
  preconditioner runs in single precision, the outer GCR in double.
* "Setup procedure": inverse iteration on a random vector, watching the
  Rayleigh quotient ``v^dag D^dag D v / v^dag v``, with the vector kept
  globally orthogonal to the ones already found.

Readings where the paper is silent (the CUDA path takes the same ones):

* Coarse site = 2 chiralities x Nv vectors (coarse dof ``Nc = 2 Nv``,
  index ``s * Nv + k``); on a coarse level the chirality of dof ``i`` is
  ``i // Nv`` (coarse ``gamma_5 = diag(+1_Nv, -1_Nv)``), which the next
  split uses.
* ``R = P^dag`` is stored instead of ``P^dag gamma_5``: with a chirality-split
  ``P``, ``gamma_5 P = P gamma_5c``, so ``(P^dag g5 D_p P)^{-1} P^dag g5
  = (P^dag D_p P)^{-1} P^dag`` -- the coarse correction is identical.
* Coarse links by directional hops: column ``(s, k)`` of ``P`` on all blocks
  at once, ``u = M^{-1} p``; the term of ``H u`` pulled across a block face in
  direction ``d`` goes to ``Y_d`` of the receiving block, every other term and
  ``P^dag p`` to ``X``.  ``D_hat = X + sum_d Y_d shift_d`` then equals
  ``P^dag D_p P`` (or ``P^dag D P`` with ``op="D"``).
* Cycle (preconditioner of ``D_r``): ``z_e`` = even part of
  ``P D_hat^{-1} R (r_e, 0)``, then ``nu_post`` minimal-residual steps on
  ``D_r`` from the residual ``r_e - D_r z_e`` (``nu_pre`` before, default 0).
  For ``D_p = [[1, X], [Y, 1]]`` the solution of ``D_p u = (r_e, 0)`` has
  ``u_e = D_r^{-1} r_e``, which is why a ``D_p``-based coarse space serves
  ``D_r``.
* Coarse solve: GCR(``restart_coarse``) on the reduced coarse system to
  ``||r|| <= tol_coarse * ||rhs||`` or ``maxit_coarse`` iterations; a coarsest
  lattice with an odd extent is solved without even-odd.
* Setup: start vector from Philox (``oracle.philox``); repeat
  ``v <- GCR_{setup_inner}(D_p, v)`` (zero start, no restart), project out the
  vectors found so far (classical Gram-Schmidt, twice), normalise,
  ``RQ = ||D_p v||^2``; stop when ``|RQ - RQ_prev| < setup_rq_tol * RQ`` or
  after ``setup_iters`` passes.
* Block Gram-Schmidt per (block, chirality): modified Gram-Schmidt, each
  vector projected twice; a vector whose norm drops below ``1e-10`` of its
  norm before projection is a breakdown (``GSBreakdown``), never silently
  fixed.
* Outer stop: ``||r_r|| <= 0.5 tol ||eta||``, then the true residual
  ``||eta - D psi|| / ||eta||`` is checked; GCR continues if it is above tol.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .dirac import LatticeLevel, inner, norm2, shift
from .krylov import SolveInfo, fgcr, mr
from .philox import gaussian_vector


class GSBreakdown(RuntimeError):
    pass


# ----------------------------------------------------------------------------- transfer
class Transfer:
    """Prolongation ``P`` (and ``R = P^dag``) from a level to the next coarser one.

    ``P`` has shape ``fine_shape + (ndof, Nv)``: ``P[x, i, k]`` is row ``(x, i)``
    of column ``(block(x), chir(i), k)``.  ``block = (bx, by, bz, bt)``."""

    def __init__(self, level: LatticeLevel, block, P: np.ndarray):
        self.level = level
        self.block = tuple(int(b) for b in block)
        bx, by, bz, bt = self.block
        lx, ly, lz, lt = level.dims
        if lx % bx or ly % by or lz % bz or lt % bt:
            raise ValueError("block does not divide the lattice")
        self.cdims = (lx // bx, ly // by, lz // bz, lt // bt)
        self.cshape = (lt // bt, lz // bz, ly // by, lx // bx)
        self.ndof = level.ndof
        self.half = level.ndof // 2
        self.P = P
        self.nv = P.shape[-1]

    def _split(self, f):
        """``(Lt, Lz, Ly, Lx, ...)`` -> ``(Tc, bt, Zc, bz, Yc, by, Xc, bx, ...)``."""
        bx, by, bz, bt = self.block
        tc, zc, yc, xc = self.cshape
        return f.reshape((tc, bt, zc, bz, yc, by, xc, bx) + f.shape[4:])

    def block_sum(self, f):
        return self._split(f).sum(axis=(1, 3, 5, 7))

    def block_expand(self, fc):
        bx, by, bz, bt = self.block
        tc, zc, yc, xc = self.cshape
        g = fc[:, None, :, None, :, None, :, None]
        g = np.broadcast_to(g, (tc, bt, zc, bz, yc, by, xc, bx) + fc.shape[4:])
        return g.reshape((tc * bt, zc * bz, yc * by, xc * bx) + fc.shape[4:])

    def restrict(self, v):
        """``r_c[xh, s, k] = sum_{x in xh} sum_{i in chir s} conj(P[x, i, k]) v[x, i]``."""
        h = self.half
        loc0 = np.einsum("...ik,...i->...k", np.conj(self.P[..., :h, :]), v[..., :h])
        loc1 = np.einsum("...ik,...i->...k", np.conj(self.P[..., h:, :]), v[..., h:])
        return self.block_sum(np.concatenate([loc0, loc1], axis=-1))

    def prolong(self, vc):
        """``e[x, i] = sum_k P[x, i, k] v_c[block(x), chir(i), k]``."""
        h, nv = self.half, self.nv
        f = self.block_expand(vc)
        out = np.empty(f.shape[:4] + (self.ndof,), dtype=np.complex128)
        out[..., :h] = np.einsum("...ik,...k->...i", self.P[..., :h, :], f[..., :nv])
        out[..., h:] = np.einsum("...ik,...k->...i", self.P[..., h:, :], f[..., nv:])
        return out


def block_gram_schmidt(level: LatticeLevel, block, vectors, breakdown_tol: float = 1e-10) -> np.ndarray:
    """Chirality split + block Gram-Schmidt of ``vectors`` (list of level vectors)
    into ``P`` of shape ``level.shape + (ndof, Nv)`` (see module header)."""
    nv = len(vectors)
    V = np.stack(vectors, axis=-1)  # (T, Z, Y, X, ndof, Nv)
    T = Transfer(level, block, np.zeros_like(V))
    h = level.ndof // 2
    P = np.zeros_like(V)
    for s in range(2):
        sub = V[..., s * h:(s + 1) * h, :]
        blk = T._split(sub)  # (Tc, bt, Zc, bz, Yc, by, Xc, bx, h, Nv)
        blk = blk.transpose(0, 2, 4, 6, 1, 3, 5, 7, 8, 9)
        cshape = blk.shape[:4]
        inner_shape = blk.shape[4:9]
        Q = blk.reshape((int(np.prod(cshape)), -1, nv)).copy()  # (nblocks, L, Nv)
        for k in range(nv):
            w = Q[:, :, k].copy()
            n0 = np.sqrt(np.sum(np.abs(w) ** 2, axis=1))
            for _ in range(2):
                for j in range(k):
                    d = np.sum(np.conj(Q[:, :, j]) * w, axis=1)
                    w = w - d[:, None] * Q[:, :, j]
            n1 = np.sqrt(np.sum(np.abs(w) ** 2, axis=1))
            if np.any(n1 < breakdown_tol * n0) or np.any(n0 == 0):
                raise GSBreakdown(f"block Gram-Schmidt breakdown at vector {k}, chirality {s}")
            Q[:, :, k] = w / n1[:, None]
        blk = Q.reshape(cshape + inner_shape + (nv,)).transpose(0, 4, 1, 5, 2, 6, 3, 7, 8, 9)
        P[..., s * h:(s + 1) * h, :] = blk.reshape(sub.shape)
    return P


# ----------------------------------------------------------------------------- coarse operator
class CoarseLevel(LatticeLevel):
    """``D_hat v(xh) = X(xh) v(xh) + sum_d Y_d(xh) v(xh + shift_d)`` on a periodic
    coarse lattice; ``M = X``, ``H`` = the Y terms."""

    def __init__(self, dims, X: np.ndarray, Y: np.ndarray):
        super().__init__(dims)
        self.ndof = X.shape[-1]
        self.X = X
        self.Y = Y
        self.Xinv = np.linalg.inv(X)

    def hop_dir(self, v, d):
        mu = d % 4
        nb = shift(v, mu, +1 if d < 4 else -1)
        return np.einsum("...ij,...j->...i", self.Y[d], nb)

    def M(self, v):
        return np.einsum("...ij,...j->...i", self.X, v)

    def Minv(self, v):
        return np.einsum("...ij,...j->...i", self.Xinv, v)


def face_masks(level: LatticeLevel, block):
    """For each direction ``d``: fine sites whose ``d`` neighbour lies in another block."""
    t, z, y, x = np.meshgrid(*[np.arange(n) for n in level.shape], indexing="ij")
    coord = (x, y, z, t)
    masks = []
    for d in range(8):
        mu = d % 4
        b = block[mu]
        if level.dims[mu] // b == 1:
            masks.append(np.zeros(level.shape, dtype=bool))
        elif d < 4:
            masks.append(coord[mu] % b == b - 1)
        else:
            masks.append(coord[mu] % b == 0)
    return masks


def build_coarse(level: LatticeLevel, transfer: Transfer, op: str = "Dp") -> CoarseLevel:
    """Galerkin coarse operator ``P^dag D_p P`` (``op="Dp"``) or ``P^dag D P``
    (``op="D"``) as coarse links ``X``, ``Y_d`` (see module header)."""
    nv, h = transfer.nv, transfer.half
    nc = 2 * nv
    cs = transfer.cshape
    X = np.zeros(cs + (nc, nc), dtype=np.complex128)
    Y = np.zeros((8,) + cs + (nc, nc), dtype=np.complex128)
    faces = [m[..., None] for m in face_masks(level, transfer.block)]
    for s in range(2):
        for k in range(nv):
            col = s * nv + k
            p = level.zeros()
            p[..., s * h:(s + 1) * h] = transfer.P[..., s * h:(s + 1) * h, k]
            if op == "Dp":
                X[..., :, col] += transfer.restrict(p)
                u = level.Minv(p)
            elif op == "D":
                X[..., :, col] += transfer.restrict(level.M(p))
                u = p
            else:
                raise ValueError(op)
            for d in range(8):
                w = level.hop_dir(u, d)
                Y[d][..., :, col] += transfer.restrict(w * faces[d])
                X[..., :, col] += transfer.restrict(w * ~faces[d])
    return CoarseLevel(transfer.cdims, X, Y)


# ----------------------------------------------------------------------------- setup
def setup_null_vectors(level: LatticeLevel, nv: int, seed: int, level_index: int, iters: int = 20,
                       inner_iters: int = 8, rq_tol: float = 0.05, history=None):
    """Inverse iteration for ``nv`` near-null vectors of ``level.Dp`` (module header)."""
    found = []
    for k in range(nv):
        v = gaussian_vector(seed, level_index, k, level.shape, level.ndof)
        rq_prev = None
        rqs = []
        for _ in range(iters):
            v, _ = fgcr(level.Dp, v, tol_abs=0.0, maxiter=inner_iters, restart=inner_iters, true_residual=False)
            for _ in range(2):
                dots = [inner(q, v) for q in found]
                for dq, q in zip(dots, found):
                    v = v - dq * q
            v = v / math.sqrt(norm2(v))
            rq = norm2(level.Dp(v))
            rqs.append(rq)
            if rq_prev is not None and abs(rq - rq_prev) < rq_tol * rq:
                break
            rq_prev = rq
        if history is not None:
            history.append(rqs)
        found.append(v)
    return found


# ----------------------------------------------------------------------------- solver
@dataclass
class MGParams:
    blocks: list                      # per coarse level: (bx, by, bz, bt)
    nv: list                          # per coarse level
    setup_iters: int = 20
    setup_inner: int = 8
    setup_rq_tol: float = 0.05
    nu_pre: int = 0
    nu_post: int = 4
    tol_coarse: float = 0.1
    maxit_coarse: int = 50
    restart_coarse: int = 32
    restart_fine: int = 16
    maxit_fine: int = 500
    seed: int = 3
    coarse_op: str = "Dp"


@dataclass
class MGInfo:
    outer_iterations: int = 0
    true_residual: float = float("nan")
    converged: bool = False
    coarse_iterations: list = field(default_factory=list)


class Multigrid:
    """Hierarchy ``levels[0..L-1]`` with transfers ``transfers[l]: l -> l+1``."""

    def __init__(self, fine: LatticeLevel, params: MGParams, null_vectors=None, setup_history=None):
        self.params = params
        self.levels = [fine]
        self.transfers = []
        for l, (blk, nv) in enumerate(zip(params.blocks, params.nv)):
            lev = self.levels[l]
            if null_vectors is not None and null_vectors[l] is not None:
                V = list(null_vectors[l])
            else:
                V = setup_null_vectors(lev, nv, params.seed, l, params.setup_iters, params.setup_inner,
                                       params.setup_rq_tol, setup_history)
            P = block_gram_schmidt(lev, blk, V)
            T = Transfer(lev, blk, P)
            self.transfers.append(T)
            self.levels.append(build_coarse(lev, T, params.coarse_op))
        self._coarse_iters = []

    def cycle(self, l: int, r):
        """Preconditioner of ``D_r`` on level ``l`` (module header)."""
        p = self.params
        lev, T = self.levels[l], self.transfers[l]
        r = r * lev.even
        z = lev.zeros()
        if p.nu_pre:
            z = mr(lev.Dr, r, p.nu_pre) * lev.even
        res = r - lev.Dr(z) if p.nu_pre else r
        ec = self.coarse_solve(l + 1, T.restrict(res))
        z = z + T.prolong(ec) * lev.even
        if p.nu_post:
            z = z + mr(lev.Dr, r - lev.Dr(z), p.nu_post) * lev.even
        return z

    def coarse_solve(self, l: int, rc):
        p = self.params
        lev = self.levels[l]
        tol = p.tol_coarse * math.sqrt(norm2(rc))
        has_next = l + 1 < len(self.levels)
        if lev.eo_ok:
            pre = (lambda r: self.cycle(l, r)) if has_next else None
            y, info = fgcr(lev.Dr, lev.b_r(rc), pre, tol_abs=tol, maxiter=p.maxit_coarse, restart=p.restart_coarse)
            self._coarse_iters.append((l, info.iterations))
            return lev.reconstruct(y, rc)
        if has_next:
            raise ValueError("only the coarsest level may lack even-odd preconditioning")
        x, info = fgcr(lev.D, rc, None, tol_abs=tol, maxiter=p.maxit_coarse, restart=p.restart_coarse)
        self._coarse_iters.append((l, info.iterations))
        return x

    def solve(self, b, tol: float = 1e-10, max_attempts: int = 5):
        """MG-preconditioned FGCR on ``D_r y_e = b_r``, then reconstruction."""
        return eo_solve(self.levels[0], b, tol, precond=lambda r: self.cycle(0, r),
                        restart=self.params.restart_fine, maxiter=self.params.maxit_fine,
                        max_attempts=max_attempts, owner=self)


def eo_solve(fine: LatticeLevel, b, tol: float = 1e-10, precond=None, restart: int = 16, maxiter: int = 5000,
             max_attempts: int = 5, owner=None):
    """Even-odd solve of ``D x = b``: FGCR on the reduced system (optionally
    preconditioned), reconstruction, true-residual check (module header)."""
    bnorm = math.sqrt(norm2(b))
    br = fine.b_r(b)
    y = None
    out = MGInfo()
    if owner is not None:
        owner._coarse_iters = []
    for _ in range(max_attempts):
        y, info = fgcr(fine.Dr, br, precond, x0=y, tol_abs=0.5 * tol * bnorm, maxiter=maxiter, restart=restart)
        out.outer_iterations += info.iterations
        x = fine.reconstruct(y, b)
        out.true_residual = math.sqrt(norm2(b - fine.D(x))) / bnorm
        if out.true_residual <= tol:
            out.converged = True
            break
    if owner is not None:
        out.coarse_iterations = list(owner._coarse_iters)
    return x, out
