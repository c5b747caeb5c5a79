"""ORACLE -- test infrastructure only.

Plain, slow, obviously-correct CPU reference for everything the CUDA library
computes.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline leg may import it; the product never does, and the two share no
code (only the seeded input generators in ``synth``).  Floating point is FP64.

Each function cites the passage of the paper it follows:

* snapping, geometry, visibility, insolation, F entries: ``vf_oracle.c``
  (Section 3, Eq. FF-def; Section 3.2 visibility; Eq. for point-sun insolation)
* ``partition``: Algorithm 2 (quadtree) and its octree analogue (Section 4.1)
* ``assemble``: Algorithms 3 and 4 (Sections 4.2, 4.3) with exact FP64 SVDs
* ``apply_blocks``: Algorithm 5 (Section 4.4)
* ``jacobi``: the Jacobi iteration for Eq. radiosity-system (Sections 3, 5.1)
* ``equilibrium_temperature``, ``equilibrium_fluxes``: the two
  time-independent systems of Section 5.1 (the second with per-facet albedo,
  emissivity and heat flux, in the printed F diag(albedo) form)
* ``flux_step``, ``flux_init``: the flux updates of Algorithm 6 (Section 5.2)
* ``disk_sun_samples``, ``insolation_disk``: the finite solar disk as a sum
  of point sources (Section 2)
* ``bowl_*``: the analytic bowl-shaped crater solution (Section 6.1)

Parity pins: see tests/test_oracle_*.py (closed forms, invariants, brute force).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lib = None

SIGMA_SB = 5.670374419e-8  # CODATA 2018; the paper gives no value


def build_oracle(force: bool = False) -> str:
    """Compile the C part of the oracle with gcc (host code, no GPU)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_oracle())
        P = ctypes.c_void_p
        I = ctypes.c_int64
        lib.or_snap.argtypes = [P, I, P, P, P]
        lib.or_snap.restype = ctypes.c_int
        lib.or_geometry.argtypes = [P, ctypes.c_double, P, I, P, P, P, P, P]
        lib.or_visibility_brute.argtypes = [P, P, I, P, P, P]
        lib.or_bvh_build.argtypes = [P, P, I, P]
        lib.or_bvh_build.restype = P
        lib.or_bvh_free.argtypes = [P]
        lib.or_visibility_rows_bvh.argtypes = [P, P, P, I, P, P, P, I, P]
        lib.or_quantize_dir.argtypes = [P, P]
        lib.or_sun_visibility.argtypes = [P, P, P, I, P, P, P, P]
        lib.or_F_rows.argtypes = [P, P, P, I, P, I, P, P]
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ------------------------------------------------------------------ mesh
@dataclass
class Mesh:
    """Snapped mesh with FP64 geometry and exact integer quantities."""
    faces: np.ndarray          # nf x 3 int32
    q: np.ndarray              # nv x 3 int64 grid coordinates
    unit: float
    base: np.ndarray           # 3 int64: grid origin = base * unit
    area: np.ndarray           # nf
    cent: np.ndarray           # nf x 3, relative to the grid origin
    nrm: np.ndarray            # nf x 3 unit normals
    c3: np.ndarray             # nf x 3 int64, 3 x centroid in grid units
    nint: np.ndarray           # nf x 3 int64, (b-a)x(c-a) in grid units
    _bvh: int | None = field(default=None, repr=False)

    @property
    def n(self) -> int:
        return self.faces.shape[0]

    def bvh(self):
        if self._bvh is None:
            self._bvh = _load().or_bvh_build(_p(self.q), _p(self.faces), self.n, _p(self.c3))
        return self._bvh

    def __del__(self):
        if self._bvh is not None and _lib is not None:
            _lib.or_bvh_free(self._bvh)
            self._bvh = None


def mesh(verts: np.ndarray, faces: np.ndarray) -> Mesh:
    """Snap the vertices to the 2^18 grid and compute A_i, x_i, n_i (Section 3)."""
    lib = _load()
    v = np.ascontiguousarray(verts, dtype=np.float64)
    f = np.ascontiguousarray(faces, dtype=np.int32)
    nv, nf = v.shape[0], f.shape[0]
    q = np.empty((nv, 3), dtype=np.int64)
    unit = np.zeros(1)
    base = np.zeros(3, dtype=np.int64)
    if lib.or_snap(_p(v), nv, _p(q), _p(unit), _p(base)) != 0:
        raise ValueError("degenerate vertex set")
    area = np.empty(nf)
    cent = np.empty((nf, 3))
    nrm = np.empty((nf, 3))
    c3 = np.empty((nf, 3), dtype=np.int64)
    nint = np.empty((nf, 3), dtype=np.int64)
    lib.or_geometry(_p(q), float(unit[0]), _p(f), nf, _p(area), _p(cent), _p(nrm), _p(c3), _p(nint))
    return Mesh(f, q, float(unit[0]), base, area, cent, nrm, c3, nint)


def visibility_brute(m: Mesh) -> np.ndarray:
    """V (N x N, uint8) by brute force over all occluders, O(N^3) (Section 3.2)."""
    V = np.empty((m.n, m.n), dtype=np.uint8)
    _load().or_visibility_brute(_p(m.q), _p(m.faces), m.n, _p(m.c3), _p(m.nint), _p(V))
    return V


def visibility_rows(m: Mesh, rows) -> np.ndarray:
    """Rows of V through the oracle's own BVH (same decisions as brute force)."""
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    V = np.empty((rows.size, m.n), dtype=np.uint8)
    _load().or_visibility_rows_bvh(m.bvh(), _p(m.q), _p(m.faces), m.n, _p(m.c3), _p(m.nint),
                                   _p(rows), rows.size, _p(V))
    return V


def quantize_dir(s) -> np.ndarray:
    s = np.ascontiguousarray(s, dtype=np.float64)
    out = np.empty(3, dtype=np.int64)
    _load().or_quantize_dir(_p(s), _p(out))
    return out


def sun_visibility(m: Mesh, s, brute: bool = False) -> np.ndarray:
    """V_sun per facet for one direction s (Eq. visibility-function)."""
    s = np.ascontiguousarray(s, dtype=np.float64)
    vis = np.empty(m.n, dtype=np.uint8)
    _load().or_sun_visibility(None if brute else m.bvh(), _p(m.q), _p(m.faces), m.n, _p(m.c3),
                              _p(m.nint), _p(s), _p(vis))
    return vis


def insolation(m: Mesh, dirs, solar_flux: float, brute: bool = False) -> np.ndarray:
    """E (N x R): E_i = S max(0, n_i . s) V_sun(i, s), sun at 1 AU
    (Eq. insolation-for-point-sun; sin of the elevation above the facet's
    tangent plane is n_i . s)."""
    dirs = np.atleast_2d(np.asarray(dirs, dtype=np.float64))
    E = np.zeros((m.n, dirs.shape[0]))
    for r, s in enumerate(dirs):
        vis = sun_visibility(m, s, brute=brute)
        E[:, r] = solar_flux * np.maximum(0.0, m.nrm @ s) * vis
    return E


def F_rows(m: Mesh, rows, Vrows: np.ndarray | None = None) -> np.ndarray:
    """Rows of F per Eq. FF-def (FP64); V from the BVH unless given."""
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    if Vrows is None:
        Vrows = visibility_rows(m, rows)
    Vrows = np.ascontiguousarray(Vrows, dtype=np.uint8)
    Fr = np.empty((rows.size, m.n))
    _load().or_F_rows(_p(m.area), _p(m.cent), _p(m.nrm), m.n, _p(rows), rows.size, _p(Vrows), _p(Fr))
    return Fr


def F_dense(m: Mesh, V: np.ndarray | None = None) -> np.ndarray:
    """The full N x N view-factor matrix (Eq. FF-def)."""
    if V is None:
        V = visibility_brute(m)
    return F_rows(m, np.arange(m.n), V)


# ------------------------------------------------------------- partition
@dataclass
class Tree:
    perm: np.ndarray           # tree position -> facet index
    first: np.ndarray          # per node (preorder ids)
    count: np.ndarray
    depth: np.ndarray
    parent: np.ndarray
    children: list             # per node: list of child ids (ascending child index)
    child_slot: np.ndarray     # per node: its child index within the parent (0..3 / 0..7)

    def is_leaf(self, k: int) -> bool:
        return len(self.children[k]) == 0


def partition(m: Mesh, kind: str = "quad", leaf_size: int = 64, max_depth: int = 32) -> Tree:
    """Algorithm 2 (quadtree on centroids) and the octree analogue (Section 4.1).

    Readings: each node splits at the midpoint of ITS OWN centroids' bounding
    box (the printed comparison against x_min/y_min is taken as x_mid/y_mid);
    a centroid on the midpoint goes to the upper child; children in the
    printed order I1 (x<,y<), I2 (x<,y>=), I3 (x>=,y<), I4 (x>=,y>=), i.e.
    child index 2[x>=]+[y>=] (octree: 4[x>=]+2[y>=]+[z>=]); empty children
    dropped; members keep their parent's order.  Recursion stops at
    count <= leaf_size, depth == max_depth, or a bounding box of zero extent.
    Comparisons are exact on the integer 3 x centroid: 2c >= lo + hi.
    """
    axes = 2 if kind == "quad" else 3
    c = m.c3[:, :axes]
    firsts, counts, depths, parents, children, slots = [], [], [], [], [], []
    perm_parts = []

    def rec(idx: np.ndarray, depth: int, parent: int, slot: int, offset: int) -> int:
        nid = len(firsts)
        firsts.append(offset)
        counts.append(idx.size)
        depths.append(depth)
        parents.append(parent)
        children.append([])
        slots.append(slot)
        if idx.size <= leaf_size or depth >= max_depth:
            perm_parts.append(idx)
            return nid
        cc = c[idx]
        lo = cc.min(axis=0)
        hi = cc.max(axis=0)
        if np.all(lo == hi):
            perm_parts.append(idx)
            return nid
        code = np.zeros(idx.size, dtype=np.int64)
        for a in range(axes):
            code = code * 2 + (2 * cc[:, a] >= lo[a] + hi[a]).astype(np.int64)
        off = offset
        for ch in range(1 << axes):
            sub = idx[code == ch]
            if sub.size == 0:
                continue
            kid = rec(sub, depth + 1, nid, ch, off)
            children[nid].append(kid)
            off += sub.size
        return nid

    rec(np.arange(m.n, dtype=np.int64), 0, -1, 0, 0)
    perm = np.concatenate(perm_parts) if perm_parts else np.zeros(0, dtype=np.int64)
    return Tree(perm.astype(np.int64), np.array(firsts), np.array(counts), np.array(depths),
                np.array(parents), children, np.array(slots))


# -------------------------------------------------------------- assembly
ZERO, DENSE, CSR, SVD, HIER = 0, 1, 2, 3, 4
TYPE_NAMES = {ZERO: "zero", DENSE: "dense", CSR: "csr", SVD: "svd", HIER: "hier"}


@dataclass
class Block:
    I: int                     # row node
    J: int                     # column node
    kind: int
    nbytes: int
    q: int = 0
    children: list = field(default_factory=list)
    U: np.ndarray | None = None   # compacted rows x q, Sigma folded in
    V: np.ndarray | None = None   # compacted cols x q
    rows_nz: np.ndarray | None = None
    cols_nz: np.ndarray | None = None
    sv: np.ndarray | None = None  # singular values of the block (probe)
    nnz: int = 0                  # nonzero entries of the block
    hier_bytes: int = -1          # bytes of the hierarchical candidate (non-leaf blocks), else -1


def nbytes_dense(m: int, n: int) -> int:
    return 4 * m * n


def nbytes_csr(m: int, nnz: int) -> int:
    return 8 * nnz + 4 * (m + 1)


def nbytes_svd(q: int, m1: int, n1: int) -> int:
    return 4 * q * (m1 + n1) + 4 * (m1 + n1)


def numerical_rank(sv: np.ndarray, tol: float) -> int:
    """Algorithm 3: smallest q >= 1 with sigma_{q+1} / sigma_1 < tol
    (sigma beyond the block's size count as zero)."""
    s1 = sv[0]
    for q in range(1, sv.size + 1):
        nxt = sv[q] if q < sv.size else 0.0
        if nxt < tol * s1:
            return q
    return sv.size


def assemble(Ft: np.ndarray, tree: Tree, tol: float, leaf_threshold: int = 4096,
             k_max: int = 128, keep_factors: bool = True):
    """Algorithms 3 and 4 on the dense FP64 matrix Ft = F[perm][:, perm].

    Readings (the paper leaves these open):
      * a leaf block is a pair of tree leaves, or |I||J| < leaf_threshold; it
        is stored dense or CSR, whichever is smaller (Alg. 4 step 2);
      * otherwise the candidates are dense, CSR, the q-truncated SVD
        (Alg. 3; q = smallest with sigma_{q+1} < tol sigma_1, the probe fails
        if q > k_max) and the hierarchical block over child pairs (a tree leaf
        stands for itself when the other side has children) (Alg. 4 steps 3-5);
      * bytes: dense 4mn, CSR 8 nnz + 4(m+1), SVD 4q(m'+n') + 4(m'+n') with
        m', n' the nonzero rows/columns; a block with no nonzero is a zero
        block of 0 bytes; ties go zero < dense < CSR < SVD < hierarchical;
      * Alg. 4 step 6: a hierarchical block whose nonzero children are all
        CSR (all dense) is coalesced into one CSR (dense) block;
      * assembly starts at the pairs of the root's children (end of 4.3).
    Returns the list of top-level Blocks (a tree of Blocks).
    """
    perm_first = tree.first
    cnt = tree.count

    def kids(X):
        return tree.children[X] if not tree.is_leaf(X) else [X]

    def rng(X):
        return slice(perm_first[X], perm_first[X] + cnt[X])

    def build(I: int, J: int) -> Block:
        A = Ft[rng(I), rng(J)]
        m, n = A.shape
        nzmask = A != 0
        nnz = int(nzmask.sum())
        if nnz == 0:
            return Block(I, J, ZERO, 0)
        rows_nz = np.nonzero(nzmask.any(axis=1))[0]
        cols_nz = np.nonzero(nzmask.any(axis=0))[0]
        cand = [(nbytes_dense(m, n), DENSE), (nbytes_csr(m, nnz), CSR)]
        leaf_block = (tree.is_leaf(I) and tree.is_leaf(J)) or m * n < leaf_threshold
        if leaf_block:
            b, kd = min(cand, key=lambda t: (t[0], t[1]))
            return Block(I, J, kd, b, nnz=nnz)
        ch = [build(a, b) for a in kids(I) for b in kids(J)]
        hb = sum(c.nbytes for c in ch)
        Ac = A[np.ix_(rows_nz, cols_nz)]
        if keep_factors:
            Uf, sv, Vt = np.linalg.svd(Ac, full_matrices=False)
        else:
            sv = np.linalg.svd(Ac, compute_uv=False)
        q = numerical_rank(sv, tol)
        svd_ok = q <= k_max
        if svd_ok:
            cand.append((nbytes_svd(q, rows_nz.size, cols_nz.size), SVD))
        cand.append((hb, HIER))
        b, kd = min(cand, key=lambda t: (t[0], t[1]))
        if kd == HIER:
            nzk = [c.kind for c in ch if c.kind != ZERO]
            if nzk and all(k == CSR for k in nzk):
                return Block(I, J, CSR, nbytes_csr(m, nnz), sv=sv, nnz=nnz, hier_bytes=hb)
            if nzk and all(k == DENSE for k in nzk):
                return Block(I, J, DENSE, nbytes_dense(m, n), sv=sv, nnz=nnz, hier_bytes=hb)
            return Block(I, J, HIER, hb, children=ch, sv=sv, nnz=nnz, hier_bytes=hb)
        if kd == SVD:
            blk = Block(I, J, SVD, b, q=q, rows_nz=rows_nz, cols_nz=cols_nz, sv=sv, nnz=nnz, hier_bytes=hb)
            if keep_factors:
                blk.U = Uf[:, :q] * sv[:q]
                blk.V = Vt[:q, :].T.copy()
            return blk
        return Block(I, J, kd, b, sv=sv, nnz=nnz, hier_bytes=hb)

    root = 0
    if tree.is_leaf(root):
        return [build(root, root)]
    return [build(I, J) for I in tree.children[root] for J in tree.children[root]]


def leaf_blocks(top) -> list:
    """Flatten a block tree to its stored (non-hierarchical) blocks."""
    out = []
    stack = list(reversed(top))
    while stack:
        b = stack.pop()
        if b.kind == HIER:
            stack.extend(reversed(b.children))
        else:
            out.append(b)
    return out


def apply_blocks(top, tree: Tree, Ft: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Algorithm 5: Y = F_hat X in tree order; dense and CSR blocks are the
    exact entries of Ft, SVD blocks their stored factors."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.zeros((tree.perm.size,) + X.shape[1:])
    for b in leaf_blocks(top):
        r0, m = tree.first[b.I], tree.count[b.I]
        c0, n = tree.first[b.J], tree.count[b.J]
        if b.kind in (DENSE, CSR):
            Y[r0:r0 + m] += Ft[r0:r0 + m, c0:c0 + n] @ X[c0:c0 + n]
        elif b.kind == SVD:
            Y[r0 + b.rows_nz] += b.U @ (b.V.T @ X[c0 + b.cols_nz])
    return Y


# ----------------------------------------------------------------- solve
def jacobi(apply, E: np.ndarray, rho, rtol: float = 1e-12, max_iter: int = 200):
    """Jacobi iteration for B = E + diag(rho) F B (Eq. radiosity-system;
    Section 3 and 5.1).  F_ii = 0, so Jacobi is the fixed point
    B_{k+1} = E + rho * (F B_k), started from B_0 = E.  A column stops once
    ||B_{k+1} - B_k||_2 <= rtol ||E||_2 and returns B_{k+1}; a column with
    E = 0 returns 0.  ``apply`` maps an N x R array to F times it.
    Returns (B, sweeps per column, final relative residual per column)."""
    E = np.asarray(E, dtype=np.float64)
    squeeze = E.ndim == 1
    if squeeze:
        E = E[:, None]
    rho = np.broadcast_to(np.asarray(rho, dtype=np.float64), (E.shape[0],))[:, None]
    R = E.shape[1]
    B = E.copy()
    enorm = np.linalg.norm(E, axis=0)
    done = enorm == 0
    B[:, done] = 0.0
    iters = np.zeros(R, dtype=np.int64)
    res = np.zeros(R)
    active = ~done
    for _ in range(max_iter):
        if not active.any():
            break
        idx = np.nonzero(active)[0]
        Bn = E[:, idx] + rho * apply(B[:, idx])
        r = np.linalg.norm(Bn - B[:, idx], axis=0) / enorm[idx]
        B[:, idx] = Bn
        iters[idx] += 1
        res[idx] = r
        active[idx[r <= rtol]] = False
    return (B[:, 0] if squeeze else B), iters, res


# --------------------------------------------------------- closed forms
def bowl_f(depth_ratio: float) -> float:
    """1/f = 1 + (D/d)^2 / 4 (Section 6.1)."""
    Dd = 1.0 / depth_ratio
    return 1.0 / (1.0 + 0.25 * Dd * Dd)


def bowl_b(f: float, albedo: float, emissivity: float) -> float:
    """b = f (eps + alpha (1 - f)) / (1 - alpha f) (Section 6.1)."""
    return f * (emissivity + albedo * (1.0 - f)) / (1.0 - albedo * f)


def bowl_shadow_temperature(S: float, elev_deg: float, albedo: float, emissivity: float,
                            depth_ratio: float) -> float:
    """Equilibrium temperature in the shadowed part of a bowl crater
    (Eq. globalsolution, shadowed case)."""
    f = bowl_f(depth_ratio)
    b = bowl_b(f, albedo, emissivity)
    q = (1.0 - albedo) * S * b * math.sin(math.radians(elev_deg))
    return (q / (emissivity * SIGMA_SB)) ** 0.25


def equilibrium_temperature(apply, Edirect: np.ndarray, albedo: float, emissivity: float,
                            rtol: float = 1e-12, max_iter: int = 500):
    """Section 5.1: Q_vis = B from B = Q_direct + albedo F B; then
    (I - F) Q_IR = F (1 - albedo) Q_vis; finally
    eps sigma T^4 = (1 - albedo) Q_vis + eps Q_IR (Eq. 3d-equilbr, H = 0)."""
    Qvis, _, _ = jacobi(apply, Edirect, albedo, rtol, max_iter)
    rhs = apply((1.0 - albedo) * Qvis)
    Qir, _, _ = jacobi(apply, rhs, 1.0, rtol, max_iter)
    absorbed = (1.0 - albedo) * Qvis + emissivity * Qir
    T = np.maximum(absorbed, 0.0) / (emissivity * SIGMA_SB)
    return T ** 0.25, Qvis, Qir


def _fixed_point(step, x0, scale, rtol, max_iter):
    """x <- step(x) from x0 until ||x_{k+1} - x_k||_2 <= rtol ||scale||_2 per column."""
    x = x0
    ref = np.linalg.norm(scale, axis=0)
    for _ in range(max_iter):
        xn = step(x)
        done = np.all(np.linalg.norm(xn - x, axis=0) <= rtol * np.maximum(ref, 1e-300))
        x = xn
        if done:
            break
    return x


def equilibrium_fluxes(apply, Edirect: np.ndarray, albedo, emissivity, H=0.0, rtol: float = 1e-13,
                       max_iter: int = 2000):
    """Section 5.1 as printed, with per-facet albedo and emissivity (N x 1
    columns or scalars) and interior heat flux H:
      (I - F diag(albedo)) Q_refl = F diag(albedo) Q_direct      (Eq. time-indep-system-1)
      (I - F) Q_IR = F (I - diag(albedo)) (Q_direct + Q_refl) + F H  (Eq. time-indep-system-2)
      eps sigma T^4 = (1 - albedo)(Q_direct + Q_refl) + eps Q_IR   (Eq. 3d-equilbr)
    each system by its fixed-point (Jacobi) iteration from 0.  Returns
    (T, Q_refl, Q_IR)."""
    a = np.asarray(albedo, dtype=np.float64)
    e = np.asarray(emissivity, dtype=np.float64)
    Ed = np.asarray(Edirect, dtype=np.float64)
    b1 = apply(a * Ed)
    Qrefl = _fixed_point(lambda x: b1 + apply(a * x), np.zeros_like(Ed), b1, rtol, max_iter)
    b2 = apply((1.0 - a) * (Ed + Qrefl) + H)
    Qir = _fixed_point(lambda x: b2 + apply(x), np.zeros_like(Ed), b2, rtol, max_iter)
    absorbed = (1.0 - a) * (Ed + Qrefl) + e * Qir
    T = (np.maximum(absorbed, 0.0) / (e * SIGMA_SB)) ** 0.25
    return T, Qrefl, Qir


# ------------------------------------------------------- Algorithm 6
def flux_init(Edirect: np.ndarray, albedo, H=0.0):
    """Algorithm 6, n = 0: Q_abs = (1 - albedo) Q_direct + H, Q_refl = 0,
    Q_IR = 0, Q_rad = Q_abs.  Returns (Q_refl, Q_IR, Q_abs, Q_rad)."""
    Ed = np.asarray(Edirect, dtype=np.float64)
    Qabs = (1.0 - np.asarray(albedo, dtype=np.float64)) * Ed + H
    return np.zeros_like(Ed), np.zeros_like(Ed), Qabs, Qabs.copy()


def flux_step(apply, Edirect_next, Qrefl, Qir, Qrad, albedo, emissivity):
    """Algorithm 6 (Section 5.2), one time step of the fluxes, one multiply
    by F per flux:
      Q_refl' = F diag(albedo) (Q_direct' + Q_refl)
      Q_IR'   = F (Q_rad + (I - diag(emissivity)) Q_IR)
      Q_abs'  = (I - diag(albedo)) (Q_direct' + Q_refl') + diag(emissivity) Q_IR'
    albedo, emissivity: scalars or per-facet columns (N x 1).  Returns
    (Q_refl', Q_IR', Q_abs')."""
    a = np.asarray(albedo, dtype=np.float64)
    e = np.asarray(emissivity, dtype=np.float64)
    Ed = np.asarray(Edirect_next, dtype=np.float64)
    Qrefl1 = apply(a * (Ed + Qrefl))
    Qir1 = apply(Qrad + (1.0 - e) * Qir)
    Qabs1 = (1.0 - a) * (Ed + Qrefl1) + e * Qir1
    return Qrefl1, Qir1, Qabs1


# ------------------------------------------------------- finite solar disk
def disk_sun_samples(s, angular_radius: float, rings: int):
    """Point sources standing for a uniformly bright solar disk of the given
    angular radius (radians) around the unit direction s (Section 2: the
    disk's flux is a sum over point sources).  The disk is cut into rings of
    equal radial width; ring k (k = 0 is the central disk) is split into
    max(1, 6k) equal sectors; each cell's point sits at its area-weighted
    mean radius and mid angle, with weight = its share of the disk's area
    (the weights sum to 1).  Returns (directions M x 3, weights M)."""
    s = np.asarray(s, dtype=np.float64)
    s = s / np.linalg.norm(s)
    a = np.array([1.0, 0.0, 0.0]) if abs(s[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    u = np.cross(s, a)
    u /= np.linalg.norm(u)
    w = np.cross(s, u)
    dirs, wts = [], []
    for k in range(rings):
        r0, r1 = k / rings, (k + 1) / rings
        nsec = max(1, 6 * k)
        area = (r1 * r1 - r0 * r0) / nsec  # share of the unit disk (pi cancels)
        rc = 0.0 if k == 0 else (2.0 / 3.0) * (r1 ** 3 - r0 ** 3) / (r1 * r1 - r0 * r0)
        for j in range(nsec):
            phi = 2.0 * math.pi * (j + 0.5) / nsec
            t = angular_radius * rc
            d = math.cos(t) * s + math.sin(t) * (math.cos(phi) * u + math.sin(phi) * w)
            dirs.append(d / np.linalg.norm(d))
            wts.append(area)
    return np.asarray(dirs), np.asarray(wts)


def insolation_disk(m: Mesh, dirs, solar_flux: float, angular_radius: float, rings: int) -> np.ndarray:
    """E (N x R) for a finite solar disk: the weighted sum over the disk's
    point sources of the point-sun insolation (Section 2), per sun direction."""
    dirs = np.atleast_2d(np.asarray(dirs, dtype=np.float64))
    E = np.zeros((m.n, dirs.shape[0]))
    for r, s in enumerate(dirs):
        pts, wts = disk_sun_samples(s, angular_radius, rings)
        E[:, r] = insolation(m, pts, solar_flux) @ wts
    return E
