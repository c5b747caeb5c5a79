"""Thin Python binding of libvf's C ABI (include/vf.h).

Argument marshalling only: every step runs in the library's CUDA kernels.
Device buffers are torch CUDA tensors (float32, contiguous); an N x R
column-major block with leading dimension N is a torch tensor of shape
(R, N).  Importing this module loads the shared library and raises
VFError if it has not been built -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libvf.so")

VF_OK, VF_E_INVAL, VF_E_NOMEM, VF_E_CUDA, VF_E_NOCONV, VF_E_TIMEOUT, VF_E_OOB, VF_E_IO, VF_E_CORRUPT = range(9)
# static scratch of vf_apply_tree_static (include/vf.h)
VF_STATIC_T_FLOATS = 4194304
VF_STATIC_PART_FLOATS = 262144
PREC = {"fp32": 0, "bf16": 1, "fp8": 2}
KIND_NAMES = {0: "zero", 1: "dense", 2: "csr", 3: "svd", 4: "hier"}


class VFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libvf status {status}: {msg}")
        self.status = status


# ------------------------------------------------------------------ structs
class MeshOpts(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32)]


class PartitionOpts(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("leaf_size", ctypes.c_int32), ("max_depth", ctypes.c_int32)]


class AssembleOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("leaf_threshold", ctypes.c_int64), ("k0", ctypes.c_int32),
                ("k_max", ctypes.c_int32), ("power_iters", ctypes.c_int32), ("verify", ctypes.c_int32),
                ("precisions", ctypes.c_uint32), ("predictor", ctypes.c_void_p), ("seed", ctypes.c_uint64),
                ("storage", ctypes.c_int32)]


class AssembleStats(ctypes.Structure):
    _fields_ = [("nblocks", ctypes.c_int64 * 5), ("bytes", ctypes.c_int64 * 5), ("nnz_visible", ctypes.c_int64),
                ("probes", ctypes.c_int64), ("probes_failed", ctypes.c_int64), ("probes_skipped", ctypes.c_int64),
                ("probes_predicted_skip", ctypes.c_int64), ("verify_failed", ctypes.c_int64),
                ("predictor_audits", ctypes.c_int64), ("predictor_audit_wins", ctypes.c_int64),
                ("predictor_fallbacks", ctypes.c_int64),
                ("max_rank", ctypes.c_int32), ("t_visibility", ctypes.c_double), ("t_stats", ctypes.c_double),
                ("t_probe", ctypes.c_double), ("t_pack", ctypes.c_double), ("t_total", ctypes.c_double)]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["nblocks"] = {KIND_NAMES[k]: int(self.nblocks[k]) for k in range(5)}
        d["bytes"] = {KIND_NAMES[k]: int(self.bytes[k]) for k in range(5)}
        return d


class SolveOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("refine", ctypes.c_int32), ("max_refine", ctypes.c_int32), ("inner_rtol", ctypes.c_double),
                ("clamp", ctypes.c_int32), ("rho", ctypes.c_float)]


class SolveStats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int32), ("refinements", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("kernels", ctypes.c_int32), ("max_rel_residual", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


# ------------------------------------------------------------------ loading
_lib = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_SIGS = {
    "vf_last_error": ([], ctypes.c_char_p),
    "vf_version": ([], ctypes.c_char_p),
    "vf_debug_fail_alloc": ([_I64], ctypes.c_int),
    "vf_set_wait_limit": ([_I32, _I64], ctypes.c_int),
    "vf_mesh_create": ([_P, _I64, _P, _I64, _P, _P], ctypes.c_int),
    "vf_mesh_destroy": ([_P], None),
    "vf_mesh_nfacets": ([_P], _I64),
    "vf_mesh_grid": ([_P, _P, _P], ctypes.c_int),
    "vf_mesh_geometry": ([_P, _P, _P, _P], ctypes.c_int),
    "vf_mesh_visibility": ([_P, _P, _I64, _P], ctypes.c_int),
    "vf_mesh_insolation": ([_P, _P, _I32, ctypes.c_double, _P, _I64, _P], ctypes.c_int),
    "vf_mesh_insolation_disk": ([_P, _P, _I32, ctypes.c_double, ctypes.c_double, _I32, _P, _I64, _P], ctypes.c_int),
    "vf_equilibrium": ([_P, _P, _I64, _I32, _P, _P, _P, _P, _P, _P, _P, _I64, _P, _P], ctypes.c_int),
    "vf_flux_step": ([_P, ctypes.c_int, _I32, _P, _P, ctypes.c_float, ctypes.c_float, _P, _P, _P, _P, _P, _I64, _P],
                     ctypes.c_int),
    "vf_partition": ([_P, _P, _P], ctypes.c_int),
    "vf_tree_destroy": ([_P], None),
    "vf_tree_nnodes": ([_P], _I64),
    "vf_tree_perm": ([_P, _P], ctypes.c_int),
    "vf_tree_nodes": ([_P, _P, _P, _P, _P], ctypes.c_int),
    "vf_assemble": ([_P, _P, _P, _P, _P], ctypes.c_int),
    "vf_hmat_destroy": ([_P], None),
    "vf_hmat_probe_log": ([_P, _P, _P, _P], ctypes.c_int),
    "vf_predictor_create": ([_I32, ctypes.c_uint64, _P], ctypes.c_int),
    "vf_predictor_destroy": ([_P], None),
    "vf_predictor_params": ([_P, _P, _P], ctypes.c_int),
    "vf_predictor_grad": ([_P, _P, _P, _I64, _P, _P], ctypes.c_int),
    "vf_predictor_train": ([_P, _P, _P, _I64, _I32, _I32, ctypes.c_float, _P], ctypes.c_int),
    "vf_predictor_predict": ([_P, _P, _I64, _P, _P], ctypes.c_int),
    "vf_hmat_nfacets": ([_P], _I64),
    "vf_hmat_blocks": ([_P, _P, _P], ctypes.c_int),
    "vf_hmat_bytes": ([_P, ctypes.c_int], _I64),
    "vf_apply": ([_P, ctypes.c_int, _P, _I64, _I32, _P, _I64, _P], ctypes.c_int),
    "vf_apply_tree": ([_P, ctypes.c_int, _P, _I32, _P, _P], ctypes.c_int),
    "vf_apply_tree_static": ([_P, ctypes.c_int, _P, _I32, _P, _P], ctypes.c_int),
    "vf_solve": ([_P, _P, _P, _I64, _P, _I64, _I32, _P, _P, _P], ctypes.c_int),
    "vf_solve_host": ([_P, _P, _P, _I64, _P, _I64, _I32, _P, _P, _P], ctypes.c_int),
    "vf_solve_batched": ([_P, _I32, _P, _P, _P, _P, _P, _P, _P, _P, _P], ctypes.c_int),
    "vf_autotune": ([_P, ctypes.c_int, _I32, _P, _P], ctypes.c_int),
    "vf_tune_set": ([_P, ctypes.c_int, _I32, _P], ctypes.c_int),
    "vf_hmat_stack": ([_P, _I32, _P], ctypes.c_int),
    "vf_hmat_nsegments": ([_P], _I32),
    "vf_hmat_trim": ([_P], ctypes.c_int),
    "vf_hmat_tensor_bytes": ([_P, _I32, _P, _P], ctypes.c_int),
    "vf_hmat_save": ([_P, ctypes.c_char_p], ctypes.c_int),
    "vf_hmat_load": ([ctypes.c_char_p, _I32, _P], ctypes.c_int),
}


def load(path: str = LIB_PATH):
    """Load libvf; raise VFError (never fall back) if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise VFError(-1, f"libvf is not built ({path} missing); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (args, res) in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def declared_symbols() -> list[str]:
    return list(_SIGS)


def _check(status: int, allow=()):
    if status != VF_OK and status not in allow:
        raise VFError(status, load().vf_last_error().decode(errors="replace"))
    return status


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _dev_ptr(t, name: str, n_rows: int | None = None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise VFError(VF_E_INVAL, f"{name}: need a contiguous float32 CUDA tensor")
    if n_rows is not None and t.shape[-1] != n_rows:
        raise VFError(VF_E_INVAL, f"{name}: last dimension {t.shape[-1]} != N = {n_rows}")
    return ctypes.c_void_p(t.data_ptr())


# ------------------------------------------------------------------ handles
class _Handle:
    _destroy = ""

    def __init__(self, ptr):
        self.ptr = ptr

    def close(self):
        if self.ptr:
            getattr(load(), self._destroy)(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mesh(_Handle):
    _destroy = "vf_mesh_destroy"

    @property
    def n(self) -> int:
        return int(load().vf_mesh_nfacets(self.ptr))


class Tree(_Handle):
    _destroy = "vf_tree_destroy"


class HMat(_Handle):
    _destroy = "vf_hmat_destroy"

    @property
    def n(self) -> int:
        return int(load().vf_hmat_nfacets(self.ptr))


class Predictor(_Handle):
    _destroy = "vf_predictor_destroy"


# rank predictor sizes (include/vf.h)
VF_PRED_NFEAT = 10
VF_PRED_NCLASS = 6
VF_PRED_NPARAM = 5254


# ------------------------------------------------------------------ API
def vf_version() -> str:
    return load().vf_version().decode()


def vf_debug_fail_alloc(nth: int):
    """Make the library's nth device allocation from now on fail (0 disarms)."""
    _check(load().vf_debug_fail_alloc(int(nth)))


def vf_set_wait_limit(polls: int, device: int = 0):
    """Polls of the CUDA-core multiply's bounded page waits (< 0: the default)."""
    _check(load().vf_set_wait_limit(int(device), int(polls)))


def vf_mesh_create(verts, faces, device: int = 0) -> Mesh:
    v = np.ascontiguousarray(verts, dtype=np.float64)
    f = np.ascontiguousarray(faces, dtype=np.int32)
    out = ctypes.c_void_p()
    opts = MeshOpts(device)
    _check(load().vf_mesh_create(_np_ptr(v), v.shape[0], _np_ptr(f), f.shape[0], ctypes.byref(opts),
                                 ctypes.byref(out)))
    return Mesh(out)


def vf_mesh_grid(m: Mesh):
    unit = ctypes.c_double()
    base = np.zeros(3, dtype=np.int64)
    _check(load().vf_mesh_grid(m.ptr, ctypes.byref(unit), _np_ptr(base)))
    return unit.value, base


def vf_mesh_geometry(m: Mesh):
    n = m.n
    area = np.empty(n)
    cent = np.empty((n, 3))
    nrm = np.empty((n, 3))
    _check(load().vf_mesh_geometry(m.ptr, _np_ptr(area), _np_ptr(cent), _np_ptr(nrm)))
    return area, cent, nrm


def vf_mesh_visibility(m: Mesh, rows=None) -> np.ndarray:
    n = m.n
    if rows is None:
        V = np.empty((n, n), dtype=np.uint8)
        _check(load().vf_mesh_visibility(m.ptr, None, n, _np_ptr(V)))
        return V
    r = np.ascontiguousarray(rows, dtype=np.int64)
    V = np.empty((r.size, n), dtype=np.uint8)
    _check(load().vf_mesh_visibility(m.ptr, _np_ptr(r), r.size, _np_ptr(V)))
    return V


def vf_mesh_insolation(m: Mesh, sun_dirs, solar_flux: float, E, stream=None):
    d = np.ascontiguousarray(np.atleast_2d(sun_dirs), dtype=np.float64)
    R = d.shape[0]
    n = m.n
    if E.shape != (R, n):
        raise VFError(VF_E_INVAL, f"E must have shape (R, N) = {(R, n)}")
    _check(load().vf_mesh_insolation(m.ptr, _np_ptr(d), R, float(solar_flux), _dev_ptr(E, "E", n), n,
                                     _stream(stream)))
    return E


def vf_mesh_insolation_disk(m: Mesh, sun_dirs, solar_flux: float, angular_radius: float, rings: int, E,
                            stream=None):
    """E (R, N) for a finite solar disk of the given angular radius (radians) around each direction."""
    d = np.ascontiguousarray(np.atleast_2d(sun_dirs), dtype=np.float64)
    R = d.shape[0]
    n = m.n
    if E.shape != (R, n):
        raise VFError(VF_E_INVAL, f"E must have shape (R, N) = {(R, n)}")
    _check(load().vf_mesh_insolation_disk(m.ptr, _np_ptr(d), R, float(solar_flux), float(angular_radius),
                                          int(rings), _dev_ptr(E, "E", n), n, _stream(stream)))
    return E


def vf_partition(m: Mesh, kind: str = "quad", leaf_size: int = 64, max_depth: int = 32) -> Tree:
    opts = PartitionOpts(0 if kind == "quad" else 1, leaf_size, max_depth)
    out = ctypes.c_void_p()
    _check(load().vf_partition(m.ptr, ctypes.byref(opts), ctypes.byref(out)))
    t = Tree(out)
    t.n = m.n
    return t


def vf_tree_perm(t: Tree) -> np.ndarray:
    perm = np.empty(t.n, dtype=np.int32)
    _check(load().vf_tree_perm(t.ptr, _np_ptr(perm)))
    return perm


def vf_tree_nodes(t: Tree) -> dict:
    k = int(load().vf_tree_nnodes(t.ptr))
    arrs = {name: np.empty(k, dtype=np.int32) for name in ("first", "count", "depth", "parent")}
    _check(load().vf_tree_nodes(t.ptr, *(_np_ptr(arrs[n]) for n in ("first", "count", "depth", "parent"))))
    return arrs


STORAGE = {"compressed": 0, "dense": 1, "csr": 2}


def vf_assemble(m: Mesh, t: Tree, tol: float = 1e-3, leaf_threshold: int = 4096, k0: int = 8, k_max: int = 128,
                power_iters: int = 2, verify: bool = True, precisions=("fp32", "bf16"), predictor=None,
                seed: int = 12345, storage: str = "compressed"):
    bits = 0
    for p in precisions:
        bits |= 1 << PREC[p]
    opts = AssembleOpts(tol, leaf_threshold, k0, k_max, power_iters, int(verify), bits,
                        predictor.ptr if predictor is not None else None, seed, STORAGE[storage])
    st = AssembleStats()
    out = ctypes.c_void_p()
    _check(load().vf_assemble(m.ptr, t.ptr, ctypes.byref(opts), ctypes.byref(out), ctypes.byref(st)))
    return HMat(out), st.as_dict()


def vf_hmat_blocks(h: HMat) -> np.ndarray:
    """Stored blocks: rows of (row node, col node, kind, q, m', n', 0)."""
    nb = ctypes.c_int64()
    _check(load().vf_hmat_blocks(h.ptr, ctypes.byref(nb), None))
    desc = np.empty((nb.value, 7), dtype=np.int32)
    _check(load().vf_hmat_blocks(h.ptr, ctypes.byref(nb), _np_ptr(desc)))
    return desc


def vf_hmat_bytes(h: HMat, precision: str = "fp32") -> int:
    return int(load().vf_hmat_bytes(h.ptr, PREC[precision]))


def vf_apply(h: HMat, X, Y, precision: str = "fp32", stream=None):
    n = h.n
    R = 1 if X.dim() == 1 else X.shape[0]
    if Y.shape != X.shape:
        raise VFError(VF_E_INVAL, "X and Y shapes differ")
    _check(load().vf_apply(h.ptr, PREC[precision], _dev_ptr(X, "X", n), n, R, _dev_ptr(Y, "Y", n), n,
                           _stream(stream)))
    return Y


def _same_shape(Xt, Yt, who: str):
    """Yt receives R x N floats: its shape must be Xt's (checked before the library is called)."""
    if tuple(Yt.shape) != tuple(Xt.shape):
        raise VFError(VF_E_INVAL, f"{who}: Yt shape {tuple(Yt.shape)} != Xt shape {tuple(Xt.shape)}")


def vf_apply_tree(h: HMat, Xt, Yt, precision: str = "fp32", stream=None):
    """The multiply alone on tree-ordered (R, N) tensors."""
    _same_shape(Xt, Yt, "vf_apply_tree")
    n = h.n
    R = 1 if Xt.dim() == 1 else Xt.shape[0]
    _check(load().vf_apply_tree(h.ptr, PREC[precision], _dev_ptr(Xt, "Xt", n), R, _dev_ptr(Yt, "Yt", n),
                                _stream(stream)))
    return Yt


def vf_apply_tree_static(h: HMat, Xt, Yt, precision: str = "fp32", stream=None):
    """vf_apply_tree with the library's fixed static scratch: no device
    allocation; synchronous; calls must not overlap in time."""
    _same_shape(Xt, Yt, "vf_apply_tree_static")
    n = h.n
    R = 1 if Xt.dim() == 1 else Xt.shape[0]
    _check(load().vf_apply_tree_static(h.ptr, PREC[precision], _dev_ptr(Xt, "Xt", n), R, _dev_ptr(Yt, "Yt", n),
                                       _stream(stream)))
    return Yt


def _solve_opts(rtol, max_iter, precision, refine, max_refine, inner_rtol, clamp, rho_uniform):
    return SolveOpts(rtol, max_iter, PREC[precision], int(refine), max_refine, inner_rtol, int(clamp),
                     float(rho_uniform))


def vf_solve(h: HMat, E, B, rho=0.12, rtol: float = 1e-6, max_iter: int = 100, precision: str = "fp32",
             refine: bool = False, max_refine: int = 8, inner_rtol: float = 1e-3, clamp: bool = False,
             stream=None) -> dict:
    """B = (I - diag(rho) F)^{-1} E.  rho: a float (uniform) or a CUDA
    tensor of N values.  Returns the solve statistics; raises on errors
    other than non-convergence (reported as stats['converged'] == 0)."""
    n = h.n
    R = 1 if E.dim() == 1 else E.shape[0]
    rho_ptr = None
    rho_u = 0.0
    if isinstance(rho, (int, float)):
        rho_u = float(rho)
    else:
        rho_ptr = _dev_ptr(rho, "rho", n)
    opts = _solve_opts(rtol, max_iter, precision, refine, max_refine, inner_rtol, clamp, rho_u)
    st = SolveStats()
    _check(load().vf_solve(h.ptr, rho_ptr, _dev_ptr(E, "E", n), n, _dev_ptr(B, "B", n), n, R, ctypes.byref(opts),
                           ctypes.byref(st), _stream(stream)), allow=(VF_E_NOCONV,))
    return st.as_dict()


def vf_solve_host(h: HMat, E: np.ndarray, B: np.ndarray, rho=0.12, rtol: float = 1e-6, max_iter: int = 100,
                  precision: str = "fp32", refine: bool = False, max_refine: int = 8, inner_rtol: float = 1e-3,
                  clamp: bool = False, stream=None) -> dict:
    """vf_solve on host arrays E, B of shape (R, N) float32 (C-contiguous,
    ideally pinned); the copies run inside the call."""
    n = h.n
    if E.dtype != np.float32 or B.dtype != np.float32 or E.shape != B.shape or E.shape[-1] != n:
        raise VFError(VF_E_INVAL, "E, B: float32 arrays of shape (R, N)")
    if not (E.flags.c_contiguous and B.flags.c_contiguous):
        raise VFError(VF_E_INVAL, "E, B must be C-contiguous")
    R = 1 if E.ndim == 1 else E.shape[0]
    rho_ptr = None
    rho_u = 0.0
    if isinstance(rho, (int, float)):
        rho_u = float(rho)
    else:
        rho = np.ascontiguousarray(rho, dtype=np.float32)
        rho_ptr = _np_ptr(rho)
    opts = _solve_opts(rtol, max_iter, precision, refine, max_refine, inner_rtol, clamp, rho_u)
    st = SolveStats()
    _check(load().vf_solve_host(h.ptr, rho_ptr, _np_ptr(E), n, _np_ptr(B), n, R, ctypes.byref(opts),
                                ctypes.byref(st), _stream(stream)), allow=(VF_E_NOCONV,))
    return st.as_dict()


def vf_solve_batched(hs, Es, Bs, rho=0.12, rtol: float = 1e-6, max_iter: int = 100, precision: str = "fp32",
                     refine: bool = False, max_refine: int = 8, inner_rtol: float = 1e-3, clamp: bool = False,
                     stream=None) -> list:
    k = len(hs)
    P = ctypes.c_void_p * k
    F = P(*[h.ptr for h in hs])
    E = P(*[_dev_ptr(e, "E", h.n).value for e, h in zip(Es, hs)])
    B = P(*[_dev_ptr(b, "B", h.n).value for b, h in zip(Bs, hs)])
    lde = (ctypes.c_int64 * k)(*[h.n for h in hs])
    R = (ctypes.c_int32 * k)(*[1 if e.dim() == 1 else e.shape[0] for e in Es])
    opts = _solve_opts(rtol, max_iter, precision, refine, max_refine, inner_rtol, clamp,
                       rho if isinstance(rho, (int, float)) else 0.0)
    rho_arr = None
    if not isinstance(rho, (int, float)):
        rho_arr = P(*[_dev_ptr(r, "rho", h.n).value for r, h in zip(rho, hs)])
    st = (SolveStats * k)()
    _check(load().vf_solve_batched(F, k, rho_arr, E, lde, B, lde, R, ctypes.byref(opts), st, _stream(stream)),
           allow=(VF_E_NOCONV,))
    return [s.as_dict() for s in st]


class EquilibriumOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("refine", ctypes.c_int32), ("albedo", ctypes.c_float), ("emissivity", ctypes.c_float)]


def _opt_vec(x, name, n):
    """(device pointer or None, uniform value) for a scalar or an N-vector CUDA tensor."""
    if isinstance(x, (int, float)):
        return None, float(x)
    return _dev_ptr(x, name, n), 0.0


def vf_equilibrium(h: HMat, E, T, albedo=0.12, emissivity=0.95, H=None, Qvis=None, Qir=None, rtol: float = 1e-6,
                   max_iter: int = 200, precision: str = "fp32", refine: bool = False, stream=None) -> list:
    """Section 5.1 equilibrium temperatures T (R, N) for the direct fluxes E (R, N);
    albedo / emissivity: floats or CUDA tensors of N values; H: None or N values.
    Returns the statistics of the Q_vis and Q_IR solves."""
    n = h.n
    R = 1 if E.dim() == 1 else E.shape[0]
    for nm, t in (("T", T), ("Qvis", Qvis), ("Qir", Qir)):
        if t is not None and tuple(t.shape) != tuple(E.shape):
            raise VFError(VF_E_INVAL, f"{nm} must have E's shape")
    ap, au = _opt_vec(albedo, "albedo", n)
    ep, eu = _opt_vec(emissivity, "emissivity", n)
    hp = None if H is None else _dev_ptr(H, "H", n)
    o = EquilibriumOpts(rtol, max_iter, PREC[precision], int(refine), au, eu)
    st = (SolveStats * 2)()
    _check(load().vf_equilibrium(h.ptr, _dev_ptr(E, "E", n), n, R, ap, ep, hp, ctypes.byref(o),
                                 None if Qvis is None else _dev_ptr(Qvis, "Qvis", n),
                                 None if Qir is None else _dev_ptr(Qir, "Qir", n), _dev_ptr(T, "T", n), n, st,
                                 _stream(stream)), allow=(VF_E_NOCONV,))
    return [x.as_dict() for x in st]


def vf_flux_step(h: HMat, Edirect_next, Qrefl, Qir, Qrad, Qabs, albedo=0.12, emissivity=0.95,
                 precision: str = "fp32", stream=None):
    """Algorithm 6: one step of the fluxes (R, N) in place (Qrefl, Qir updated, Qabs written)."""
    n = h.n
    R = 1 if Edirect_next.dim() == 1 else Edirect_next.shape[0]
    for nm, t in (("Qrefl", Qrefl), ("Qir", Qir), ("Qrad", Qrad), ("Qabs", Qabs)):
        if tuple(t.shape) != tuple(Edirect_next.shape):
            raise VFError(VF_E_INVAL, f"{nm} must have Edirect_next's shape")
    ap, au = _opt_vec(albedo, "albedo", n)
    ep, eu = _opt_vec(emissivity, "emissivity", n)
    _check(load().vf_flux_step(h.ptr, PREC[precision], R, ap, ep, au, eu, _dev_ptr(Edirect_next, "Edirect_next", n),
                               _dev_ptr(Qrefl, "Qrefl", n), _dev_ptr(Qir, "Qir", n), _dev_ptr(Qrad, "Qrad", n),
                               _dev_ptr(Qabs, "Qabs", n), n, _stream(stream)))


class Tune(ctypes.Structure):
    _fields_ = [("rb", ctypes.c_int32), ("tensor", ctypes.c_int32), ("rhs_block", ctypes.c_int32),
                ("us_per_rhs", ctypes.c_float)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


def vf_autotune(h: HMat, precision: str = "fp32", R: int = 1, stream=None) -> dict:
    """Time the multiply's candidate configurations for (precision, R) and keep the fastest in h."""
    t = Tune()
    _check(load().vf_autotune(h.ptr, PREC[precision], R, ctypes.byref(t), _stream(stream)))
    return t.as_dict()


def vf_tune_set(h: HMat, precision: str, R: int, rb: int, tensor: int = 0, rhs_block: int = 0):
    t = Tune(rb, tensor, rhs_block, 0.0)
    _check(load().vf_tune_set(h.ptr, PREC[precision], R, ctypes.byref(t)))


def vf_hmat_stack(hs) -> HMat:
    """The block-diagonal composition of the matrices hs (facets mesh after mesh)."""
    k = len(hs)
    P = ctypes.c_void_p * k
    out = ctypes.c_void_p()
    _check(load().vf_hmat_stack(P(*[h.ptr for h in hs]), k, ctypes.byref(out)))
    return HMat(out)


def vf_hmat_tensor_bytes(h: HMat, terms: int = 1) -> dict:
    """Bytes of the tensor-core pages of h (terms 1: BF16, 2: hi/lo split, 3: FP8), in all and by record kind."""
    tot = ctypes.c_int64()
    kinds = (ctypes.c_int64 * 5)()
    _check(load().vf_hmat_tensor_bytes(h.ptr, terms, ctypes.byref(tot), kinds))
    return {"total": tot.value, "dense": kinds[0], "csr": kinds[1], "svd_u": kinds[2], "svd_v": kinds[3],
            "empty": kinds[4]}


def vf_hmat_trim(h: HMat):
    """Free the workspaces, tensor pages and stacks cached on h (rebuilt on demand)."""
    _check(load().vf_hmat_trim(h.ptr))


def vf_hmat_nsegments(h: HMat) -> int:
    return int(load().vf_hmat_nsegments(h.ptr))


def vf_hmat_save(h: HMat, path: str):
    _check(load().vf_hmat_save(h.ptr, path.encode()))


def vf_hmat_load(path: str, device: int = 0) -> HMat:
    out = ctypes.c_void_p()
    _check(load().vf_hmat_load(path.encode(), device, ctypes.byref(out)))
    return HMat(out)


@dataclass
class Problem:
    """A mesh with its tree and compressed matrix, kept alive together."""
    mesh: Mesh
    tree: Tree
    hmat: HMat
    stats: dict


def build_problem(verts, faces, kind: str = "quad", leaf_size: int = 64, tol: float = 1e-3, device: int = 0,
                  **assemble_kw) -> Problem:
    m = vf_mesh_create(verts, faces, device)
    t = vf_partition(m, kind, leaf_size)
    h, st = vf_assemble(m, t, tol=tol, **assemble_kw)
    return Problem(m, t, h, st)


# ------------------------------------------------------------------ rank predictor
def _f32(a, shape_tail=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a


def vf_hmat_probe_log(h: HMat):
    """The assembly's probe log: (features n x VF_PRED_NFEAT float32, labels n int32)."""
    n = ctypes.c_int64(0)
    _check(load().vf_hmat_probe_log(h.ptr, ctypes.byref(n), None, None))
    X = np.zeros((n.value, VF_PRED_NFEAT), dtype=np.float32)
    y = np.zeros(n.value, dtype=np.int32)
    if n.value:
        _check(load().vf_hmat_probe_log(h.ptr, ctypes.byref(n), X.ctypes.data_as(ctypes.c_void_p),
                                        y.ctypes.data_as(ctypes.c_void_p)))
    return X, y


def vf_predictor_create(seed: int = 0, device: int = 0) -> Predictor:
    out = ctypes.c_void_p()
    _check(load().vf_predictor_create(device, ctypes.c_uint64(seed), ctypes.byref(out)))
    return Predictor(out.value)


def vf_predictor_params(p: Predictor, set_to=None) -> np.ndarray:
    """Flat parameters + feature means and scales (VF_PRED_NPARAM + 20 float32);
    with set_to, load those first."""
    if set_to is not None:
        s = _f32(set_to)
        if s.size != VF_PRED_NPARAM + 2 * VF_PRED_NFEAT:
            raise VFError(VF_E_INVAL, "parameter vector has the wrong size")
        _check(load().vf_predictor_params(p.ptr, None, s.ctypes.data_as(ctypes.c_void_p)))
    out = np.zeros(VF_PRED_NPARAM + 2 * VF_PRED_NFEAT, dtype=np.float32)
    _check(load().vf_predictor_params(p.ptr, out.ctypes.data_as(ctypes.c_void_p), None))
    return out


def _xy(X, y):
    X = _f32(X)
    y = np.ascontiguousarray(y, dtype=np.int32)
    if X.ndim != 2 or X.shape[1] != VF_PRED_NFEAT or y.shape != (X.shape[0],):
        raise VFError(VF_E_INVAL, "features must be (n, VF_PRED_NFEAT) with n labels")
    return X, y


def vf_predictor_grad(p: Predictor, X, y):
    """(mean loss, gradient VF_PRED_NPARAM float32) on the samples."""
    X, y = _xy(X, y)
    loss = ctypes.c_double(0.0)
    g = np.zeros(VF_PRED_NPARAM, dtype=np.float32)
    _check(load().vf_predictor_grad(p.ptr, X.ctypes.data_as(ctypes.c_void_p), y.ctypes.data_as(ctypes.c_void_p),
                                    X.shape[0], ctypes.byref(loss), g.ctypes.data_as(ctypes.c_void_p)))
    return loss.value, g


def vf_predictor_train(p: Predictor, X, y, epochs: int = 20, batch: int = 1024, lr: float = 2e-3) -> float:
    X, y = _xy(X, y)
    loss = ctypes.c_double(0.0)
    _check(load().vf_predictor_train(p.ptr, X.ctypes.data_as(ctypes.c_void_p), y.ctypes.data_as(ctypes.c_void_p),
                                     X.shape[0], epochs, batch, ctypes.c_float(lr), ctypes.byref(loss)))
    return loss.value


def vf_predictor_predict(p: Predictor, X):
    """(classes int32, probabilities n x VF_PRED_NCLASS float32)."""
    X = _f32(X)
    n = X.shape[0]
    cls = np.zeros(n, dtype=np.int32)
    prob = np.zeros((n, VF_PRED_NCLASS), dtype=np.float32)
    _check(load().vf_predictor_predict(p.ptr, X.ctypes.data_as(ctypes.c_void_p), n,
                                       cls.ctypes.data_as(ctypes.c_void_p), prob.ctypes.data_as(ctypes.c_void_p)))
    return cls, prob
