"""ctypes binding of libtrbl.so: same names as the C entry points, plus two
small owning wrappers (Basis, Hamiltonian) and ``solve``."""
from __future__ import annotations

import ctypes as C
from typing import Sequence

import numpy as np

from . import build as _build

TRBL_OK, TRBL_ERR_ARG, TRBL_ERR_CUDA, TRBL_ERR_OOM, TRBL_ERR_BREAKDOWN, TRBL_ERR_NOCONV = range(6)
TRBL_F32, TRBL_F64 = 0, 1
TRBL_PREC_F64, TRBL_PREC_MIXED = 1, 2
TRBL_PROJ_TENSOR, TRBL_PROJ_CUDA_CORE = 0, 1
TRBL_REORTH_SELECTIVE, TRBL_REORTH_TWICE = 0, 1
TRBL_NOALLOC_SCRATCH_BYTES = 8 << 20  # include/trbl.h
TRBL_APPLY_GROUPED, TRBL_APPLY_FAST, TRBL_APPLY_GROUPED_X2, TRBL_APPLY_SPLIT, TRBL_APPLY_SPLIT_X4, TRBL_APPLY_SPLIT_TMA = \
    0, 1, 2, 3, 4, 5
TRBL_TUNE_CANDIDATES = 15


class TrblError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("trbl error %d: %s" % (code, msg))
        self.code = code


class trbl_space(C.Structure):
    _fields_ = [("n_states", C.c_int), ("twoj", C.POINTER(C.c_int)), ("twom", C.POINTER(C.c_int)),
                ("orbit", C.POINTER(C.c_int)), ("n_particles", C.c_int)]


class trbl_basis_sizes(C.Structure):
    _fields_ = [("dim", C.c_int64), ("n_det", C.c_int32 * 2), ("n_blocks", C.c_int32),
                ("n_jumps", C.c_int64 * 2), ("n_delta", C.c_int32)]


class trbl_params(C.Structure):
    _fields_ = [("nev", C.c_int), ("q", C.c_int), ("max_basis", C.c_int), ("keep", C.c_int),
                ("tol", C.c_double), ("precision", C.c_int), ("max_iter", C.c_int),
                ("check_every", C.c_int), ("seed", C.c_uint64), ("normH", C.c_double),
                ("projections", C.c_int), ("reorth", C.c_int), ("refine", C.c_int)]


class trbl_stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("restarts", C.c_int), ("converged", C.c_int),
                ("status", C.c_int), ("normH", C.c_double), ("ms_total", C.c_double),
                ("ms_apply", C.c_double), ("ms_orth", C.c_double), ("ms_qr", C.c_double),
                ("ms_ritz", C.c_double), ("ms_restart", C.c_double), ("basis_size", C.c_int), ("second_passes", C.c_int),
                ("ms_copy_in", C.c_double), ("ms_copy_out", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_LIB = None
_VP = C.c_void_p
_DP = C.POINTER(C.c_double)


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libtrbl.so, building it first when a source is newer.  Raises if it
    cannot be built or loaded: there is no fallback path."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.build()
    L = C.CDLL(path)
    sig = {
        "trbl_basis_create": (C.c_int, [C.POINTER(trbl_space), C.POINTER(trbl_space), C.c_int, C.POINTER(_VP)]),
        "trbl_basis_destroy": (None, [_VP]),
        "trbl_basis_info": (C.c_int, [_VP, C.POINTER(trbl_basis_sizes)]),
        "trbl_basis_export": (C.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
        "trbl_basis_export_jumps": (C.c_int, [_VP, C.c_int, _VP, _VP, _VP, _VP, _VP]),
        "trbl_hamiltonian_create": (C.c_int, [_VP, _DP, _DP, _DP, _DP, _DP, C.POINTER(_VP)]),
        "trbl_hamiltonian_destroy": (None, [_VP]),
        "trbl_apply_block": (C.c_int, [_VP, _VP, C.c_int64, _VP, C.c_int64, C.c_int, C.c_int, _VP]),
        "trbl_solve": (C.c_int, [_VP, C.POINTER(trbl_params), _DP, _DP, _VP, C.POINTER(trbl_stats), _VP]),
        "trbl_solver_create": (C.c_int, [_VP, C.POINTER(trbl_params), _VP, C.POINTER(_VP)]),
        "trbl_solver_step": (C.c_int, [_VP, C.POINTER(C.c_int)]),
        "trbl_solver_step_host": (C.c_int, [_VP, _VP, _VP, C.POINTER(C.c_int)]),
        "trbl_solver_block": (C.c_int, [_VP, C.POINTER(_VP), C.POINTER(C.c_int64)]),
        "trbl_solver_stats": (C.c_int, [_VP, C.POINTER(trbl_stats)]),
        "trbl_solver_finish": (C.c_int, [_VP, _DP, _DP, _VP, C.POINTER(trbl_stats)]),
        "trbl_solver_destroy": (None, [_VP]),
        "trbl_solver_state_bytes": (C.c_int, [_VP, C.POINTER(C.c_int64)]),
        "trbl_solver_save": (C.c_int, [_VP, _VP, C.c_int64]),
        "trbl_solver_load": (C.c_int, [_VP, _VP, C.c_int64]),
        "trbl_block_dot": (C.c_int, [_VP, C.c_int64, C.c_int, _VP, C.c_int64, C.c_int, C.c_int64, C.c_int, _VP, _VP]),
        "trbl_block_dot_noalloc": (C.c_int, [_VP, C.c_int64, C.c_int, _VP, C.c_int64, C.c_int, C.c_int64, C.c_int,
                                             _VP, _VP]),
        "trbl_block_dot_tc": (C.c_int, [_VP, C.c_int64, C.c_int, _VP, C.c_int64, C.c_int, C.c_int64, _VP, _VP]),
        "trbl_block_update": (C.c_int, [_VP, C.c_int64, C.c_int, _VP, C.c_int64, C.c_int, _VP, C.c_int64,
                                        C.c_int64, C.c_double, C.c_double, C.c_int, C.c_int, _VP]),
        "trbl_param_count": (C.c_int, [_VP, C.POINTER(C.c_int64)]),
        "trbl_grad": (C.c_int, [_VP, _VP, C.c_int64, C.c_int, C.c_int, _DP, C.c_int64, _VP]),
        "trbl_grad_clusters": (C.c_int, [_VP, _VP, C.c_int64, C.c_int, C.c_int, C.POINTER(C.c_int), C.c_int, _DP,
                                         C.c_int64, _VP]),
        "trbl_solve_batch": (C.c_int, [C.POINTER(_VP), C.c_int, C.POINTER(trbl_params), _DP, _DP, _VP,
                                       C.POINTER(C.c_int), C.POINTER(trbl_stats), _VP]),
        "trbl_apply_autotune": (C.c_int, [_VP, C.c_int, C.c_int, C.POINTER(C.c_float), C.POINTER(C.c_int), _VP]),
        "trbl_apply_set_rows": (C.c_int, [_VP, C.c_int]),
        "trbl_apply_set_shape": (C.c_int, [_VP, C.c_int, C.c_int, C.c_int]),
        "trbl_apply_get_shape": (C.c_int, [_VP, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "trbl_apply_set_compensated": (C.c_int, [_VP, C.c_int]),
        "trbl_host_alloc": (C.c_int, [C.c_size_t, C.c_int, C.POINTER(_VP), C.POINTER(C.c_int)]),
        "trbl_host_free": (C.c_int, [_VP]),
        "trbl_shard_plan": (C.c_int, [_VP, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
        "trbl_shard_sources": (C.c_int, [_VP, C.c_int64, C.c_int64, C.POINTER(C.c_int64), C.c_int64,
                                         C.POINTER(C.c_int64)]),
        "trbl_hamiltonian_set_rows": (C.c_int, [_VP, C.c_int64, C.c_int64]),
        "trbl_kernel_launches": (C.c_longlong, []),
        "trbl_last_error": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _LIB = L
    return L


def trbl_kernel_launches() -> int:
    return int(lib().trbl_kernel_launches())


def trbl_last_error() -> str:
    return lib().trbl_last_error().decode()


def _check(rc: int):
    if rc != TRBL_OK:
        raise TrblError(rc, trbl_last_error())


def _iarr(x: Sequence[int]):
    a = (C.c_int * len(x))(*[int(v) for v in x])
    return a


def _space(sp, k: int):
    """trbl_space from an object with twoj/twom/orbit sequences (e.g. synth.ModelSpace)."""
    tj, tm, ob = _iarr(sp.twoj), _iarr(sp.twom), _iarr(sp.orbit)
    s = trbl_space(len(sp.twom), tj, tm, ob, int(k))
    return s, (tj, tm, ob)


def _f64(a: np.ndarray):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_DP)


# ---- raw entry points (same names as the C ABI) ------------------------------

def trbl_basis_create(spaceA, kA: int, spaceB, kB: int, twoM: int) -> int:
    sA, keepA = _space(spaceA, kA)
    sB, keepB = _space(spaceB, kB)
    out = _VP()
    _check(lib().trbl_basis_create(C.byref(sA), C.byref(sB), int(twoM), C.byref(out)))
    return out.value


def trbl_basis_destroy(b: int):
    lib().trbl_basis_destroy(b)


def trbl_basis_info(b: int) -> dict:
    s = trbl_basis_sizes()
    _check(lib().trbl_basis_info(b, C.byref(s)))
    return {"dim": s.dim, "n_det": (s.n_det[0], s.n_det[1]), "n_blocks": s.n_blocks,
            "n_jumps": (s.n_jumps[0], s.n_jumps[1]), "n_delta": s.n_delta}


def trbl_basis_export(b: int):
    info = trbl_basis_info(b)
    nA, nB = info["n_det"]
    bitsA = np.zeros(nA, np.uint32)
    mA = np.zeros(nA, np.int32)
    bitsB = np.zeros(nB, np.uint32)
    mB = np.zeros(nB, np.int32)
    blocks = np.zeros((info["n_blocks"], 7), np.int64)
    _check(lib().trbl_basis_export(b, bitsA.ctypes.data, mA.ctypes.data, bitsB.ctypes.data,
                                   mB.ctypes.data, blocks.ctypes.data))
    return bitsA, mA, bitsB, mB, blocks


def trbl_basis_export_jumps(b: int, species: int):
    n = trbl_basis_info(b)["n_jumps"][species]
    tgt, src, a, c = (np.zeros(n, np.int32) for _ in range(4))
    sign = np.zeros(n, np.int8)
    _check(lib().trbl_basis_export_jumps(b, int(species), tgt.ctypes.data, src.ctypes.data,
                                         a.ctypes.data, c.ctypes.data, sign.ctypes.data))
    return tgt, src, a, c, sign


def trbl_hamiltonian_create(b: int, h1A, h1B, VAA, VBB, VAB) -> int:
    arrs = [_f64(x) for x in (h1A, h1B, VAA, VBB, VAB)]
    out = _VP()
    _check(lib().trbl_hamiltonian_create(b, *[p for _, p in arrs], C.byref(out)))
    return out.value


def trbl_hamiltonian_destroy(h: int):
    lib().trbl_hamiltonian_destroy(h)


def trbl_apply_block(h: int, V_ptr: int, ldv: int, W_ptr: int, ldw: int, q: int, dtype: int,
                     stream: int = 0):
    _check(lib().trbl_apply_block(h, V_ptr, int(ldv), W_ptr, int(ldw), int(q), int(dtype), stream))


def trbl_block_dot(B_ptr: int, ldb: int, m: int, W_ptr: int, ldw: int, q: int, D: int, dtype: int,
                   C_ptr: int, stream: int = 0):
    _check(lib().trbl_block_dot(B_ptr, int(ldb), int(m), W_ptr, int(ldw), int(q), int(D), int(dtype), C_ptr,
                                stream))


def trbl_block_dot_noalloc(B_ptr: int, ldb: int, m: int, W_ptr: int, ldw: int, q: int, D: int, dtype: int,
                           C_ptr: int, stream: int = 0):
    """Allocation-free C = B^T W (see include/trbl.h): scratch is a fixed
    array compiled into the library; overlapping calls on one device race."""
    _check(lib().trbl_block_dot_noalloc(B_ptr, int(ldb), int(m), W_ptr, int(ldw), int(q), int(D), int(dtype),
                                        C_ptr, stream))


def trbl_block_dot_tc(B_ptr: int, ldb: int, m: int, W_ptr: int, ldw: int, q: int, D: int, C_ptr: int,
                      stream: int = 0):
    _check(lib().trbl_block_dot_tc(B_ptr, int(ldb), int(m), W_ptr, int(ldw), int(q), int(D), C_ptr, stream))


def trbl_block_update(In_ptr: int, ldi: int, K: int, U_ptr: int, ldu: int, n: int, Out_ptr: int, ldo: int, D: int,
                      alpha: float, beta: float, dtype: int, algo: int, stream: int = 0):
    _check(lib().trbl_block_update(In_ptr, int(ldi), int(K), U_ptr, int(ldu), int(n), Out_ptr, int(ldo), int(D),
                                   float(alpha), float(beta), int(dtype), int(algo), stream))


def block_dot(B, W, stream=None, tensor_cores=False):
    """C = B^T W (FP64, m x q) for torch CUDA tensors B (D x m) and W (D x q);
    tensor_cores=True uses trbl_block_dot_tc (FP32 data only)."""
    import torch
    if B.dtype != W.dtype or B.stride(1) != 1 or W.stride(1) != 1 or B.shape[0] != W.shape[0]:
        raise ValueError("B and W must share dtype and rows, with unit column stride")
    dt = TRBL_F64 if B.dtype == torch.float64 else TRBL_F32
    C = torch.empty((B.shape[1], W.shape[1]), dtype=torch.float64, device=B.device)
    s = stream if stream is not None else torch.cuda.current_stream(B.device)
    if tensor_cores:
        trbl_block_dot_tc(B.data_ptr(), B.stride(0), B.shape[1], W.data_ptr(), W.stride(0), W.shape[1], B.shape[0],
                          C.data_ptr(), s.cuda_stream)
    else:
        trbl_block_dot(B.data_ptr(), B.stride(0), B.shape[1], W.data_ptr(), W.stride(0), W.shape[1], B.shape[0], dt,
                       C.data_ptr(), s.cuda_stream)
    return C


def block_update(In, U, Out, alpha=-1.0, beta=1.0, algo=TRBL_PROJ_TENSOR, stream=None):
    """Out = alpha * In U + beta * Out in place (In: D x K, U: K x n FP64, Out:
    D x n, torch CUDA tensors with unit column stride); returns Out."""
    import torch
    if In.dtype != Out.dtype or In.stride(1) != 1 or Out.stride(1) != 1 or In.shape[0] != Out.shape[0]:
        raise ValueError("In and Out must share dtype and rows, with unit column stride")
    U = U.to(device=In.device, dtype=torch.float64).contiguous()
    dt = TRBL_F64 if In.dtype == torch.float64 else TRBL_F32
    s = stream if stream is not None else torch.cuda.current_stream(In.device)
    trbl_block_update(In.data_ptr(), In.stride(0), In.shape[1], U.data_ptr(), U.stride(0), U.shape[1],
                      Out.data_ptr(), Out.stride(0), In.shape[0], alpha, beta, dt, algo, s.cuda_stream)
    return Out


def trbl_solve(h: int, params: trbl_params, evals_ptr, resid_ptr, evecs_ptr: int,
               stats: trbl_stats, stream: int = 0) -> int:
    rc = lib().trbl_solve(h, C.byref(params), evals_ptr, resid_ptr, evecs_ptr, C.byref(stats), stream)
    return rc


# ---- owning wrappers ---------------------------------------------------------

class Basis:
    """Two-species M-scheme basis built by the library (host-side tables)."""

    def __init__(self, spaceA, kA: int, spaceB, kB: int, twoM: int):
        self.handle = None
        self.handle = trbl_basis_create(spaceA, kA, spaceB, kB, twoM)
        self.twomA, self.twomB = tuple(int(x) for x in spaceA.twom), tuple(int(x) for x in spaceB.twom)
        self.info = trbl_basis_info(self.handle)
        self.dim = self.info["dim"]

    def export(self):
        return trbl_basis_export(self.handle)

    def export_jumps(self, species: int):
        return trbl_basis_export_jumps(self.handle, species)

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.trbl_basis_destroy(self.handle)
            self.handle = None


class Hamiltonian:
    """Device tables of H on a Basis (current CUDA device)."""

    def __init__(self, basis: Basis, h1A, h1B, VAA, VBB, VAB):
        self.handle = None
        self.basis = basis
        self.handle = trbl_hamiltonian_create(basis.handle, h1A, h1B, VAA, VBB, VAB)

    @classmethod
    def from_interaction(cls, basis: Basis, inter):
        return cls(basis, inter.h1A, inter.h1B, inter.VAA, inter.VBB, inter.VAB)

    def apply(self, V, W=None, stream=None):
        """W = H V for a torch CUDA tensor V of shape (D, q), float32 or float64."""
        import torch
        if V.dim() != 2 or V.shape[0] != self.basis.dim or V.stride(1) != 1:
            raise ValueError("V must be (D, q) with unit column stride")
        if not V.is_cuda:
            raise ValueError("V must be a CUDA tensor")
        if V.dtype == torch.float64:
            dt = TRBL_F64
        elif V.dtype == torch.float32:
            dt = TRBL_F32
        else:
            raise ValueError("V must be float32 or float64")
        if W is None:
            W = torch.empty_like(V, memory_format=torch.contiguous_format)
        if W.shape != V.shape or W.dtype != V.dtype or W.stride(1) != 1:
            raise ValueError("W must match V's shape and dtype with unit column stride")
        s = stream if stream is not None else torch.cuda.current_stream(V.device)
        trbl_apply_block(self.handle, V.data_ptr(), V.stride(0), W.data_ptr(), W.stride(0),
                         V.shape[1], dt, s.cuda_stream)
        return W

    def set_rows(self, row_begin: int, row_end: int):
        """Restrict the product to W rows [row_begin, row_end) (slab boundaries;
        0 and D restore the whole product)."""
        _check(lib().trbl_hamiltonian_set_rows(self.handle, int(row_begin), int(row_end)))

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.trbl_hamiltonian_destroy(self.handle)
            self.handle = None


def solve(h: Hamiltonian, nev: int, q: int, max_basis: int, tol: float,
          precision: int = TRBL_PREC_F64, keep: int = 0, max_iter: int = 0,
          check_every: int = 0, seed: int = 1, normH: float = 0.0, want_vectors: bool = True,
          stream=None, raise_on_noconv: bool = True, projections: int = TRBL_PROJ_TENSOR,
          reorth: int = TRBL_REORTH_SELECTIVE, refine: bool = False):
    """Lowest nev eigenpairs by trbl_solve.  Returns (evals, resid, evecs or None, stats dict).
    refine (mixed precision): iterate on until the true residuals meet tol."""
    import torch
    D = h.basis.dim
    p = _params(nev, q, max_basis, tol, precision, keep, max_iter, check_every, seed, normH, projections, reorth,
                refine)
    st = trbl_stats()
    ev = np.zeros(nev)
    rs = np.zeros(nev)
    X = None
    if want_vectors:
        dt = torch.float64 if precision == TRBL_PREC_F64 else torch.float32
        X = torch.empty((D, nev), dtype=dt, device="cuda")
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = trbl_solve(h.handle, p, ev.ctypes.data_as(_DP), rs.ctypes.data_as(_DP),
                    X.data_ptr() if X is not None else None, st, s.cuda_stream)
    if rc != TRBL_OK and not (rc == TRBL_ERR_NOCONV and not raise_on_noconv):
        raise TrblError(rc, trbl_last_error())
    d = st.as_dict()
    d["rc"] = rc
    return ev, rs, X, d


def _params(nev, q, max_basis, tol, precision=TRBL_PREC_F64, keep=0, max_iter=0, check_every=0, seed=1,
            normH=0.0, projections=TRBL_PROJ_TENSOR, reorth=TRBL_REORTH_SELECTIVE, refine=False):
    return trbl_params(int(nev), int(q), int(max_basis), int(keep), float(tol), int(precision),
                       int(max_iter), int(check_every), int(seed), float(normH), int(projections), int(reorth),
                       int(bool(refine)))


def trbl_solver_create(h: int, params: trbl_params, stream: int = 0) -> int:
    out = _VP()
    _check(lib().trbl_solver_create(h, C.byref(params), stream, C.byref(out)))
    return out.value


def trbl_solver_step(sv: int) -> int:
    c = C.c_int(-1)
    _check(lib().trbl_solver_step(sv, C.byref(c)))
    return c.value


def trbl_solver_step_host(sv: int, block_in: int, block_out: int) -> int:
    c = C.c_int(-1)
    _check(lib().trbl_solver_step_host(sv, block_in, block_out, C.byref(c)))
    return c.value


def trbl_solver_block(sv: int):
    p = _VP()
    n = C.c_int64()
    _check(lib().trbl_solver_block(sv, C.byref(p), C.byref(n)))
    return p.value, n.value


def trbl_solver_stats(sv: int) -> dict:
    st = trbl_stats()
    _check(lib().trbl_solver_stats(sv, C.byref(st)))
    return st.as_dict()


def trbl_solver_destroy(sv: int):
    lib().trbl_solver_destroy(sv)


def trbl_solver_state_bytes(sv: int) -> int:
    n = C.c_int64()
    _check(lib().trbl_solver_state_bytes(sv, C.byref(n)))
    return n.value


def trbl_solver_save(sv: int, host_ptr: int, nbytes: int):
    _check(lib().trbl_solver_save(sv, host_ptr, nbytes))


def trbl_solver_load(sv: int, host_ptr: int, nbytes: int):
    _check(lib().trbl_solver_load(sv, host_ptr, nbytes))


def shard_plan(basis: "Basis", nranks: int):
    """(bounds[nranks + 1], work[nranks]): slab-aligned row ranges of W
    balanced by generated elements (trbl_shard_plan)."""
    bounds = (C.c_int64 * (nranks + 1))()
    work = (C.c_int64 * nranks)()
    _check(lib().trbl_shard_plan(basis.handle, int(nranks), bounds, work))
    return list(bounds), list(work)


def shard_sources(basis: "Basis", row_begin: int, row_end: int):
    """[(begin, end), ...]: the V rows the product of W rows [row_begin,
    row_end) reads (trbl_shard_sources)."""
    n = C.c_int64()
    _check(lib().trbl_shard_sources(basis.handle, int(row_begin), int(row_end), None, 0, C.byref(n)))
    r = (C.c_int64 * (2 * max(n.value, 1)))()
    _check(lib().trbl_shard_sources(basis.handle, int(row_begin), int(row_end), r, n.value, C.byref(n)))
    return [(r[2 * i], r[2 * i + 1]) for i in range(n.value)]


class HostBuffer:
    """Page-locked host memory (trbl_host_alloc); .array is a numpy view,
    .ptr the address, .numa_node the GPU's nearest host memory node (-1 if
    the device reports none)."""

    def __init__(self, nbytes: int, device: int = 0, dtype=np.float32):
        p, node = _VP(), C.c_int()
        _check(lib().trbl_host_alloc(int(nbytes), int(device), C.byref(p), C.byref(node)))
        self.ptr, self.nbytes, self.numa_node = p.value, int(nbytes), node.value
        n = int(nbytes) // np.dtype(dtype).itemsize
        buf = (C.c_char * int(nbytes)).from_address(self.ptr)
        self.array = np.frombuffer(buf, dtype=dtype, count=n)

    def data_ptr(self) -> int:
        return self.ptr

    def free(self):
        if getattr(self, "ptr", None):
            self.array = None
            _check(lib().trbl_host_free(self.ptr))
            self.ptr = None

    def __del__(self):
        if getattr(self, "ptr", None) and _LIB is not None:
            self.array = None
            _LIB.trbl_host_free(self.ptr)
            self.ptr = None


class Solver:
    """Stepwise thick-restart block Lanczos (trbl_solver_* entry points)."""

    def __init__(self, h: Hamiltonian, nev: int, q: int, max_basis: int, tol: float,
                 precision: int = TRBL_PREC_F64, keep: int = 0, check_every: int = 0, seed: int = 1,
                 normH: float = 0.0, stream=None, projections: int = TRBL_PROJ_TENSOR, max_iter: int = 0,
                 reorth: int = TRBL_REORTH_SELECTIVE):
        import torch
        self.h = h
        self.nev, self.q, self.precision = nev, q, precision
        self.handle = None
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        self.params = _params(nev, q, max_basis, tol, precision, keep, max_iter, check_every, seed, normH,
                              projections, reorth)
        self.handle = trbl_solver_create(h.handle, self.params, s.cuda_stream)

    def step(self) -> int:
        return trbl_solver_step(self.handle)

    def step_host(self, block_in, block_out) -> int:
        """One step with V_k read from / V_{k+1} written to host tensors (pinned for speed)."""
        return trbl_solver_step_host(self.handle, block_in.data_ptr() if block_in is not None else None,
                                     block_out.data_ptr() if block_out is not None else None)

    def block(self):
        return trbl_solver_block(self.handle)

    def save(self) -> np.ndarray:
        """Checkpoint: the solver's state between steps as a host byte array."""
        buf = np.empty(trbl_solver_state_bytes(self.handle), dtype=np.uint8)
        trbl_solver_save(self.handle, buf.ctypes.data, buf.nbytes)
        return buf

    def load(self, state: np.ndarray):
        """Resume from a checkpoint taken by save() (same sizes and precision)."""
        state = np.ascontiguousarray(state, dtype=np.uint8)
        trbl_solver_load(self.handle, state.ctypes.data, state.nbytes)

    def stats(self) -> dict:
        return trbl_solver_stats(self.handle)

    def fill(self) -> int:
        """Lanczos vectors in the basis now."""
        return self.stats()["basis_size"]

    def finish(self, want_vectors: bool = True, raise_on_noconv: bool = True):
        import torch
        D = self.h.basis.dim
        ev = np.zeros(self.nev)
        rs = np.zeros(self.nev)
        X = None
        if want_vectors:
            dt = torch.float64 if self.precision == TRBL_PREC_F64 else torch.float32
            X = torch.empty((D, self.nev), dtype=dt, device="cuda")
        st = trbl_stats()
        rc = lib().trbl_solver_finish(self.handle, ev.ctypes.data_as(_DP), rs.ctypes.data_as(_DP),
                                      X.data_ptr() if X is not None else None, C.byref(st))
        if rc != TRBL_OK and not (rc == TRBL_ERR_NOCONV and not raise_on_noconv):
            raise TrblError(rc, trbl_last_error())
        d = st.as_dict()
        d["rc"] = rc
        return ev, rs, X, d

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.trbl_solver_destroy(self.handle)
            self.handle = None


# ---- Hellmann-Feynman gradient -------------------------------------------------

def trbl_param_count(b: int) -> int:
    n = C.c_int64()
    _check(lib().trbl_param_count(b, C.byref(n)))
    return n.value


def trbl_grad(h: int, X_ptr: int, ldx: int, nvec: int, dtype: int, out: np.ndarray, stream: int = 0):
    _check(lib().trbl_grad(h, X_ptr, int(ldx), int(nvec), int(dtype), out.ctypes.data_as(_DP), int(out.size),
                           stream))


def _canonical_params(twomA, twomB):
    """(kind, indices) of every parameter in trbl_param_count's order."""
    out = []
    for name, m in (("h1A", twomA), ("h1B", twomB)):
        n = len(m)
        for a in range(n):
            for c in range(a, n):
                if m[a] == m[c]:
                    out.append((name, (a, c)))
    for name, m in (("VAA", twomA), ("VBB", twomB)):
        n = len(m)
        pairs = [(i, j) for i in range(n) for j in range(i + 1, n)]
        for I in range(len(pairs)):
            for J in range(I, len(pairs)):
                (i, j), (k, l) = pairs[I], pairs[J]
                if m[i] + m[j] == m[k] + m[l]:
                    out.append((name, (i, j, k, l)))
    nB = len(twomB)
    pairs = [(a, b) for a in range(len(twomA)) for b in range(nB)]
    for I in range(len(pairs)):
        for J in range(I, len(pairs)):
            (a, b), (c, d) = pairs[I], pairs[J]
            if twomA[a] + twomB[b] == twomA[c] + twomB[d]:
                out.append(("VAB", (a, b, c, d)))
    return out


def arrays_from_theta(twomA, twomB, theta):
    """Dense coefficient arrays (h1A, h1B, VAA, VBB, VAB) of trbl_hamiltonian_create
    from a parameter vector in trbl_param_count's order."""
    nA, nB = len(twomA), len(twomB)
    A = {"h1A": np.zeros((nA, nA)), "h1B": np.zeros((nB, nB)), "VAA": np.zeros((nA,) * 4),
         "VBB": np.zeros((nB,) * 4), "VAB": np.zeros((nA, nB, nA, nB))}
    theta = np.asarray(theta, dtype=np.float64)
    params = _canonical_params(twomA, twomB)
    if len(params) != theta.size:
        raise ValueError("theta has %d entries, the spaces have %d parameters" % (theta.size, len(params)))
    for (name, ix), x in zip(params, theta):
        T = A[name]
        if len(ix) == 2:
            T[ix[0], ix[1]] = x
            T[ix[1], ix[0]] = x
        else:
            i, j, k, l = ix
            T[i, j, k, l] = x
            T[k, l, i, j] = x
    return A["h1A"], A["h1B"], A["VAA"], A["VBB"], A["VAB"]


def clusters_of(evals, gap):
    """Index lists of consecutive eigenvalues closer than gap."""
    out, cur = [], [0]
    for k in range(1, len(evals)):
        if evals[k] - evals[k - 1] < gap:
            cur.append(k)
        else:
            out.append(cur)
            cur = [k]
    out.append(cur)
    return out


def hf_gradient(h: "Hamiltonian", X, cols=None, stream=None) -> np.ndarray:
    """sum over the selected columns x of X of <x| dH/dtheta |x> (trbl_grad),
    in chunks of at most 32 columns."""
    import torch
    if cols is None:
        cols = list(range(X.shape[1]))
    dt = TRBL_F64 if X.dtype == torch.float64 else TRBL_F32
    n = trbl_param_count(h.basis.handle)
    total = np.zeros(n)
    part = np.zeros(n)
    s = stream if stream is not None else torch.cuda.current_stream(X.device)
    for c0 in range(0, len(cols), 32):
        sub = X[:, cols[c0:c0 + 32]].contiguous()
        trbl_grad(h.handle, sub.data_ptr(), sub.stride(0), sub.shape[1], dt, part, s.cuda_stream)
        total += part
    return total


class LowestEigenvalues:
    """torch.autograd.Function computing the nev lowest eigenvalues of H(theta)
    with trbl_solve and their Hellmann-Feynman gradient with trbl_grad_clusters.

    Within a cluster of levels closer than cluster_tol * ||H|| only the sum of
    the derivatives is defined; backward gives each member the cluster's mean
    derivative (exact for losses symmetric within a cluster)."""

    @staticmethod
    def apply(theta, basis, nev, q, max_basis, tol, precision=TRBL_PREC_F64, cluster_tol=1e-8, seed=1):
        import torch

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, th):
                b = basis
                twomA, twomB = b.twomA, b.twomB
                h = Hamiltonian(b, *arrays_from_theta(twomA, twomB, th.detach().cpu().numpy()))
                ev, rs, X, st = solve(h, nev, q, max_basis, tol, precision=precision, seed=seed)
                cl = clusters_of(ev, cluster_tol * max(st["normH"], 1e-300))
                G = np.zeros((nev, th.numel()))
                for c, g in zip(cl, hf_gradient_clusters(h, X, cl)):
                    for k in c:
                        G[k] = g / len(c)
                ctx.save_for_backward(torch.from_numpy(G).to(th.dtype))
                return torch.from_numpy(ev).to(th.dtype)

            @staticmethod
            def backward(ctx, gout):
                (G,) = ctx.saved_tensors
                return gout @ G

        return _Fn.apply(theta)


# ---- batched solve and autotuner ---------------------------------------------

def solve_batch(hs, nev: int, q: int, max_basis: int, tol: float, precision: int = TRBL_PREC_F64,
                keep: int = 0, max_iter: int = 0, check_every: int = 0, seed: int = 1, normH: float = 0.0,
                want_vectors: bool = False, want_resid: bool = True, stream=None,
                projections: int = TRBL_PROJ_TENSOR, reorth: int = TRBL_REORTH_SELECTIVE):
    """trbl_solve_batch over Hamiltonians on one basis or on bases of
    different dimension.  Returns (evals [nset, nev], resid [nset, nev] or
    None, vectors or None, per-set status, stats dict); vectors is a
    [nset, D, nev] tensor when every set has the same dimension, else a list
    of [D_s, nev] views (set-major in one buffer)."""
    import torch
    nset = len(hs)
    dims = [h.basis.dim for h in hs]
    p = _params(nev, q, max_basis, tol, precision, keep, max_iter, check_every, seed, normH, projections, reorth)
    arr = (_VP * nset)(*[h.handle for h in hs])
    ev = np.zeros((nset, nev))
    rs = np.zeros((nset, nev)) if want_resid else None
    status = (C.c_int * nset)()
    X = buf = None
    if want_vectors:
        dt = torch.float64 if precision == TRBL_PREC_F64 else torch.float32
        buf = torch.empty(sum(dims) * nev, dtype=dt, device="cuda")
        if len(set(dims)) == 1:
            X = buf.view(nset, dims[0], nev)
        else:
            offs = np.concatenate([[0], np.cumsum(dims)]) * nev
            X = [buf[offs[i]:offs[i + 1]].view(dims[i], nev) for i in range(nset)]
    st = trbl_stats()
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = lib().trbl_solve_batch(arr, nset, C.byref(p), ev.ctypes.data_as(_DP),
                                rs.ctypes.data_as(_DP) if rs is not None else None,
                                buf.data_ptr() if buf is not None else None, status, C.byref(st), s.cuda_stream)
    d = st.as_dict()
    d["rc"] = rc
    d["message"] = trbl_last_error() if rc else ""
    return ev, rs, X, list(status), d


def apply_autotune(h: "Hamiltonian", q: int, dtype: int = TRBL_F32, stream=None):
    """Times the product for each launch shape (kernel, neutron rows per work
    item, blocks per SM; TRBL_TUNE_CANDIDATES of them, NaN where a shape does
    not apply) and keeps the fastest; returns (times in ms, rows chosen)."""
    import torch
    ms = (C.c_float * TRBL_TUNE_CANDIDATES)()
    best = C.c_int()
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().trbl_apply_autotune(h.handle, int(q), int(dtype), ms, C.byref(best), s.cuda_stream))
    return list(ms), best.value


def apply_set_rows(h: "Hamiltonian", rows_per_item: int):
    """Sets the product's neutron rows per work item."""
    _check(lib().trbl_apply_set_rows(h.handle, int(rows_per_item)))


def apply_set_shape(h: "Hamiltonian", kernel: int, rows_per_item: int, blocks_per_sm: int = 8):
    """Sets the product's kernel, rows per work item and blocks per SM."""
    _check(lib().trbl_apply_set_shape(h.handle, int(kernel), int(rows_per_item), int(blocks_per_sm)))


def apply_set_compensated(h: "Hamiltonian", on: bool):
    """Compensated (TwoSum) row sums in the FP32 fast product on or off."""
    _check(lib().trbl_apply_set_compensated(h.handle, 1 if on else 0))


def apply_get_shape(h: "Hamiltonian"):
    """(kernel, rows per work item, blocks per SM) of the product."""
    k, r, b = C.c_int(), C.c_int(), C.c_int()
    _check(lib().trbl_apply_get_shape(h.handle, C.byref(k), C.byref(r), C.byref(b)))
    return k.value, r.value, b.value


def hf_gradient_clusters(h: "Hamiltonian", X, clusters, stream=None):
    """Hellmann-Feynman gradients of several level clusters (lists of
    consecutive column indices of X, as clusters_of returns) with one
    trbl_grad_clusters pass per group of up to 32 columns; returns one
    array per cluster (a cluster of more than 32 columns goes through
    hf_gradient)."""
    import torch
    dt = TRBL_F64 if X.dtype == torch.float64 else TRBL_F32
    n = trbl_param_count(h.basis.handle)
    s = stream if stream is not None else torch.cuda.current_stream(X.device)
    out = [None] * len(clusters)
    k = 0
    while k < len(clusters):
        if len(clusters[k]) > 32:
            out[k] = hf_gradient(h, X, clusters[k], stream)
            k += 1
            continue
        group, cols = [], []
        while k < len(clusters) and len(clusters[k]) <= 32 and len(cols) + len(clusters[k]) <= 32:
            group.append(k)
            cols.extend(clusters[k])
            k += 1
        sub = X[:, cols].contiguous()
        first = [0]
        for g in group:
            first.append(first[-1] + len(clusters[g]))
        fa = (C.c_int * len(first))(*first)
        res = np.zeros((len(group), n))
        _check(lib().trbl_grad_clusters(h.handle, sub.data_ptr(), sub.stride(0), sub.shape[1], dt, fa, len(group),
                                        res.ctypes.data_as(_DP), n, s.cuda_stream))
        for i, g in enumerate(group):
            out[g] = res[i]
    return out
