"""Thin Python binding of libsfem.so (include/sfem.h).

Argument marshalling only: every step of setup, assembly, operator apply and
solve runs in the library's CUDA kernels.  PyTorch provides device memory
(through the library's allocator hooks, backed by torch's caching allocator)
and the CUDA stream.  If the library is missing the import of this module
fails; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libsfem.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "sfem.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libsfem.so not built ({LIB_PATH}); run __graft_entry__.build() "
                      "or python paper_2001_08849_gb300/build.py")
lib = ctypes.CDLL(LIB_PATH)

# ---- status codes and enums (include/sfem.h) --------------------------------
SFEM_OK, SFEM_EINVAL, SFEM_EMESH, SFEM_ENOMEM = 0, -1, -2, -3
SFEM_ENOCONV, SFEM_EBREAKDOWN, SFEM_ECUDA, SFEM_ETIMEOUT = -4, -5, -6, -7
SFEM_OP_CSR64, SFEM_OP_MF64, SFEM_OP_MF32, SFEM_OP_MF32_F64, SFEM_OP_NS64, SFEM_OP_ES64 = 0, 1, 2, 3, 4, 5
SFEM_SOLVE_PCG64, SFEM_SOLVE_IR32_64, SFEM_SOLVE_FPCG_LEARNED, SFEM_SOLVE_FCG_CNET = 0, 1, 2, 3

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class sfem_opts(ctypes.Structure):
    _fields_ = [("inputs_on_device", ctypes.c_int), ("nrhs", ctypes.c_int),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", ctypes.c_void_p),
                ("reserved", ctypes.c_int * 8)]


class sfem_mesh_info(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "n_nodes", "n_tets", "ndof", "n_faces", "n_interior", "n_boundary", "n_dir", "nrhs", "nnz",
        "n_slivers", "n_bad_tets", "n_bad_faces", "max_tets_per_node")] + [
        (n, ctypes.c_double) for n in ("min_quality", "min_volume", "max_volume", "setup_ms")]


class sfem_csr(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("nnz", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class sfem_solve_opts(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("op64", ctypes.c_int), ("rhs", ctypes.c_int),
                ("u_on_device", ctypes.c_int), ("warm_start", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("tol", ctypes.c_double), ("inner_tol", ctypes.c_double), ("max_outer", ctypes.c_int),
                ("check_every", ctypes.c_int), ("learned", ctypes.c_void_p), ("fp32_vectors", ctypes.c_int),
                ("learned_window", ctypes.c_int), ("learned_pace", ctypes.c_int), ("precond", ctypes.c_int),
                ("bc", ctypes.c_int), ("penalty_exp", ctypes.c_int)]


class sfem_solve_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int), ("outer_iterations", ctypes.c_int),
                ("fallbacks", ctypes.c_int), ("true_relres", ctypes.c_double), ("bnorm", ctypes.c_double),
                ("solve_ms", ctypes.c_double), ("learned_iterations", ctypes.c_int), ("reserved", ctypes.c_int * 3)]


class sfem_batch_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("inner_tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("max_rounds", ctypes.c_int), ("iters_per_launch", ctypes.c_int), ("u_on_device", ctypes.c_int),
                ("warm_start", ctypes.c_int), ("autotune", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("precond", ctypes.c_int), ("patch_nodes", ctypes.c_int), ("reserved", ctypes.c_int * 3)]


class sfem_batch_stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int), ("ctas_per_sm", ctypes.c_int), ("graph", ctypes.c_int),
                ("n_systems", ctypes.c_int), ("total_iterations", ctypes.c_longlong), ("ms", ctypes.c_double),
                ("fallback_systems", ctypes.c_int), ("launch_iterations", ctypes.c_int),
                ("fallback_ms", ctypes.c_float), ("reserved", ctypes.c_int * 1)]


class sfem_coarse_opts(ctypes.Structure):
    _fields_ = [("patch_dims", ctypes.c_int * 3), ("patch_nodes", ctypes.c_int), ("assembly", ctypes.c_int),
                ("factor", ctypes.c_int), ("reserved", ctypes.c_int * 6)]


class sfem_learned_opts(ctypes.Structure):
    _fields_ = [("patch_dims", ctypes.c_int * 3), ("patch_nodes", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("reserved", ctypes.c_int * 6)]


class sfem_cnet_opts(ctypes.Structure):
    _fields_ = [("hidden", ctypes.c_int), ("seed", ctypes.c_uint64), ("reserved", ctypes.c_int * 6)]


class sfem_cnet_run(ctypes.Structure):
    _fields_ = [("window", ctypes.c_int), ("snap_every", ctypes.c_int), ("X", ctypes.c_void_p),
                ("T", ctypes.c_void_p), ("cap_rows", ctypes.c_int64), ("rows", ctypes.c_int64),
                ("reserved", ctypes.c_int * 4)]


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_F = ctypes.c_float
_SIG = {
    "sfem_cnet_create": (ctypes.c_int, [ctypes.POINTER(_P), _P, ctypes.POINTER(sfem_cnet_opts)]),
    "sfem_cnet_destroy": (None, [_P]),
    "sfem_cnet_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(_I64)]),
    "sfem_cnet_set_params": (ctypes.c_int, [_P, _P, _I64]),
    "sfem_cnet_get_params": (ctypes.c_int, [_P, _P, _I64]),
    "sfem_cnet_forward": (ctypes.c_int, [_P, _P, _P, _P, _I64]),
    "sfem_cnet_loss_grad": (ctypes.c_int, [_P, _P, _P, _I64, _P, ctypes.POINTER(ctypes.c_double)]),
    "sfem_cnet_train": (ctypes.c_int, [_P, _P, _P, _I64, _I64, ctypes.c_int, _F, ctypes.c_uint64,
                                       ctypes.POINTER(ctypes.c_double)]),
    "sfem_cnet_correction": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(ctypes.c_double)]),
    "sfem_cnet_random_rows": (ctypes.c_int, [_P, _P, _P, _P, _I64, _I64, ctypes.c_uint64]),
    "sfem_cnet_solve": (ctypes.c_int, [_P, _P, ctypes.POINTER(sfem_solve_opts), _P, ctypes.POINTER(sfem_cnet_run),
                                       ctypes.POINTER(sfem_solve_info)]),
    "sfem_mesh_setup": (ctypes.c_int, [ctypes.POINTER(_P), _P, _I64, _P, _I64, ctypes.c_double, ctypes.c_double,
                                       _P, _P, _I64, _P, _P, _I64, ctypes.POINTER(sfem_opts), _P]),
    "sfem_assemble": (ctypes.c_int, [_P, ctypes.POINTER(sfem_csr)]),
    "sfem_apply": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_int]),
    "sfem_solve": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(sfem_solve_opts), ctypes.POINTER(sfem_solve_info)]),
    "sfem_get_info": (ctypes.c_int, [_P, ctypes.POINTER(sfem_mesh_info)]),
    "sfem_get_geometry": (ctypes.c_int, [_P, _P, _P]),
    "sfem_get_neighbors": (ctypes.c_int, [_P, _P]),
    "sfem_get_faces": (ctypes.c_int, [_P, _P, _P, _P]),
    "sfem_get_rhs": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "sfem_get_diag": (ctypes.c_int, [_P, _P]),
    "sfem_recover": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "sfem_selftest_barrier": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    "sfem_destroy": (None, [_P]),
    "sfem_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "sfem_last_error": (ctypes.c_char_p, []),
    "sfem_version": (ctypes.c_int, []),
    "sfem_time_operator": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "sfem_launch_count": (ctypes.c_int64, []),
    "sfem_gemm_f32": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, ctypes.c_int, _P,
                                     ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "sfem_tile_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.c_int]),
    "sfem_apply_noalloc": (ctypes.c_int, [_P, _P, _P]),
    "sfem_batch_solve": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(_P),
                                        ctypes.POINTER(sfem_batch_opts), ctypes.POINTER(sfem_solve_info),
                                        ctypes.POINTER(sfem_batch_stats)]),
    "sfem_coarse_setup": (ctypes.c_int, [_P, ctypes.POINTER(sfem_coarse_opts)]),
    "sfem_coarse_info": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_double)]),
    "sfem_coarse_apply": (ctypes.c_int, [_P, _P, _P]),
    "sfem_learned_create": (ctypes.c_int, [ctypes.POINTER(_P), _P, ctypes.POINTER(sfem_learned_opts)]),
    "sfem_learned_destroy": (None, [_P]),
    "sfem_learned_info": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "sfem_learned_set_params": (ctypes.c_int, [_P, _P, _I64]),
    "sfem_learned_get_params": (ctypes.c_int, [_P, _P, _I64]),
    "sfem_learned_export": (ctypes.c_int, [_P, _P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "sfem_learned_import": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    "sfem_learned_forward": (ctypes.c_int, [_P, _P, _P, _I64]),
    "sfem_learned_sample": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "sfem_learned_correction": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(ctypes.c_double)]),
    "sfem_learned_collect": (ctypes.c_int, [_P, _P, ctypes.POINTER(sfem_solve_opts), _P, _P, _P, _I64,
                                            ctypes.POINTER(_I64), ctypes.POINTER(sfem_solve_info)]),
    "sfem_learned_loss_grad": (ctypes.c_int, [_P, _P, _P, _I64, _P, ctypes.POINTER(ctypes.c_double)]),
    "sfem_learned_adam": (ctypes.c_int, [_P, _P, _F, _F, _F, _F]),
    "sfem_learned_train": (ctypes.c_int, [_P, _P, _P, _I64, _I64, ctypes.c_int, _F, ctypes.c_uint64,
                                          ctypes.POINTER(ctypes.c_double)]),
}
for _name, (_res, _args) in _SIG.items():
    _fn = getattr(lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


def header_functions() -> list:
    """Names of the functions declared in include/sfem.h."""
    with open(HEADER) as fh:
        src = fh.read()
    return sorted(set(re.findall(r"\b(sfem_[a-z0-9_]+)\s*\(", src)))


class SfemError(RuntimeError):
    def __init__(self, status: int, what: str):
        msg = lib.sfem_last_error().decode() or lib.sfem_strerror(status).decode()
        super().__init__(f"{what}: {lib.sfem_strerror(status).decode()} ({status}): {msg}")
        self.status = status


def _check(status: int, what: str):
    if status != SFEM_OK:
        raise SfemError(status, what)


def _ptr(a):
    """Data pointer of a torch tensor or a C-contiguous numpy array."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("arrays must be C-contiguous")
    return a.ctypes.data


class _DeviceArray:
    """__cuda_array_interface__ view of library-owned device memory."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3}


def _torch():
    import torch
    return torch


class TorchAllocator:
    """Allocator hooks that route the library's device allocations through
    torch's caching allocator on the current device."""

    def __init__(self, device=None):
        torch = _torch()
        self.device = torch.cuda.current_device() if device is None else device

        def _alloc(nbytes, stream, user):
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), self.device, stream or 0))

        def _free(ptr, nbytes, stream, user):
            torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc = ALLOC_FN(_alloc)
        self.free = FREE_FN(_free)


def current_stream_handle() -> int:
    return _torch().cuda.current_stream().cuda_stream


# ---- functions with the ABI's names -----------------------------------------

def sfem_mesh_setup(xyz, tets, E, nu, dir_dofs=None, dir_vals=None, trac_tris=None, trac=None,
                    inputs_on_device=False, stream=None, allocator="torch"):
    """Create a context (see include/sfem.h).  Host inputs are numpy arrays
    (float64 / int32, C-contiguous); device inputs are torch CUDA tensors.
    trac has shape (nrhs, n_tri, 3).  Returns (handle, keepalive) where
    keepalive must outlive the handle (it pins the allocator callbacks)."""
    n_nodes = int(xyz.shape[0])
    n_tets = int(tets.shape[0])
    n_dir = 0 if dir_dofs is None else int(dir_dofs.shape[0])
    n_tri = 0 if trac_tris is None else int(trac_tris.shape[0])
    nrhs = 1 if trac is None else int(trac.shape[0]) if trac.ndim == 3 else 1
    opts = sfem_opts()
    opts.inputs_on_device = 1 if inputs_on_device else 0
    opts.nrhs = nrhs
    keep = [opts]
    if allocator == "torch":
        al = TorchAllocator()
        opts.alloc, opts.free = al.alloc, al.free
        keep.append(al)
    if stream is None:
        stream = current_stream_handle()
    h = _P()
    st = lib.sfem_mesh_setup(ctypes.byref(h), _ptr(xyz), n_nodes, _ptr(tets), n_tets, float(E), float(nu),
                             _ptr(dir_dofs), _ptr(dir_vals), n_dir, _ptr(trac_tris), _ptr(trac), n_tri,
                             ctypes.byref(opts), stream)
    if st != SFEM_OK:
        err = SfemError(st, "sfem_mesh_setup")
        err.handle = h.value
        err.keepalive = keep
        if h.value:
            err.info = sfem_get_info(h.value)
            lib.sfem_destroy(h)
        raise err
    return h.value, keep


def sfem_get_info(h) -> dict:
    info = sfem_mesh_info()
    _check(lib.sfem_get_info(h, ctypes.byref(info)), "sfem_get_info")
    return {k: getattr(info, k) for k, _ in info._fields_ if k != "reserved"}


def sfem_assemble(h):
    """Assemble K; returns torch CUDA views (row_ptr, col, val) of the
    library-owned CSR (valid until sfem_destroy)."""
    torch = _torch()
    csr = sfem_csr()
    _check(lib.sfem_assemble(h, ctypes.byref(csr)), "sfem_assemble")
    rp = torch.as_tensor(_DeviceArray(csr.row_ptr, (csr.n_rows + 1,), "<i8"), device="cuda")
    col = torch.as_tensor(_DeviceArray(csr.col, (csr.nnz,), "<i4"), device="cuda")
    val = torch.as_tensor(_DeviceArray(csr.val, (csr.nnz,), "<f8"), device="cuda")
    return rp, col, val


def sfem_apply(h, u, y, op=SFEM_OP_MF64, nrhs=1):
    """y = A u on device tensors (float64 for CSR64/MF64/MF32_F64, float32 for MF32)."""
    _check(lib.sfem_apply(h, _ptr(u), _ptr(y), int(op), int(nrhs)), "sfem_apply")


def sfem_apply_noalloc(h, u, y):
    """y = A u (FP64 matrix-free, one load case) without any device
    allocation; u, y are float64 CUDA tensors (see include/sfem.h)."""
    _check(lib.sfem_apply_noalloc(h, _ptr(u), _ptr(y)), "sfem_apply_noalloc")


def solve_opts(kind=SFEM_SOLVE_PCG64, op64=SFEM_OP_MF64, rhs=0, tol=1e-8, max_iter=0, inner_tol=0.0,
               max_outer=0, check_every=0, u_on_device=False, warm_start=False, learned=None, fp32_vectors=False,
               learned_window=0, learned_pace=0, precond=0, bc=0, penalty_exp=0):
    o = sfem_solve_opts()
    o.kind, o.op64, o.rhs = int(kind), int(op64), int(rhs)
    o.u_on_device, o.warm_start = int(bool(u_on_device)), int(bool(warm_start))
    o.max_iter, o.tol, o.inner_tol = int(max_iter), float(tol), float(inner_tol)
    o.max_outer, o.check_every = int(max_outer), int(check_every)
    o.learned = learned.h if isinstance(learned, Learned) else learned
    o.fp32_vectors = int(fp32_vectors)
    o.learned_window, o.learned_pace = int(learned_window), int(learned_pace)
    o.precond = int(precond)
    o.bc, o.penalty_exp = int(bc), int(penalty_exp)
    return o


def sfem_solve(h, u, opts: sfem_solve_opts, f_extra=None, check=True) -> dict:
    """Solve into u (numpy float64 host array, or a CUDA tensor when
    opts.u_on_device).  Returns the solve info as a dict."""
    info = sfem_solve_info()
    st = lib.sfem_solve(h, _ptr(f_extra), _ptr(u), ctypes.byref(opts), ctypes.byref(info))
    out = {k: getattr(info, k) for k, _ in info._fields_ if k != "reserved"}
    if check and st not in (SFEM_OK,):
        raise SfemError(st, "sfem_solve")
    return out


def batch_opts(tol=1e-8, inner_tol=0.0, max_iter=0, max_rounds=0, iters_per_launch=0, u_on_device=False,
               warm_start=False, autotune=True, use_graph=True, precond=0, patch_nodes=0):
    o = sfem_batch_opts()
    o.precond, o.patch_nodes = int(precond), int(patch_nodes)
    o.tol, o.inner_tol = float(tol), float(inner_tol)
    o.max_iter, o.max_rounds, o.iters_per_launch = int(max_iter), int(max_rounds), int(iters_per_launch)
    o.u_on_device, o.warm_start = int(bool(u_on_device)), int(bool(warm_start))
    o.autotune, o.use_graph = int(bool(autotune)), int(bool(use_graph))
    return o


def sfem_batch_solve(handles, us, opts: sfem_batch_opts, n_systems: int, check=True):
    """Solve all load cases of all contexts together.  us[i] holds nrhs_i x
    ndof_i float64 values (numpy host arrays, or CUDA tensors with
    opts.u_on_device).  Returns (list of per-system info dicts, stats dict)."""
    n = len(handles)
    harr = (_P * n)(*handles)
    uarr = (_P * n)(*[_ptr(x) for x in us])
    infos = (sfem_solve_info * n_systems)()
    stats = sfem_batch_stats()
    st = lib.sfem_batch_solve(harr, n, uarr, ctypes.byref(opts), infos, ctypes.byref(stats))
    out = [{k: getattr(i, k) for k, _ in i._fields_ if k != "reserved"} for i in infos]
    sd = {k: getattr(stats, k) for k, _ in stats._fields_ if k != "reserved"}
    if check and st != SFEM_OK:
        raise SfemError(st, "sfem_batch_solve")
    return out, sd


def sfem_get_geometry(h, n_tets):
    vol = np.zeros(n_tets)
    grad = np.zeros((n_tets, 4, 3))
    _check(lib.sfem_get_geometry(h, _ptr(vol), _ptr(grad)), "sfem_get_geometry")
    return vol, grad


def sfem_get_neighbors(h, n_tets):
    nbr = np.zeros((n_tets, 4), np.int32)
    _check(lib.sfem_get_neighbors(h, _ptr(nbr)), "sfem_get_neighbors")
    return nbr


def sfem_get_faces(h, n_faces):
    nodes = np.zeros((n_faces, 5), np.int32)
    tets = np.zeros((n_faces, 2), np.int32)
    Vk = np.zeros(n_faces)
    _check(lib.sfem_get_faces(h, _ptr(nodes), _ptr(tets), _ptr(Vk)), "sfem_get_faces")
    return nodes, tets, Vk


def sfem_get_rhs(h, ndof, rhs=0):
    b = np.zeros(ndof)
    _check(lib.sfem_get_rhs(h, _ptr(b), int(rhs)), "sfem_get_rhs")
    return b


def sfem_get_diag(h, ndof):
    d = np.zeros(ndof)
    _check(lib.sfem_get_diag(h, _ptr(d)), "sfem_get_diag")
    return d


def sfem_destroy(h):
    if h:
        lib.sfem_destroy(h)


def sfem_recover(h, u, faces=True, nodes=True) -> dict:
    """Strain and stress recovery (sfem_recover): u a CUDA float64 tensor of
    ndof values.  Returns CUDA float64 tensors: face_strain, face_stress
    (n_faces x 6, library face order) if faces; node_strain, node_stress
    (n_nodes x 6) and node_vm (n_nodes) if nodes.  Voigt order xx, yy, zz,
    yz, zx, xy with engineering shear strains."""
    import torch
    info = sfem_get_info(h)
    nf, nn = info["n_faces"], info["n_nodes"]
    kw = dict(dtype=torch.float64, device=u.device)
    out = {}
    if faces:
        out["face_strain"] = torch.empty((nf, 6), **kw)
        out["face_stress"] = torch.empty((nf, 6), **kw)
    if nodes:
        out["node_strain"] = torch.empty((nn, 6), **kw)
        out["node_stress"] = torch.empty((nn, 6), **kw)
        out["node_vm"] = torch.empty(nn, **kw)
    names = ("face_strain", "face_stress", "node_strain", "node_stress", "node_vm")
    _check(lib.sfem_recover(h, _ptr(u), *[_ptr(out.get(k)) for k in names]), "sfem_recover")
    return out


def sfem_selftest_barrier(h) -> tuple:
    """(status, wait_ms) of the grid barrier's bounded-wait self-test; status
    SFEM_ETIMEOUT is the expected outcome."""
    st, ms = ctypes.c_int(), ctypes.c_double()
    _check(lib.sfem_selftest_barrier(h, ctypes.byref(st), ctypes.byref(ms)), "sfem_selftest_barrier")
    return st.value, ms.value


def sfem_time_operator(h, op=SFEM_OP_MF32, reps=20) -> float:
    """Mean device milliseconds of one raw operator application."""
    ms = ctypes.c_double()
    _check(lib.sfem_time_operator(h, int(op), int(reps), ctypes.byref(ms)), "sfem_time_operator")
    return ms.value


def sfem_launch_count() -> int:
    return int(lib.sfem_launch_count())


def sfem_gemm_f32(A, B, ta=False, tb=False, C=None) -> tuple:
    """(C, ms): C = op(A) op(B) for contiguous FP32 CUDA tensors (op(X) = X^T
    when its flag is set) by the tensor-core training GEMM; ms is its device
    time."""
    M = A.shape[1] if ta else A.shape[0]
    K = A.shape[0] if ta else A.shape[1]
    N = B.shape[0] if tb else B.shape[1]
    if (B.shape[1] if tb else B.shape[0]) != K:
        raise ValueError("inner dimensions differ")
    if C is None:
        import torch
        C = torch.empty((M, N), dtype=torch.float32, device=A.device)
    ms = ctypes.c_double()
    lda, ldb = max(A.shape[1], 1), max(B.shape[1], 1)  # an empty operand (K = 0) is never read
    _check(lib.sfem_gemm_f32(M, N, K, _ptr(A), lda, int(bool(ta)), _ptr(B), ldb, int(bool(tb)),
                             _ptr(C), C.shape[1], ctypes.byref(ms)), "sfem_gemm_f32")
    return C, ms.value


TILE_INFO_KEYS = ("n_tiles", "max_halo", "max_nodes", "slot_stride", "total_halo", "total_nodes",
                  "smem_per_tile_cta", "smem_prefetch_cta", "prefetch_grid", "prefetch_threads")


def sfem_tile_info(h) -> dict:
    """Layout of the FP32 tiled operator and which of its two kernels runs
    (see include/sfem.h)."""
    out = (ctypes.c_int64 * len(TILE_INFO_KEYS))()
    _check(lib.sfem_tile_info(h, out, len(TILE_INFO_KEYS)), "sfem_tile_info")
    return dict(zip(TILE_INFO_KEYS, (int(v) for v in out)))


def sfem_strerror(status: int) -> str:
    return lib.sfem_strerror(status).decode()


# ---- two-level preconditioner ---------------------------------------------------

def sfem_coarse_setup(h, patch_dims=(0, 0, 0), patch_nodes=0, assembly=0, factor=0) -> dict:
    """Build the Galerkin coarse space of context h; returns its info."""
    o = sfem_coarse_opts()
    for a in range(3):
        o.patch_dims[a] = int(patch_dims[a])
    o.patch_nodes, o.assembly, o.factor = int(patch_nodes), int(assembly), int(factor)
    _check(lib.sfem_coarse_setup(h, ctypes.byref(o)), "sfem_coarse_setup")
    return sfem_coarse_info(h)


def sfem_coarse_info(h) -> dict:
    dims = (ctypes.c_int * 3)()
    nc, probes, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(lib.sfem_coarse_info(h, dims, ctypes.byref(nc), ctypes.byref(probes), ctypes.byref(ms)),
           "sfem_coarse_info")
    return {"patch_dims": tuple(dims), "n_coarse": nc.value, "probes": probes.value, "setup_ms": ms.value}


def sfem_coarse_apply(h, r, z):
    """z = D^-1 r + P Pi C Pi^T r (float64 CUDA tensors of ndof entries)."""
    _check(lib.sfem_coarse_apply(h, _ptr(r), _ptr(z)), "sfem_coarse_apply")


# ---- learned coarse correction ------------------------------------------------

N_PARAMS = 84 * 128 + 128 + 128 * 128 + 128 + 128 * 3 + 3


class Learned:
    """An sfem_learned model on the mesh of context `h` (see include/sfem.h).
    Device arrays are torch CUDA tensors (float32 features / targets,
    float64 vectors).  `keepalive` pins the context's allocator callbacks."""

    def __init__(self, h, patch_dims=(0, 0, 0), patch_nodes=0, seed=0, keepalive=None):
        o = sfem_learned_opts()
        for a in range(3):
            o.patch_dims[a] = int(patch_dims[a])
        o.patch_nodes, o.seed = int(patch_nodes), int(seed)
        m = _P()
        _check(lib.sfem_learned_create(ctypes.byref(m), h, ctypes.byref(o)), "sfem_learned_create")
        self.h = m.value
        self._keep = keepalive
        dims = (ctypes.c_int * 3)()
        P, n = ctypes.c_int(), ctypes.c_int()
        _check(lib.sfem_learned_info(self.h, dims, ctypes.byref(P), ctypes.byref(n)), "sfem_learned_info")
        self.patch_dims, self.n_patches, self.n_params = tuple(dims), P.value, n.value

    def set_params(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float32)
        _check(lib.sfem_learned_set_params(self.h, _ptr(th), th.size), "sfem_learned_set_params")

    def get_params(self):
        th = np.zeros(self.n_params, np.float32)
        _check(lib.sfem_learned_get_params(self.h, _ptr(th), th.size), "sfem_learned_get_params")
        return th

    def export_blob(self) -> bytes:
        size = ctypes.c_size_t()
        _check(lib.sfem_learned_export(self.h, None, 0, ctypes.byref(size)), "sfem_learned_export")
        buf = ctypes.create_string_buffer(size.value)
        _check(lib.sfem_learned_export(self.h, buf, size.value, ctypes.byref(size)), "sfem_learned_export")
        return buf.raw

    def import_blob(self, blob: bytes):
        _check(lib.sfem_learned_import(self.h, blob, len(blob)), "sfem_learned_import")

    def forward(self, X, Y):
        _check(lib.sfem_learned_forward(self.h, _ptr(X), _ptr(Y), int(X.shape[0])), "sfem_learned_forward")

    def sample(self, ctx_h, r, X, e=None, T=None):
        _check(lib.sfem_learned_sample(self.h, ctx_h, _ptr(r), _ptr(e), _ptr(X), _ptr(T)), "sfem_learned_sample")

    def correction(self, ctx_h, r, z) -> float:
        a = ctypes.c_double()
        _check(lib.sfem_learned_correction(self.h, ctx_h, _ptr(r), _ptr(z), ctypes.byref(a)),
               "sfem_learned_correction")
        return a.value

    def collect(self, ctx_h, opts, u_star, X, T, row0=0):
        """Snapshots of a flexible-PCG run into X[row0:], T[row0:]; returns
        (rows written, solve info dict)."""
        rows = _I64()
        info = sfem_solve_info()
        cap = int(X.shape[0]) - int(row0)
        Xp = _ptr(X) + 84 * 4 * int(row0)
        Tp = _ptr(T) + 3 * 4 * int(row0)
        _check(lib.sfem_learned_collect(self.h, ctx_h, ctypes.byref(opts), _ptr(u_star), Xp, Tp, cap,
                                        ctypes.byref(rows), ctypes.byref(info)), "sfem_learned_collect")
        return rows.value, {k: getattr(info, k) for k, _ in info._fields_ if k != "reserved"}

    def loss_grad(self, X, T, grad=None) -> float:
        loss = ctypes.c_double()
        _check(lib.sfem_learned_loss_grad(self.h, _ptr(X), _ptr(T), int(X.shape[0]), _ptr(grad),
                                          ctypes.byref(loss)), "sfem_learned_loss_grad")
        return loss.value

    def adam(self, grad=None, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        _check(lib.sfem_learned_adam(self.h, _ptr(grad), lr, b1, b2, eps), "sfem_learned_adam")

    def train(self, X, T, rows=None, batch_rows=4096, epochs=1, lr=1e-3, seed=0) -> float:
        rows = int(X.shape[0]) if rows is None else int(rows)
        loss = ctypes.c_double()
        _check(lib.sfem_learned_train(self.h, _ptr(X), _ptr(T), rows, int(batch_rows), int(epochs), float(lr),
                                      int(seed), ctypes.byref(loss)), "sfem_learned_train")
        return loss.value

    def close(self):
        if self.h:
            lib.sfem_learned_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class CNet:
    """An sfem_cnet model (learned coarse solve) on the coarse space of
    context `h` (see include/sfem.h).  Device arrays are torch CUDA tensors
    (float32 rows of n_coarse values, float64 vectors)."""

    def __init__(self, h, hidden=0, seed=0, keepalive=None):
        o = sfem_cnet_opts()
        o.hidden, o.seed = int(hidden), int(seed)
        m = _P()
        _check(lib.sfem_cnet_create(ctypes.byref(m), h, ctypes.byref(o)), "sfem_cnet_create")
        self.h = m.value
        self._keep = keepalive
        nc, hid, npar = ctypes.c_int(), ctypes.c_int(), _I64()
        _check(lib.sfem_cnet_info(self.h, ctypes.byref(nc), ctypes.byref(hid), ctypes.byref(npar)), "sfem_cnet_info")
        self.n_coarse, self.hidden, self.n_params = nc.value, hid.value, npar.value

    def set_params(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float32)
        _check(lib.sfem_cnet_set_params(self.h, _ptr(th), th.size), "sfem_cnet_set_params")

    def get_params(self):
        th = np.zeros(self.n_params, np.float32)
        _check(lib.sfem_cnet_get_params(self.h, _ptr(th), th.size), "sfem_cnet_get_params")
        return th

    def forward(self, ctx_h, X, Y):
        _check(lib.sfem_cnet_forward(self.h, ctx_h, _ptr(X), _ptr(Y), int(X.shape[0])), "sfem_cnet_forward")

    def loss_grad(self, X, T, grad=None) -> float:
        loss = ctypes.c_double()
        _check(lib.sfem_cnet_loss_grad(self.h, _ptr(X), _ptr(T), int(X.shape[0]), _ptr(grad), ctypes.byref(loss)),
               "sfem_cnet_loss_grad")
        return loss.value

    def train(self, X, T, rows=None, batch_rows=1024, epochs=1, lr=1e-3, seed=0) -> float:
        rows = int(X.shape[0]) if rows is None else int(rows)
        loss = ctypes.c_double()
        _check(lib.sfem_cnet_train(self.h, _ptr(X), _ptr(T), rows, int(batch_rows), int(epochs), float(lr),
                                   int(seed), ctypes.byref(loss)), "sfem_cnet_train")
        return loss.value

    def random_rows(self, ctx_h, X, T, first, count, seed=0):
        _check(lib.sfem_cnet_random_rows(self.h, ctx_h, _ptr(X), _ptr(T), int(first), int(count), int(seed)),
               "sfem_cnet_random_rows")

    def correction(self, ctx_h, r, z) -> float:
        a = ctypes.c_double()
        _check(lib.sfem_cnet_correction(self.h, ctx_h, _ptr(r), _ptr(z), ctypes.byref(a)), "sfem_cnet_correction")
        return a.value

    def close(self):
        if self.h:
            lib.sfem_cnet_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cnet_solve(model, ctx_h, u, opts, window=0, snap_every=0, X=None, T=None, rows=0, check=True):
    """sfem_cnet_solve: u (float64 tensor, device when opts.u_on_device),
    model a CNet or None (Jacobi); appends training rows to X, T (float32
    CUDA tensors of cap x n_coarse) when snap_every > 0.  Returns (info
    dict, rows)."""
    run = sfem_cnet_run()
    run.window, run.snap_every = int(window), int(snap_every)
    run.X, run.T = _ptr(X), _ptr(T)
    run.cap_rows = 0 if X is None else int(X.shape[0])
    run.rows = int(rows)
    info = sfem_solve_info()
    st = lib.sfem_cnet_solve(model.h if model is not None else None, ctx_h, ctypes.byref(opts), _ptr(u),
                             ctypes.byref(run), ctypes.byref(info))
    out = {k: getattr(info, k) for k, _ in info._fields_ if k != "reserved"}
    if check and st != SFEM_OK:
        raise SfemError(st, "sfem_cnet_solve")
    return out, int(run.rows)


# ---- convenience wrapper ----------------------------------------------------

class FsFem:
    """Owns one library context built from an inputs.kuhn_beam.Problem-like
    object (mesh.xyz, mesh.tets, E, nu, dir_dofs, dir_vals, trac_tris, trac)."""

    def __init__(self, problem, on_device=False, stream=None):
        m = problem.mesh
        xyz = np.ascontiguousarray(m.xyz, dtype=np.float64)
        tets = np.ascontiguousarray(m.tets, dtype=np.int32)
        dd = np.ascontiguousarray(problem.dir_dofs, dtype=np.int32)
        dv = np.ascontiguousarray(problem.dir_vals, dtype=np.float64)
        tt = np.ascontiguousarray(problem.trac_tris, dtype=np.int32)
        tr = np.ascontiguousarray(problem.trac, dtype=np.float64)
        if on_device:
            torch = _torch()
            xyz, tets, dd, dv, tt, tr = (torch.from_numpy(a).cuda() for a in (xyz, tets, dd, dv, tt, tr))
        self.inputs = (xyz, tets, dd, dv, tt, tr)
        self.h, self._keep = sfem_mesh_setup(xyz, tets, problem.E, problem.nu, dd, dv, tt, tr,
                                             inputs_on_device=on_device, stream=stream)
        self.info = sfem_get_info(self.h)
        self.ndof = self.info["ndof"]

    def close(self):
        if self.h:
            sfem_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
