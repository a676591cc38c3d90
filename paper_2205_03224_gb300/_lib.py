"""ctypes binding of libgemslr.so (the C ABI declared in include/gemslr.h).

Argument marshalling only: every step of the solve runs in the library's CUDA
kernels.  Device arrays are torch CUDA tensors; the current torch stream is
passed to the library.  If the shared library has not been built this module
raises instead of falling back to anything else.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgemslr.so")
MAX_LEVELS = 16

P = ctypes.c_void_p
i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double


class CSR(ctypes.Structure):
    _fields_ = [("n", i64), ("rowptr", P), ("colind", P), ("val", P)]


class Partition(ctypes.Structure):
    _fields_ = [("nlev", i32), ("perm", P), ("level_ptr", P), ("nblk", P), ("block_ptr", P)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class Options(ctypes.Structure):
    _fields_ = [("ilu_kind", i32), ("ilut_tau", f64), ("ilut_lfil", i32), ("rank", i32 * MAX_LEVELS),
                ("precision", i32), ("arnoldi_tol", f64), ("arnoldi_max_cycles", i32),
                ("strict_pivots", i32), ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN), ("alloc_ctx", P),
                ("lowrank_method", i32), ("lowrank_power", i32), ("shift", f64)]


class Mat(ctypes.Structure):
    _fields_ = [("nrows", i64), ("ncols", i64), ("rowptr", P), ("colind", P), ("val", P)]


class LevelFactors(ctypes.Structure):
    _fields_ = [("L", Mat), ("U", Mat), ("E", Mat), ("F", Mat), ("k", i32), ("W", P), ("H", P),
                ("L_im", P), ("U_im", P), ("W_im", P), ("H_im", P)]


class Factors(ctypes.Structure):
    _fields_ = [("nlev", i32), ("levels", ctypes.POINTER(LevelFactors)), ("last_L", Mat), ("last_U", Mat),
                ("last_L_im", P), ("last_U_im", P)]


class LearnedOpts(ctypes.Structure):
    _fields_ = [("channels", i32), ("npairs", i32), ("epochs", i32), ("batch", i32), ("lr", f64),
                ("seed", ctypes.c_uint64)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("restart", i32), ("maxit", i32), ("rtol", f64), ("ortho", i32)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", i32), ("restarts", i32), ("converged", i32), ("reorth", i32),
                ("rel_res_est", f64), ("rel_res_true", f64), ("t_total_ms", f64)]


STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_PARTITION", 3: "ERR_ZERO_PIVOT", 4: "ERR_NOT_CONVERGED",
          5: "ERR_NAN", 6: "ERR_TIMEOUT", 7: "ERR_CUDA", 8: "ERR_NOMEM", 9: "ERR_UNSUPPORTED"}

EXPORTED = [
    "gemslr_default_options", "gemslr_partition_geometric", "gemslr_local_order", "gemslr_setup", "gemslr_setup_from_factors",
    "gemslr_factor_sizes", "gemslr_export_factors", "gemslr_apply", "gemslr_fgmres_solve",
    "gemslr_get_stats", "gemslr_last_error", "gemslr_destroy", "gemslr_kernel_launches",
    "gemslr_profile_enable", "gemslr_profile_reset", "gemslr_profile_read",
    "gemslr_setup_batch", "gemslr_setup_batch_from_factors", "gemslr_batch_apply", "gemslr_batch_fgmres_solve", "gemslr_batch_stats",
    "gemslr_batch_last_error", "gemslr_batch_destroy",
    "gemslr_learned_train", "gemslr_learned_enable", "gemslr_learned_info", "gemslr_learned_params",
    "gemslr_learned_loss_grad", "gemslr_apply_static", "gemslr_selftest_wait", "gemslr_set_inner_steps",
    "gemslr_save_factors", "gemslr_load_factors", "gemslr_zapply", "gemslr_zfgmres_solve",
]

_lib = None


class GemslrError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def load():
    """Load libgemslr.so (raises if it is missing: build it with __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing; run paper_2205_03224_gb300.build.build() first")
    L = ctypes.CDLL(LIB_PATH)
    L.gemslr_default_options.argtypes = [ctypes.POINTER(Options)]
    L.gemslr_default_options.restype = None
    L.gemslr_partition_geometric.argtypes = [ctypes.POINTER(CSR), P, i32, i32, i32, P, P, P, P]
    L.gemslr_local_order.argtypes = [i64, P, ctypes.POINTER(Partition), i32, P]
    L.gemslr_setup.argtypes = [ctypes.POINTER(CSR), ctypes.POINTER(Partition), ctypes.POINTER(Options), ctypes.POINTER(P)]
    L.gemslr_setup_from_factors.argtypes = [ctypes.POINTER(CSR), ctypes.POINTER(Partition),
                                            ctypes.POINTER(Factors), ctypes.POINTER(Options), ctypes.POINTER(P)]
    L.gemslr_factor_sizes.argtypes = [P, P, i64]
    L.gemslr_export_factors.argtypes = [P, ctypes.POINTER(Factors)]
    L.gemslr_apply.argtypes = [P, P, P, i32, P]
    L.gemslr_fgmres_solve.argtypes = [P, P, P, i32, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo), P]
    L.gemslr_zapply.argtypes = [P, P, P, i32, P]
    L.gemslr_zfgmres_solve.argtypes = [P, P, P, i32, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo), P]
    L.gemslr_get_stats.argtypes = [P, P, i32]
    L.gemslr_last_error.restype = ctypes.c_char_p
    L.gemslr_last_error.argtypes = []
    L.gemslr_destroy.argtypes = [P]
    L.gemslr_destroy.restype = None
    L.gemslr_kernel_launches.restype = ctypes.c_uint64
    L.gemslr_kernel_launches.argtypes = []
    L.gemslr_profile_enable.argtypes = [i32]
    L.gemslr_profile_enable.restype = None
    L.gemslr_profile_reset.argtypes = []
    L.gemslr_profile_reset.restype = None
    L.gemslr_profile_read.argtypes = [ctypes.c_char_p, ctypes.c_size_t, P, P, i32]
    L.gemslr_profile_read.restype = i32
    L.gemslr_setup_batch.argtypes = [i32, ctypes.POINTER(CSR), ctypes.POINTER(Partition), ctypes.POINTER(Options),
                                     ctypes.POINTER(P)]
    L.gemslr_setup_batch_from_factors.argtypes = [i32, ctypes.POINTER(CSR), ctypes.POINTER(Partition),
                                                  ctypes.POINTER(Factors), ctypes.POINTER(Options),
                                                  ctypes.POINTER(P)]
    L.gemslr_batch_apply.argtypes = [P, P, P, i32, P]
    L.gemslr_batch_fgmres_solve.argtypes = [P, P, P, i32, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo), P]
    L.gemslr_batch_stats.argtypes = [P, P, i32]
    L.gemslr_batch_last_error.restype = ctypes.c_char_p
    L.gemslr_batch_last_error.argtypes = []
    L.gemslr_learned_train.argtypes = [P, P, ctypes.POINTER(LearnedOpts), P]
    L.gemslr_learned_enable.argtypes = [P, i32]
    L.gemslr_set_inner_steps.argtypes = [P, i32]
    L.gemslr_save_factors.argtypes = [P, ctypes.c_char_p]
    L.gemslr_load_factors.argtypes = [P, P, ctypes.c_char_p, P, P]
    L.gemslr_learned_info.argtypes = [P, P]
    L.gemslr_learned_params.argtypes = [P, i32, P, i64]
    L.gemslr_learned_loss_grad.argtypes = [P, i32, P, P, P, P]
    L.gemslr_apply_static.argtypes = [P, P, P, P]
    L.gemslr_selftest_wait.argtypes = [i64]
    L.gemslr_batch_destroy.argtypes = [P]
    L.gemslr_batch_destroy.restype = None
    for name in EXPORTED:
        fn = getattr(L, name)
        if name not in ("gemslr_default_options", "gemslr_last_error", "gemslr_destroy", "gemslr_kernel_launches",
                        "gemslr_profile_enable", "gemslr_profile_reset", "gemslr_profile_read",
                        "gemslr_batch_last_error", "gemslr_batch_destroy"):
            fn.restype = ctypes.c_int
    _lib = L
    return L


def check(status, batch=False):
    if status != 0:
        lib = load()
        msg = lib.gemslr_batch_last_error() if batch else lib.gemslr_last_error()
        raise GemslrError(status, msg.decode())


def ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def csr_struct(A, keep):
    """gemslr_csr for an object with rowptr/colind/val (or scipy csr); ``keep`` holds the arrays."""
    if hasattr(A, "indptr"):
        rp, ci, v = A.indptr, A.indices, A.data
    else:
        rp, ci, v = A.rowptr, A.colind, A.val
    rp = np.ascontiguousarray(rp, dtype=np.int64)
    ci = np.ascontiguousarray(ci, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.float64)
    keep.extend([rp, ci, v])
    return CSR(len(rp) - 1, ptr(rp), ptr(ci), ptr(v))


def partition_struct(part, keep):
    arrs = [np.ascontiguousarray(part["perm"], dtype=np.int32),
            np.ascontiguousarray(part["level_ptr"], dtype=np.int64),
            np.ascontiguousarray(part["nblk"], dtype=np.int32),
            np.ascontiguousarray(part["block_ptr"], dtype=np.int64)]
    keep.extend(arrs)
    return Partition(len(arrs[2]), *[ptr(a) for a in arrs])


def mat_struct(M, keep):
    """gemslr_mat from a scipy CSR matrix (real)."""
    return mat_struct_z(M, keep)[0]


def mat_struct_z(M, keep):
    """(gemslr_mat, imaginary parts or None) from a scipy CSR matrix, real or complex."""
    import scipy.sparse as sp
    M = sp.csr_matrix(M)
    M.sort_indices()
    rp = np.ascontiguousarray(M.indptr, dtype=np.int64)
    ci = np.ascontiguousarray(M.indices, dtype=np.int32)
    v = np.ascontiguousarray(M.data.real, dtype=np.float64)
    keep.extend([rp, ci, v])
    im = None
    if np.iscomplexobj(M.data):
        vi = np.ascontiguousarray(M.data.imag, dtype=np.float64)
        keep.append(vi)
        im = ptr(vi)
    return Mat(M.shape[0], M.shape[1], ptr(rp), ptr(ci), ptr(v)), im


def kernel_launches():
    return int(load().gemslr_kernel_launches())


def selftest_wait(cycles):
    """Status name of gemslr_selftest_wait (\"ERR_TIMEOUT\" is the expected outcome)."""
    return STATUS.get(load().gemslr_selftest_wait(int(cycles)), "?")


def profile_enable(on=True):
    load().gemslr_profile_enable(1 if on else 0)


def profile_reset():
    load().gemslr_profile_reset()


def profile_read():
    """{kernel name: (total ms, launches)} accumulated since the last reset."""
    lib = load()
    buf = ctypes.create_string_buffer(1 << 16)
    ms = np.zeros(256)
    cnt = np.zeros(256, dtype=np.int64)
    k = lib.gemslr_profile_read(buf, len(buf), ptr(ms), ptr(cnt), 256)
    names = buf.value.decode().split("\n")[:k]
    return {nm: (float(ms[i]), int(cnt[i])) for i, nm in enumerate(names)}
