"""Thin ctypes binding of libh2gb (argument marshalling only).

Every function keeps the name of its C entry point in ``include/h2gb.h``.
Host arrays are numpy arrays; device pointers are plain integers (for
example ``torch.Tensor.data_ptr()``).  A non-OK status raises ``H2Error``
with the library's message.  Importing this module fails loudly when the
compiled library is missing: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libh2gb.so")

STATUS = {0: "H2_OK", 1: "H2_EINVAL", 2: "H2_ENOMEM", 3: "H2_ECUDA", 4: "H2_ETIMEOUT",
          5: "H2_EDEVICE", 6: "H2_EINTERNAL"}

EXPORTS = [
    "h2_ctx_create", "h2_ctx_destroy", "h2_last_error", "h2_ctx_synchronize",
    "h2_matrix_create", "h2_matrix_free", "h2_matrix_clone",
    "h2_tree_sizes", "h2_tree_clusters", "h2_tree_blocks", "h2_tree_permutation",
    "h2_set_basis", "h2_set_couplings", "h2_set_nearfield", "h2_data_sizes", "h2_get_ranks",
    "h2_get_basis", "h2_get_couplings", "h2_get_nearfield", "h2_get_leaf", "h2_get_transfer",
    "h2_get_coupling",
    "h2_batch_create", "h2_batch_free", "h2_batch_factor_layout", "h2_batch_factor_sizes",
    "h2_batch_execute", "h2_batch_execute_host", "h2_batch_execute_host_compact", "h2_batch_host_bytes",
    "h2_batch_result_size",
    "h2_batch_result_offsets", "h2_batch_task_info", "h2_batch_apply",
    "h2_batch_stats", "h2_batch_set_timing", "h2_batch_phase_stats", "h2_batch_item_info", "h2_batch_item_tile",
    "h2_batch_update_items", "h2_batch_set_mode", "h2_batch_paths", "h2_lowrank_update",
    "h2_lowrank_update_noalloc", "h2_lowrank_update_sequence", "h2_matvec", "h2_block_to_dense",
    "h2_sequence_waves", "h2_check_reciprocal", "h2_debug_fail_allocation",
    "h2_stats", "h2_build_fem", "h2_lr_factor", "h2_lr_factor_many", "h2_lr_solve", "h2_pcg", "h2_lr_error", "h2_mul", "h2_inverse",
    "h2_pcg_inverse", "h2_chol_factor", "h2_chol_solve", "h2_pcg_chol", "h2_chol_error", "h2_chol_factor_many",
]

PHASES = ("base_weights", "rfactor", "norms", "weights", "truncate", "reproject", "exact", "bases")

MODE_AUTO, MODE_EXACT = 0, 1


class H2Error(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (STATUS.get(status, status), message))
        self.status = status


if not os.path.exists(LIB_PATH):
    raise ImportError("libh2gb.so is not built (run paper_1402_5056_gb300.build.build()); "
                      "there is no CPU fallback")
_lib = C.CDLL(LIB_PATH)

_p = C.c_void_p
_i64 = C.c_int64
_i32 = C.c_int32
_int = C.c_int
_dbl = C.c_double
_pp = C.POINTER(C.c_void_p)


def _sig(name, restype, *args):
    f = getattr(_lib, name)
    f.restype = restype
    f.argtypes = list(args)
    return f


_sig("h2_ctx_create", _int, _int, _p, _pp)
_sig("h2_ctx_destroy", None, _p)
_sig("h2_last_error", C.c_char_p, _p)
_sig("h2_ctx_synchronize", _int, _p)
_sig("h2_matrix_create", _int, _p, _p, _i64, _int, _int, _dbl, _dbl, _int, _pp)
_sig("h2_matrix_free", None, _p)
_sig("h2_matrix_clone", _int, _p, _p, _pp)
_sig("h2_tree_sizes", _int, _p, _p, _p, _p, _p, _p, _p)
_sig("h2_tree_clusters", _int, _p, _p, _p, _p, _p, _p, _p, _p)
_sig("h2_tree_blocks", _int, _p, _p, _p, _p, _p)
_sig("h2_tree_permutation", _int, _p, _p)
_sig("h2_set_basis", _int, _p, _p, _int, _p, _p, _p)
_sig("h2_set_couplings", _int, _p, _p, _p)
_sig("h2_set_nearfield", _int, _p, _p, _p)
_sig("h2_data_sizes", _int, _p, _int, _p, _p, _p, _p)
_sig("h2_get_ranks", _int, _p, _int, _p)
_sig("h2_get_basis", _int, _p, _p, _int, _p, _p)
_sig("h2_get_couplings", _int, _p, _p, _p)
_sig("h2_get_nearfield", _int, _p, _p, _p)
_sig("h2_get_leaf", _int, _p, _p, _int, _i64, _p)
_sig("h2_get_transfer", _int, _p, _p, _int, _i64, _p)
_sig("h2_get_coupling", _int, _p, _p, _i64, _p)
_sig("h2_batch_create", _int, _p, _p, _i64, _p, _int, _pp)
_sig("h2_batch_free", None, _p)
_sig("h2_batch_factor_layout", _int, _p, _i64, _p, _p, _p, _p)
_sig("h2_batch_factor_sizes", _int, _p, _p, _p)
_sig("h2_batch_execute", _int, _p, _p, _p, _p, _dbl)
_sig("h2_batch_execute_host", _int, _p, _p, _p, _p, _dbl, _p)
_sig("h2_batch_execute_host_compact", _int, _p, _p, _p, _p, _dbl, _p, _p)
_sig("h2_batch_host_bytes", _int, _p, _p, _p)
_sig("h2_batch_result_size", _int, _p, _p)
_sig("h2_sequence_waves", _int, _p, _i64, _p, _p, _p)
_sig("h2_block_to_dense", _int, _p, _p, _i64, _p, _i64)
_sig("h2_check_reciprocal", _int, _p, _p, _i64, _p)
_sig("h2_debug_fail_allocation", _int, _i64)


class Options(C.Structure):
    """h2_options of include/h2gb.h."""
    _fields_ = [("eps", C.c_double), ("eta", C.c_double), ("leaf_size", C.c_int), ("precision", C.c_int),
                ("trunc_norm", C.c_int), ("weighting", C.c_int), ("max_rank", C.c_int)]


FP64, MIXED_FP32 = 0, 1

_sig("h2_build_fem", _int, _p, _int, _i64, _i64, _p, C.POINTER(Options), _pp)
_sig("h2_lr_factor", _int, _p, _p, C.POINTER(Options), _p)
_sig("h2_lr_solve", _int, _p, _p, _i64, _p, _i64)
_sig("h2_pcg", _int, _p, _p, _p, _p, _p, _dbl, _int, _p, _p)
_sig("h2_lr_error", _int, _p, _p, _p, _p, _int, _p)
_sig("h2_inverse", _int, _p, _p, _p, _p, _p)
_sig("h2_stats", _int, _p, _p, _p)
_sig("h2_lr_factor_many", _int, _p, _p, _i64, _p, _int, _p)
_sig("h2_pcg_inverse", _int, _p, _p, _p, _p, _p, _dbl, _int, _p, _p)
_sig("h2_chol_factor", _int, _p, _p, C.POINTER(Options), _p)
_sig("h2_chol_solve", _int, _p, _p, _i64, _p, _i64)
_sig("h2_pcg_chol", _int, _p, _p, _p, _p, _p, _dbl, _int, _p, _p)
_sig("h2_chol_error", _int, _p, _p, _p, _p, _int, _p)
_sig("h2_chol_factor_many", _int, _p, _p, _i64, _p, _int, _p)
_sig("h2_mul", _int, _p, _dbl, _p, _i64, _p, _i64, _p, _i64, _dbl, _p)
_sig("h2_matvec", _int, _p, _p, _i64, _dbl, _p, _i64, _dbl, _p, _i64)
_sig("h2_lowrank_update_sequence", _int, _p, _p, _i64, _p, _int, _p, _p, _dbl, _p)
_sig("h2_batch_result_offsets", _int, _p, _p, _p)
_sig("h2_batch_task_info", _int, _p, _i64, _p)
_sig("h2_batch_apply", _int, _p, _p, _i64, _p, _p, _p)
_sig("h2_batch_stats", _int, _p, _p, _p, _p, _p, _p)
_sig("h2_batch_set_timing", _int, _p, _int)
_sig("h2_batch_set_mode", _int, _p, _int)
_sig("h2_batch_paths", _int, _p, _p, _p)
_sig("h2_batch_phase_stats", _int, _p, _p, _int, _p, _p, _p)
_sig("h2_batch_item_info", _int, _p, _i64, _p)
_sig("h2_batch_item_tile", _int, _p, _p, _i64, _int, _p)
_sig("h2_batch_update_items", _int, _p, _i64, _p, _p)
_sig("h2_lowrank_update", _int, _p, _p, _i64, _int, _p, _i64, _p, _i64, _dbl)
_sig("h2_lowrank_update_noalloc", _int, _p, _p, _i64, _int, _p, _i64, _p, _i64, _dbl)


def _check(status: int, ctx=None):
    if status != 0:
        msg = _lib.h2_last_error(ctx)
        raise H2Error(status, msg.decode() if msg else "")


def _ptr(a):
    """Host pointer of a contiguous numpy array (or None)."""
    if a is None:
        return None
    assert isinstance(a, np.ndarray) and (a.flags.c_contiguous or a.flags.f_contiguous)
    return a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).ravel(order="A"))


# ------------------------------------------------------------------ context
def h2_ctx_create(device: int = 0, stream: int | None = None):
    out = C.c_void_p()
    st = _lib.h2_ctx_create(int(device), C.c_void_p(stream) if stream else None, C.byref(out))
    _check(st)
    return out.value


def h2_ctx_destroy(ctx):
    _lib.h2_ctx_destroy(ctx)


def h2_last_error(ctx) -> str:
    m = _lib.h2_last_error(ctx)
    return m.decode() if m else ""


def h2_ctx_synchronize(ctx):
    _check(_lib.h2_ctx_synchronize(ctx), ctx)


# ------------------------------------------------------------------- matrix
def h2_matrix_create(ctx, points, leaf_size: int, eta: float, pad: float = 0.0, kcap: int = 16):
    """``ctx`` may be None: structure only (trees, no device storage)."""
    pts = np.ascontiguousarray(points, dtype=np.float64)
    n, dim = pts.shape
    out = C.c_void_p()
    _check(_lib.h2_matrix_create(ctx, _ptr(pts), n, dim, int(leaf_size), float(eta), float(pad),
                                 int(kcap), C.byref(out)), ctx)
    return out.value


def h2_matrix_free(Z):
    _lib.h2_matrix_free(Z)


def h2_matrix_clone(ctx, Z):
    out = C.c_void_p()
    _check(_lib.h2_matrix_clone(ctx, Z, C.byref(out)), ctx)
    return out.value


def h2_tree_sizes(Z) -> dict:
    v = [C.c_int64() for _ in range(5)]
    d = C.c_int()
    _check(_lib.h2_tree_sizes(Z, *[C.byref(x) for x in v], C.byref(d)))
    return dict(n=v[0].value, n_clusters=v[1].value, n_blocks=v[2].value, n_admissible=v[3].value,
                n_inadmissible=v[4].value, depth=d.value)


def h2_tree_clusters(Z) -> dict:
    nc = h2_tree_sizes(Z)["n_clusters"]
    off = np.zeros(nc, np.int64)
    size = np.zeros(nc, np.int64)
    a32 = [np.zeros(nc, np.int32) for _ in range(5)]
    _check(_lib.h2_tree_clusters(Z, _ptr(off), _ptr(size), *[_ptr(a) for a in a32]))
    return dict(offset=off, size=size, father=a32[0], son0=a32[1], son1=a32[2], level=a32[3],
                subtree=a32[4])


def h2_tree_blocks(Z) -> dict:
    nb = h2_tree_sizes(Z)["n_blocks"]
    a = [np.zeros(nb, np.int32) for _ in range(4)]
    _check(_lib.h2_tree_blocks(Z, *[_ptr(x) for x in a]))
    return dict(row=a[0], col=a[1], kind=a[2], father=a[3])


def h2_tree_permutation(Z) -> np.ndarray:
    n = h2_tree_sizes(Z)["n"]
    p = np.zeros(n, np.int64)
    _check(_lib.h2_tree_permutation(Z, _ptr(p)))
    return p


# --------------------------------------------------------------------- data
def h2_set_basis(ctx, Z, side: int, ranks, leaf_data, transfer_data):
    r = np.ascontiguousarray(ranks, dtype=np.int32)
    _check(_lib.h2_set_basis(ctx, Z, int(side), _ptr(r), _ptr(_f64(leaf_data)), _ptr(_f64(transfer_data))), ctx)


def h2_set_couplings(ctx, Z, data):
    _check(_lib.h2_set_couplings(ctx, Z, _ptr(_f64(data))), ctx)


def h2_set_nearfield(ctx, Z, data):
    _check(_lib.h2_set_nearfield(ctx, Z, _ptr(_f64(data))), ctx)


def h2_data_sizes(Z, side: int) -> dict:
    v = [C.c_int64() for _ in range(4)]
    _check(_lib.h2_data_sizes(Z, int(side), *[C.byref(x) for x in v]))
    return dict(leaf=v[0].value, transfer=v[1].value, coupling=v[2].value, nearfield=v[3].value)


def h2_get_ranks(Z, side: int) -> np.ndarray:
    r = np.zeros(h2_tree_sizes(Z)["n_clusters"], np.int32)
    _check(_lib.h2_get_ranks(Z, int(side), _ptr(r)))
    return r


def h2_get_basis(ctx, Z, side: int):
    s = h2_data_sizes(Z, side)
    leaf = np.zeros(s["leaf"])
    tr = np.zeros(s["transfer"])
    _check(_lib.h2_get_basis(ctx, Z, int(side), _ptr(leaf), _ptr(tr)), ctx)
    return h2_get_ranks(Z, side), leaf, tr


def h2_get_couplings(ctx, Z) -> np.ndarray:
    out = np.zeros(h2_data_sizes(Z, 0)["coupling"])
    _check(_lib.h2_get_couplings(ctx, Z, _ptr(out)), ctx)
    return out


def h2_get_nearfield(ctx, Z) -> np.ndarray:
    out = np.zeros(h2_data_sizes(Z, 0)["nearfield"])
    _check(_lib.h2_get_nearfield(ctx, Z, _ptr(out)), ctx)
    return out


def h2_get_leaf(ctx, Z, side: int, cluster: int, rows: int, rank: int) -> np.ndarray:
    out = np.zeros(rows * rank)
    _check(_lib.h2_get_leaf(ctx, Z, int(side), int(cluster), _ptr(out)), ctx)
    return out.reshape((rows, rank), order="F")


def h2_get_transfer(ctx, Z, side: int, cluster: int, rows: int, cols: int) -> np.ndarray:
    out = np.zeros(rows * cols)
    _check(_lib.h2_get_transfer(ctx, Z, int(side), int(cluster), _ptr(out)), ctx)
    return out.reshape((rows, cols), order="F")


def h2_get_coupling(ctx, Z, block: int, rows: int, cols: int) -> np.ndarray:
    out = np.zeros(rows * cols)
    _check(_lib.h2_get_coupling(ctx, Z, int(block), _ptr(out)), ctx)
    return out.reshape((rows, cols), order="F")


# ------------------------------------------------------------------ updates
def h2_batch_create(ctx, Z, blocks, u: int):
    """``ctx`` may be None: host-only plan (no device buffers)."""
    b = np.ascontiguousarray(blocks, dtype=np.int64)
    out = C.c_void_p()
    _check(_lib.h2_batch_create(ctx, Z, len(b), _ptr(b), int(u), C.byref(out)), ctx)
    return out.value


def h2_batch_free(P):
    _lib.h2_batch_free(P)


def h2_batch_factor_layout(P, j: int):
    v = [C.c_int64() for _ in range(4)]
    _check(_lib.h2_batch_factor_layout(P, int(j), *[C.byref(x) for x in v]))
    return tuple(x.value for x in v)   # rows_A, off_A, rows_B, off_B


def h2_batch_factor_sizes(P):
    a, b = C.c_int64(), C.c_int64()
    _check(_lib.h2_batch_factor_sizes(P, C.byref(a), C.byref(b)))
    return a.value, b.value


def h2_batch_execute(ctx, P, A_dev: int, B_dev: int, eps: float):
    _check(_lib.h2_batch_execute(ctx, P, C.c_void_p(A_dev), C.c_void_p(B_dev), float(eps)), ctx)


def h2_batch_result_size(P) -> int:
    n = C.c_int64()
    _check(_lib.h2_batch_result_size(P, C.byref(n)))
    return n.value


def _host_buffer(a, n, dtype, what):
    """A caller's output array: contiguous, of the dtype, at least n long."""
    if not (isinstance(a, np.ndarray) and a.dtype == dtype and a.flags.c_contiguous and a.size >= n):
        raise ValueError("%s must be a contiguous %s array of at least %d entries" % (what, np.dtype(dtype), n))
    return a


def h2_batch_execute_host(ctx, P, A_host, B_host, eps: float, result=None):
    if result is None:
        result = np.zeros(h2_batch_result_size(P))
    _host_buffer(result, h2_batch_result_size(P), np.float64, "result")
    _check(_lib.h2_batch_execute_host(ctx, P, _ptr(_f64(A_host)), _ptr(_f64(B_host)), float(eps),
                                      _ptr(result)), ctx)
    return result


def h2_batch_execute_host_compact(ctx, P, A_host, B_host, eps: float, result=None, copied=None):
    """Compact host result: (result, copied); copied[b] = 1 where block task
    b keeps its coupling padded with zeros (its piece is then unspecified
    when `result` is page-locked)."""
    n_tasks = h2_batch_stats(None, P, flops=False)["block_tasks"]
    if result is None:
        result = np.zeros(h2_batch_result_size(P))
    if copied is None:
        copied = np.zeros(n_tasks, np.int8)
    _host_buffer(result, h2_batch_result_size(P), np.float64, "result")
    _host_buffer(copied, n_tasks, np.int8, "copied")
    _check(_lib.h2_batch_execute_host_compact(ctx, P, _ptr(_f64(A_host)), _ptr(_f64(B_host)), float(eps),
                                              _ptr(result), _ptr(copied)), ctx)
    return result, copied


def h2_batch_host_bytes(P):
    """(h2d, d2h): bytes the last host execution copied each way."""
    a, c = C.c_int64(), C.c_int64()
    _check(_lib.h2_batch_host_bytes(P, C.byref(a), C.byref(c)))
    return a.value, c.value


def h2_batch_apply(ctx, P, j: int, A_dev: int, B_dev: int, dst):
    _check(_lib.h2_batch_apply(ctx, P, int(j), C.c_void_p(A_dev), C.c_void_p(B_dev), dst), ctx)


def h2_batch_stats(ctx, P, flops: bool = True) -> dict:
    a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
    f = C.c_double()
    _check(_lib.h2_batch_stats(ctx, P, C.byref(a), C.byref(b), C.byref(c), C.byref(f) if flops else None), ctx)
    return dict(cluster_tasks=a.value, block_tasks=b.value, launches=c.value, flops=f.value if flops else None)


def h2_batch_set_timing(P, on):
    """on: False/0 off, True/1 phase events, 2 phase events with every phase
    on the context's stream (no overlap between phases)."""
    _check(_lib.h2_batch_set_timing(P, 2 if on == 2 else (1 if on else 0)))


def h2_batch_set_mode(P, mode: int):
    """MODE_AUTO: certified Gram path, exact path for the updates it does not
    cover; MODE_EXACT: exact path for every update."""
    _check(_lib.h2_batch_set_mode(P, int(mode)))


def h2_batch_paths(ctx, P, count: int) -> np.ndarray:
    """Per update of the last execution: 1 if the exact path computed it."""
    out = np.zeros(max(count, 1), dtype=np.int32)
    _check(_lib.h2_batch_paths(ctx, P, out.ctypes.data))
    return out[:count]


def h2_batch_phase_stats(ctx, P, phase: int, flops: bool = True) -> dict:
    n = C.c_int64()
    ms = C.c_double()
    f = C.c_double()
    _check(_lib.h2_batch_phase_stats(ctx, P, int(phase), C.byref(n), C.byref(ms),
                                     C.byref(f) if flops else None), ctx)
    return dict(launches=n.value, ms=ms.value, flops=f.value if flops else None)


def h2_batch_result_offsets(P):
    """(item_off, task_off): offsets of the pieces of the host result."""
    st = h2_batch_stats(None, P, flops=False)
    io = np.zeros(st["cluster_tasks"], np.int64)
    to = np.zeros(st["block_tasks"], np.int64)
    _check(_lib.h2_batch_result_offsets(P, _ptr(io), _ptr(to)))
    return io, to


def h2_batch_task_info(P, task: int) -> dict:
    a = np.zeros(6, np.int32)
    _check(_lib.h2_batch_task_info(P, int(task), _ptr(a)))
    return dict(update=int(a[0]), block=int(a[1]), row_item=int(a[2]), col_item=int(a[3]), kt=int(a[4]),
                ls=int(a[5]))


def h2_batch_item_info(P, item: int) -> dict:
    a = np.zeros(8, np.int32)
    _check(_lib.h2_batch_item_info(P, int(item), _ptr(a)))
    return dict(update=int(a[0]), side=int(a[1]), cluster=int(a[2]), k=int(a[3]), rank=int(a[4]),
                flags=int(a[5]))


def h2_batch_item_tile(ctx, P, item: int, which: int) -> np.ndarray:
    out = np.zeros(32 * 32)
    _check(_lib.h2_batch_item_tile(ctx, P, int(item), int(which), _ptr(out)), ctx)
    return out.reshape((32, 32), order="F")


def h2_batch_update_items(P, j: int):
    a, c = C.c_int64(), C.c_int64()
    _check(_lib.h2_batch_update_items(P, int(j), C.byref(a), C.byref(c)))
    return a.value, c.value


def h2_lowrank_update(ctx, Z, block: int, u: int, A_dev: int, lda: int, B_dev: int, ldb: int, eps: float):
    _check(_lib.h2_lowrank_update(ctx, Z, int(block), int(u), C.c_void_p(A_dev), int(lda),
                                  C.c_void_p(B_dev), int(ldb), float(eps)), ctx)


def h2_lowrank_update_noalloc(ctx, Z, block: int, u: int, A_dev: int, lda: int, B_dev: int, ldb: int,
                              eps: float):
    """Same update as h2_lowrank_update with no device allocation (fixed
    library-internal scratch; see include/h2gb.h for the limits)."""
    _check(_lib.h2_lowrank_update_noalloc(ctx, Z, int(block), int(u), C.c_void_p(A_dev), int(lda),
                                          C.c_void_p(B_dev), int(ldb), float(eps)), ctx)


def h2_lowrank_update_sequence(ctx, Z, blocks, u: int, A_dev: int, B_dev: int, eps: float) -> int:
    """Updates applied in order (waves of non-conflicting updates); A_dev,
    B_dev: device pointers to the factors concatenated in order.  Returns
    the number of waves."""
    bl = np.ascontiguousarray(blocks, dtype=np.int64)
    w = C.c_int64()
    _check(_lib.h2_lowrank_update_sequence(ctx, Z, len(bl), _ptr(bl), int(u), C.c_void_p(A_dev), C.c_void_p(B_dev),
                                           float(eps), C.byref(w)), ctx)
    return w.value


def h2_matvec(ctx, Z, nrhs: int, alpha: float, X_dev: int, ldx: int, beta: float, Y_dev: int, ldy: int):
    """Y <- alpha Z X + beta Y on the context's stream (device pointers,
    column-major, rows in tree order)."""
    _check(_lib.h2_matvec(ctx, Z, int(nrhs), float(alpha), C.c_void_p(X_dev), int(ldx), float(beta),
                          C.c_void_p(Y_dev), int(ldy)), ctx)


def h2_block_to_dense(ctx, Z, block: int, out_dev: int, ld: int):
    """Z|_{t x s} of a block-tree node into a device array (column-major)."""
    _check(_lib.h2_block_to_dense(ctx, Z, int(block), C.c_void_p(out_dev), int(ld)), ctx)


def h2_sequence_waves(Z, blocks):
    """Waves of h2_lowrank_update_sequence for these blocks (host only)."""
    bl = np.ascontiguousarray(blocks, dtype=np.int64)
    wave = np.zeros(len(bl), np.int32)
    n = C.c_int64()
    _check(_lib.h2_sequence_waves(Z, len(bl), _ptr(bl), _ptr(wave), C.byref(n)))
    return wave, n.value


def h2_check_reciprocal(ctx, d_dev: int, n: int, out_dev: int):
    """The pivot reciprocal of the factorisation kernels, element by element
    (device arrays of n doubles)."""
    _check(_lib.h2_check_reciprocal(ctx, C.c_void_p(d_dev), int(n), C.c_void_p(out_dev)), ctx)


def h2_debug_fail_allocation(n: int):
    """Make the n-th device allocation of the library from now on fail with
    H2_ENOMEM (n = 0: off).  A test hook for the error paths."""
    _check(_lib.h2_debug_fail_allocation(int(n)))


def options(eps=1e-4, eta=2.0, leaf_size=32, precision=0, max_rank=0):
    return Options(float(eps), float(eta), int(leaf_size), int(precision), 0, 0, int(max_rank))


def h2_build_fem(ctx, dim: int, cells: int, checker: int, sigma, opt):
    """P1 FEM stiffness matrix on the unit square/cube as an H^2 matrix."""
    sg = np.ascontiguousarray(sigma, dtype=np.float64)
    assert sg.size == checker ** dim
    out = C.c_void_p()
    _check(_lib.h2_build_fem(ctx, int(dim), int(cells), int(checker), sg.ctypes.data, C.byref(opt), C.byref(out)),
           ctx)
    return out


def h2_lr_factor(ctx, Z, opt):
    """In-place H^2-LR; returns counts, the largest rank and the wall time by activity."""
    st = np.zeros(15, dtype=np.int64)
    _check(_lib.h2_lr_factor(ctx, Z, C.byref(opt), st.ctypes.data), ctx)
    return {"updates": int(st[0]), "products": int(st[1]), "max_rank": int(st[2]),
            "seconds": {"updates": st[3] / 1e6, "terms": st[4] / 1e6, "temporaries": st[5] / 1e6,
                        "solves": st[6] / 1e6, "leaf_lu": st[7] / 1e6},
            "update_seconds": {"plan": st[8] / 1e6, "enqueue": st[9] / 1e6, "wait": st[10] / 1e6,
                               "total": st[11] / 1e6},
            "temporaries": {"count": int(st[13]), "columns": int(st[14]), "wait_seconds": st[12] / 1e6}}


def h2_lr_factor_many(ctx, Zs, opt, threads: int = 0):
    """h2_lr_factor of independent matrices side by side; returns per-matrix
    statistics (updates, products, max_rank)."""
    arr = (C.c_void_p * len(Zs))(*Zs)
    st = np.zeros(3 * max(len(Zs), 1), np.int64)
    _check(_lib.h2_lr_factor_many(ctx, arr, len(Zs), C.byref(opt), int(threads), _ptr(st)), ctx)
    return [{"updates": int(st[3 * i]), "products": int(st[3 * i + 1]), "max_rank": int(st[3 * i + 2])}
            for i in range(len(Zs))]


def h2_chol_factor_many(ctx, Zs, opt, threads: int = 0):
    """h2_chol_factor of independent matrices side by side; returns per-matrix
    statistics (updates, products, max_rank)."""
    arr = (C.c_void_p * len(Zs))(*Zs)
    st = np.zeros(3 * max(len(Zs), 1), np.int64)
    _check(_lib.h2_chol_factor_many(ctx, arr, len(Zs), C.byref(opt), int(threads), _ptr(st)), ctx)
    return [{"updates": int(st[3 * i]), "products": int(st[3 * i + 1]), "max_rank": int(st[3 * i + 2])}
            for i in range(len(Zs))]


def h2_lr_solve(ctx, LR, nrhs: int, X_dev: int, ldx: int):
    _check(_lib.h2_lr_solve(ctx, LR, int(nrhs), C.c_void_p(X_dev), int(ldx)), ctx)


def h2_pcg(ctx, A, LR, b_dev: int, x_dev: int, tol: float, maxit: int):
    """Preconditioned CG; returns (iterations, relative residual)."""
    it = C.c_int(0)
    rr = C.c_double(0.0)
    _check(_lib.h2_pcg(ctx, A, LR, C.c_void_p(b_dev), C.c_void_p(x_dev), float(tol), int(maxit), C.byref(it),
                       C.byref(rr)), ctx)
    return it.value, rr.value


def h2_lr_error(ctx, A, LR, v_dev: int, iters: int):
    err = C.c_double(0.0)
    _check(_lib.h2_lr_error(ctx, A, LR, C.c_void_p(v_dev), int(iters), C.byref(err)), ctx)
    return err.value


def h2_stats(Z):
    """Size and rank statistics of an H^2 matrix (host data only)."""
    out = np.zeros(12, np.int64)
    depth = int(h2_tree_sizes(Z)["depth"])
    lv = np.zeros(depth + 1, np.int32)
    _check(_lib.h2_stats(Z, _ptr(out), _ptr(lv)))
    keys = ("n", "n_clusters", "n_blocks", "n_admissible", "n_inadmissible", "depth", "rank_capacity",
            "max_rank_rows", "max_rank_cols", "device_bytes", "value_bytes", "rank_sum_rows")
    d = {k: int(v) for k, v in zip(keys, out)}
    d["max_rank_per_level"] = [int(x) for x in lv]
    return d


def h2_inverse(ctx, A, opt):
    """Approximate inverse of A (block Gauss elimination); A is consumed.
    Returns (C, stats) with C a new matrix handle."""
    out = C.c_void_p()
    st = np.zeros(3, np.int64)
    _check(_lib.h2_inverse(ctx, A, C.byref(opt), C.byref(out), _ptr(st)), ctx)
    return out.value, {"updates": int(st[0]), "products": int(st[1]), "max_rank": int(st[2])}


def h2_pcg_inverse(ctx, A, Cinv, b_dev: int, x_dev: int, tol: float, maxit: int):
    it = C.c_int()
    rr = C.c_double()
    _check(_lib.h2_pcg_inverse(ctx, A, Cinv, C.c_void_p(b_dev), C.c_void_p(x_dev), float(tol), int(maxit),
                               C.byref(it), C.byref(rr)), ctx)
    return it.value, rr.value


def h2_chol_factor(ctx, Z, opt):
    """In-place approximate Cholesky factorisation; returns counts and the largest rank."""
    st = np.zeros(3, dtype=np.int64)
    _check(_lib.h2_chol_factor(ctx, Z, C.byref(opt), st.ctypes.data), ctx)
    return {"updates": int(st[0]), "products": int(st[1]), "max_rank": int(st[2])}


def h2_chol_solve(ctx, F, nrhs: int, X_dev: int, ldx: int):
    _check(_lib.h2_chol_solve(ctx, F, int(nrhs), C.c_void_p(X_dev), int(ldx)), ctx)


def h2_pcg_chol(ctx, A, F, b_dev: int, x_dev: int, tol: float, maxit: int):
    """CG preconditioned by the Cholesky factor; returns (iterations, relative residual)."""
    it = C.c_int()
    rr = C.c_double()
    _check(_lib.h2_pcg_chol(ctx, A, F, C.c_void_p(b_dev), C.c_void_p(x_dev), float(tol), int(maxit),
                            C.byref(it), C.byref(rr)), ctx)
    return it.value, rr.value


def h2_chol_error(ctx, A, F, v_dev: int, iters: int):
    err = C.c_double(0.0)
    _check(_lib.h2_chol_error(ctx, A, F, C.c_void_p(v_dev), int(iters), C.byref(err)), ctx)
    return err.value


def h2_mul(ctx, alpha: float, X, bx: int, Y, by: int, Z, bz: int, eps: float) -> int:
    """Z|_bz += alpha X|_bx Y|_by (three matrices on one block tree); returns
    the number of local updates."""
    n = C.c_int64(0)
    _check(_lib.h2_mul(ctx, float(alpha), X, int(bx), Y, int(by), Z, int(bz), float(eps), C.byref(n)), ctx)
    return n.value

