"""ctypes binding of the C ABI declared in include/dgwave.h.

Argument marshalling only: every computation runs in libdgwave.so.  The
functions keep the C names; pointers are plain integers (device pointers
from ``tensor.data_ptr()``, streams from ``torch.cuda.Stream.cuda_stream``).
Loading fails loudly when the library has not been built.
"""
import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
# DGWAVE_CHECKED=1: the checked build (device-side index checks that report
# DG_ERR_INDEX instead of faulting), built by build(checked=True)
CHECKED = os.environ.get("DGWAVE_CHECKED", "") == "1"
LIB_PATH = os.path.join(_PKG, "libdgwave_checked.so" if CHECKED else "libdgwave.so")

DG_OK = 0
DG_ERR_ARG = 1
DG_ERR_MESH_DEGENERATE = 2
DG_ERR_MESH_NONCONFORMING = 3
DG_ERR_ORDER = 4
DG_ERR_CUDA = 5
DG_ERR_OOM = 6
DG_ERR_NONFINITE = 7
DG_ERR_NO_DEVICE = 8
DG_ERR_TIMEOUT = 9
DG_ERR_IO = 10
DG_ERR_INDEX = 11
DG_CKPT_HOST = 1
DG_FP64 = 0
DG_FP32 = 1
DG_SETUP_HOST_ONLY = 1
DG_SETUP_SIMT = 2
DG_SETUP_TC_TF32 = 4
DG_SETUP_TC_BF16 = 8
DG_SETUP_TC_BF16X3 = 16
DG_SETUP_TC = 32
DG_SETUP_ELEMENT_THREADS = 64
DG_STATIC_SCRATCH_BYTES = 32 * 1024 * 1024
DG_BATCH_NO_GRAPH = 1
DG_BATCH_NO_ADAPT = 2
DG_BATCH_SPLIT = 4
DG_BATCH_MODE_CONCURRENT, DG_BATCH_MODE_SPLIT = 0, 1
DG_KERNEL_TENSOR_CORES, DG_KERNEL_CUDA_CORES, DG_KERNEL_ELEMENT_THREADS = 0, 1, 2
DG_SERVER_SEQUENTIAL = 1
DG_REQUEST_QUEUED, DG_REQUEST_RUNNING, DG_REQUEST_DONE, DG_REQUEST_FAILED = 0, 1, 2, 3
DG_REQUEST_CANCELLED = 4
DG_N_MAX = 7

_STATUS_NAMES = {
    0: "DG_OK", 1: "DG_ERR_ARG", 2: "DG_ERR_MESH_DEGENERATE", 3: "DG_ERR_MESH_NONCONFORMING",
    4: "DG_ERR_ORDER", 5: "DG_ERR_CUDA", 6: "DG_ERR_OOM", 7: "DG_ERR_NONFINITE",
    8: "DG_ERR_NO_DEVICE", 9: "DG_ERR_TIMEOUT", 10: "DG_ERR_IO", 11: "DG_ERR_INDEX",
}

c_void_p = ctypes.c_void_p


class dg_request_info(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int32), ("N", ctypes.c_int32),
                ("K", ctypes.c_int64), ("nsteps", ctypes.c_int64), ("dt", ctypes.c_double),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double), ("t_retired", ctypes.c_double)]


class dg_point_source(ctypes.Structure):
    _fields_ = [("x", ctypes.c_double), ("y", ctypes.c_double), ("f", ctypes.c_double),
                ("t0", ctypes.c_double), ("amplitude", ctypes.c_double)]
c_i32 = ctypes.c_int32
c_i64 = ctypes.c_int64
c_dbl = ctypes.c_double
P = ctypes.POINTER

# (name, restype, argtypes) of every exported entry point
SIGNATURES = [
    ("dg_mesh_create", c_i32, [c_void_p, c_void_p, c_i64, c_void_p, c_i64, P(c_void_p)]),
    ("dg_mesh_info", c_i32, [c_void_p, P(c_i64), P(c_i64), P(c_i64)]),
    ("dg_mesh_connectivity", c_i32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    ("dg_mesh_destroy", None, [c_void_p]),
    ("dg_operator_setup", c_i32, [c_void_p, c_i32, c_i32, c_i32, P(c_void_p)]),
    ("dg_operator_setup_media", c_i32, [c_void_p, c_i32, c_void_p, c_i32, c_i32, P(c_void_p)]),
    ("dg_operator_set_alpha", c_i32, [c_void_p, c_dbl]),
    ("dg_operator_set_face_pairs", c_i32, [c_void_p, c_i32]),
    ("dg_operator_set_source", c_i32, [c_void_p, c_void_p]),
    ("dg_operator_set_block_elems", c_i32, [c_void_p, c_i32]),
    ("dg_operator_kernel", c_i32, [c_void_p, P(c_i32), P(c_i32)]),
    ("dg_operator_tune", c_i32, [c_void_p, c_i32, c_void_p, P(c_dbl), P(c_dbl)]),
    ("dg_get_info", c_i32, [c_void_p, P(c_i32), P(c_i32), P(c_i64), P(c_i64)]),
    ("dg_get_nodes", c_i32, [c_void_p, c_void_p, c_void_p]),
    ("dg_get_reference", c_i32, [c_void_p] + [c_void_p] * 6),
    ("dg_get_geometry", c_i32, [c_void_p] + [c_void_p] * 8),
    ("dg_get_maps", c_i32, [c_void_p, c_void_p, c_void_p]),
    ("dg_cfl_dt", c_i32, [c_void_p, c_dbl, P(c_dbl)]),
    ("dg_lsrk_coefficients", c_i32, [c_void_p, c_void_p, c_void_p]),
    ("dg_op_destroy", None, [c_void_p]),
    ("dg_rhs", c_i32, [c_void_p, c_void_p, c_void_p, c_dbl, c_void_p]),
    ("dg_step", c_i32, [c_void_p, c_void_p, c_void_p, c_dbl, c_dbl, c_i32, c_void_p]),
    ("dg_solve", c_i32, [c_void_p, c_void_p, c_void_p, c_dbl, c_dbl, P(c_i32), P(c_dbl), c_void_p]),
    ("dg_step_static", c_i32, [c_void_p, c_void_p, c_void_p, c_dbl, c_dbl, c_i32, c_void_p]),
    ("dg_step_host", c_i32, [c_void_p, c_void_p, c_void_p, c_void_p, c_dbl, c_dbl, c_i32, c_void_p]),
    ("dg_step_host_jobs", c_i32, [c_void_p, c_i32, c_void_p, c_void_p, c_dbl, c_dbl, c_i32,
                                  c_void_p]),
    ("dg_step_host_jobs_work_bytes", c_i64, [c_void_p]),
    ("dg_check_finite", c_i32, [c_void_p, c_void_p, c_void_p]),
    ("dg_sync_check", c_i32, [c_void_p, c_void_p]),
    ("dg_launch_count", c_i64, [c_void_p]),
    ("dg_test_wait_timeout", c_i32, [c_void_p, c_void_p]),
    ("dg_test_fail_alloc", c_i32, [c_i32]),
    ("dg_test_fail_alloc_pending", c_i32, []),
    ("dg_checkpoint_save", c_i32, [c_void_p, c_void_p, c_i64, c_i32, c_dbl, c_i64, ctypes.c_char_p]),
    ("dg_checkpoint_load", c_i32, [c_void_p, ctypes.c_char_p, c_void_p, c_i64, c_i32, P(c_dbl),
                                   P(c_i64)]),
    ("dg_batch_create", c_i32, [c_void_p, c_i32, P(c_void_p)]),
    ("dg_batch_destroy", None, [c_void_p]),
    ("dg_batch_add", c_i32, [c_void_p, c_void_p, c_dbl, c_void_p, c_void_p, P(c_i32)]),
    ("dg_batch_remove", c_i32, [c_void_p, c_i32]),
    ("dg_batch_info", c_i32, [c_void_p, c_i32, P(c_i32), P(c_i64), P(c_dbl), P(c_i64)]),
    ("dg_batch_set_fields", c_i32, [c_void_p, c_i32, c_void_p, c_i64, c_void_p]),
    ("dg_batch_get_fields", c_i32, [c_void_p, c_i32, c_void_p, c_i64, c_void_p]),
    ("dg_batch_step", c_i32, [c_void_p, c_i32, c_void_p]),
    ("dg_batch_tune", c_i32, [c_void_p, c_i32, c_void_p]),
    ("dg_batch_plan", c_i32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    ("dg_batch_plan_ctas", c_i32, [c_void_p, c_void_p, c_i32, c_void_p]),
    ("dg_batch_launch_mode", c_i32, [c_void_p, P(c_i32), P(c_dbl), P(c_dbl)]),
    ("dg_batch_set_block_elems", c_i32, [c_void_p, c_i32, c_i32]),
    ("dg_batch_block_elems", c_i32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    ("dg_batch_sync_check", c_i32, [c_void_p, c_void_p]),
    ("dg_batch_launch_count", c_i64, [c_void_p]),
    ("dg_server_clock", c_dbl, []),
    ("dg_server_create", c_i32, [c_void_p, c_i32, P(c_void_p)]),
    ("dg_server_destroy", None, [c_void_p]),
    ("dg_server_submit", c_i32, [c_void_p, c_void_p, c_dbl, c_void_p, c_void_p, c_void_p, P(c_i64)]),
    ("dg_server_wait", c_i32, [c_void_p, c_i64, c_dbl, c_void_p]),
    ("dg_server_info", c_i32, [c_void_p, c_i64, c_void_p]),
    ("dg_server_release", c_i32, [c_void_p, c_i64]),
    ("dg_server_cancel", c_i32, [c_void_p, c_i64]),
    ("dg_server_set_work_limit", c_i32, [c_void_p, c_i64]),
    ("dg_server_stats", c_i32, [c_void_p, P(c_i64), P(c_i64), P(c_i64), P(c_i64)]),
    ("dg_partition_create", c_i32, [c_void_p, c_i32, P(c_void_p)]),
    ("dg_partition_destroy", None, [c_void_p]),
    ("dg_partition_info", c_i32, [c_void_p, c_i32, P(c_i64), P(c_i64), P(c_i32), P(c_i32),
                                  P(c_i64), P(c_i64)]),
    ("dg_partition_elements", c_i32, [c_void_p, c_i32, c_void_p]),
    ("dg_partition_ghosts", c_i32, [c_void_p, c_i32, c_void_p]),
    ("dg_partition_conn", c_i32, [c_void_p, c_i32, c_void_p]),
    ("dg_partition_exchange_plan", c_i32, [c_void_p, c_i32] + [c_void_p] * 6),
    ("dg_partition_set_fields", c_i32, [c_void_p, c_void_p, c_i64, c_void_p]),
    ("dg_partition_get_fields", c_i32, [c_void_p, c_void_p, c_i64, c_void_p]),
    ("dg_partition_exchange", c_i32, [c_void_p, c_void_p]),
    ("dg_partition_step", c_i32, [c_void_p, c_dbl, c_i32, c_void_p]),
    ("dg_partition_sync_check", c_i32, [c_void_p, c_void_p]),
    ("dg_last_error", ctypes.c_char_p, []),
]

_lib = None


class DGError(RuntimeError):
    def __init__(self, status, where, message):
        self.status = status
        super().__init__("%s failed with %s: %s" % (where, _STATUS_NAMES.get(status, status), message))


def load(path=None):
    """Load libdgwave.so (once) and declare its signatures."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError("libdgwave.so not built (expected at %s); run __graft_entry__.build()" % p)
    lib = ctypes.CDLL(p)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def check(status, where):
    if status != DG_OK:
        msg = load().dg_last_error()
        raise DGError(status, where, msg.decode() if msg else "")
    return status
