"""GB300-native nodal discontinuous Galerkin solver for the 2D TM Maxwell
system (Kloeckner, Warburton, Hesthaven, "Solving Wave Equations on
Unstructured Geometries"): right-hand side + LSRK(5,4) in hand-written CUDA
for sm_103a behind the C ABI of include/dgwave.h.

This module is the thin Python binding: functions named like the C entry
points marshal numpy arrays / torch tensors into pointers and call the
library.  PyTorch supplies device memory and streams only.  There is no CPU
fallback: every call raises if libdgwave.so is missing or the call fails.
"""
import ctypes

import numpy as np

from . import _lib
from ._lib import (  # noqa: F401
    DG_FP32,
    DG_FP64,
    DG_N_MAX,
    DG_SETUP_HOST_ONLY,
    DGError,
)

__all__ = [
    "dg_mesh_create", "dg_mesh_info", "dg_mesh_connectivity", "dg_mesh_destroy",
    "dg_operator_setup", "dg_operator_setup_media", "dg_operator_set_alpha",
    "dg_operator_set_face_pairs", "dg_operator_set_source", "dg_operator_set_block_elems",
    "dg_operator_kernel", "dg_operator_tune",
    "dg_get_info", "dg_get_nodes", "dg_get_reference",
    "dg_get_geometry", "dg_get_maps", "dg_cfl_dt", "dg_lsrk_coefficients",
    "dg_op_destroy", "dg_rhs", "dg_step", "dg_step_static", "dg_solve", "dg_step_host",
    "dg_step_host_jobs", "dg_step_host_jobs_work_bytes", "dg_test_fail_alloc",
    "dg_test_fail_alloc_pending",
    "dg_check_finite", "dg_sync_check", "dg_launch_count", "dg_last_error", "dg_test_wait_timeout",
    "dg_checkpoint_save", "dg_checkpoint_load",
    "dg_batch_create", "dg_batch_destroy", "dg_batch_add", "dg_batch_remove", "dg_batch_info",
    "dg_batch_set_fields", "dg_batch_get_fields", "dg_batch_step", "dg_batch_tune",
    "dg_batch_plan", "dg_batch_plan_ctas", "dg_batch_launch_mode", "dg_batch_set_block_elems",
    "dg_batch_block_elems", "dg_batch_sync_check",
    "dg_batch_launch_count",
    "dg_server_clock", "dg_server_create", "dg_server_destroy", "dg_server_submit",
    "dg_server_wait", "dg_server_info", "dg_server_release", "dg_server_cancel", "dg_server_stats",
    "dg_server_set_work_limit",
    "dg_partition_create", "dg_partition_destroy", "dg_partition_info", "dg_partition_elements",
    "dg_partition_ghosts", "dg_partition_conn", "dg_partition_exchange_plan",
    "dg_partition_set_fields", "dg_partition_get_fields", "dg_partition_exchange",
    "dg_partition_step", "dg_partition_sync_check",
    "Solver", "Batch", "Server", "Partition", "DGError", "DG_FP32", "DG_FP64",
]


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t):
    return ctypes.c_void_p(t.data_ptr())


# ------------------------------------------------------------------ mesh
def dg_mesh_create(VX, VY, EToV):
    VX = np.ascontiguousarray(VX, dtype=np.float64)
    VY = np.ascontiguousarray(VY, dtype=np.float64)
    E = np.ascontiguousarray(EToV, dtype=np.int32)
    h = ctypes.c_void_p()
    _lib.check(_lib.load().dg_mesh_create(_ptr(VX), _ptr(VY), VX.size, _ptr(E), E.shape[0],
                                          ctypes.byref(h)), "dg_mesh_create")
    return h.value


def dg_mesh_info(mesh):
    K, nf, nb = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _lib.check(_lib.load().dg_mesh_info(mesh, ctypes.byref(K), ctypes.byref(nf), ctypes.byref(nb)),
               "dg_mesh_info")
    return K.value, nf.value, nb.value


def dg_mesh_connectivity(mesh):
    K = dg_mesh_info(mesh)[0]
    EToE = np.empty((K, 3), np.int32)
    EToF = np.empty((K, 3), np.int32)
    EToV = np.empty((K, 3), np.int32)
    _lib.check(_lib.load().dg_mesh_connectivity(mesh, _ptr(EToE), _ptr(EToF), _ptr(EToV)),
               "dg_mesh_connectivity")
    return EToE, EToF, EToV


def dg_mesh_destroy(mesh):
    if mesh:
        _lib.load().dg_mesh_destroy(mesh)


# -------------------------------------------------------------- operator
def dg_operator_setup(mesh, N, precision=DG_FP32, flags=0):
    h = ctypes.c_void_p()
    _lib.check(_lib.load().dg_operator_setup(mesh, N, precision, flags, ctypes.byref(h)),
               "dg_operator_setup")
    return h.value


def dg_operator_setup_media(mesh, N, eps, precision=DG_FP32, flags=0):
    e = np.ascontiguousarray(eps, dtype=np.float64)
    h = ctypes.c_void_p()
    _lib.check(_lib.load().dg_operator_setup_media(mesh, N, _ptr(e), precision, flags,
                                                   ctypes.byref(h)), "dg_operator_setup_media")
    return h.value


def dg_operator_set_alpha(op, alpha):
    _lib.check(_lib.load().dg_operator_set_alpha(op, alpha), "dg_operator_set_alpha")


def dg_operator_set_face_pairs(op, enable):
    _lib.check(_lib.load().dg_operator_set_face_pairs(op, int(bool(enable))),
               "dg_operator_set_face_pairs")


def dg_operator_set_source(op, source):
    """source: None (remove) or (x, y, f, t0, amplitude) of a Ricker point source."""
    src = None if source is None else ctypes.byref(_lib.dg_point_source(*[float(v) for v in source]))
    _lib.check(_lib.load().dg_operator_set_source(op, src), "dg_operator_set_source")


def dg_operator_set_block_elems(op, elems):
    _lib.check(_lib.load().dg_operator_set_block_elems(op, int(elems)),
               "dg_operator_set_block_elems")


def dg_operator_kernel(op):
    """("tensor cores" | "cuda cores" | "element threads", elements per block)."""
    k, e = ctypes.c_int32(), ctypes.c_int32()
    _lib.check(_lib.load().dg_operator_kernel(op, ctypes.byref(k), ctypes.byref(e)),
               "dg_operator_kernel")
    names = {_lib.DG_KERNEL_CUDA_CORES: "cuda cores",
             _lib.DG_KERNEL_ELEMENT_THREADS: "element threads"}
    return (names.get(k.value, "tensor cores"), e.value)


def dg_operator_tune(op, reps=5, stream=None):
    """Returns (ms per launch on the tensor cores, on the CUDA cores); -1
    for operators whose kernel the set-up fixed."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _lib.check(_lib.load().dg_operator_tune(op, reps, _stream_handle(stream), ctypes.byref(a),
                                            ctypes.byref(b)), "dg_operator_tune")
    return a.value, b.value


def dg_get_info(op):
    Np, Nfp = ctypes.c_int32(), ctypes.c_int32()
    K, fs = ctypes.c_int64(), ctypes.c_int64()
    _lib.check(_lib.load().dg_get_info(op, ctypes.byref(Np), ctypes.byref(Nfp), ctypes.byref(K),
                                       ctypes.byref(fs)), "dg_get_info")
    return Np.value, Nfp.value, K.value, fs.value


def dg_get_nodes(op):
    Np, _, K, _ = dg_get_info(op)
    x = np.empty((K, Np))
    y = np.empty((K, Np))
    _lib.check(_lib.load().dg_get_nodes(op, _ptr(x), _ptr(y)), "dg_get_nodes")
    return x, y


def dg_get_reference(op):
    Np, Nfp, _, _ = dg_get_info(op)
    out = {"r": np.empty(Np), "s": np.empty(Np), "Dr": np.empty((Np, Np)),
           "Ds": np.empty((Np, Np)), "LIFT": np.empty((Np, 3 * Nfp)),
           "Fmask": np.empty((3, Nfp), np.int32)}
    _lib.check(_lib.load().dg_get_reference(op, *[_ptr(out[k]) for k in
                                                  ("r", "s", "Dr", "Ds", "LIFT", "Fmask")]),
               "dg_get_reference")
    return out


def dg_get_geometry(op):
    _, _, K, _ = dg_get_info(op)
    names = ("rx", "ry", "sx", "sy", "J", "nx", "ny", "Fscale")
    out = {n: np.empty(K) for n in names[:5]}
    out.update({n: np.empty((K, 3)) for n in names[5:]})
    _lib.check(_lib.load().dg_get_geometry(op, *[_ptr(out[n]) for n in names]), "dg_get_geometry")
    return out


def dg_get_maps(op):
    _, Nfp, K, _ = dg_get_info(op)
    vM = np.empty((K, 3 * Nfp), np.int64)
    vP = np.empty((K, 3 * Nfp), np.int64)
    _lib.check(_lib.load().dg_get_maps(op, _ptr(vM), _ptr(vP)), "dg_get_maps")
    return vM, vP


def dg_cfl_dt(op, cfl=1.0):
    dt = ctypes.c_double()
    _lib.check(_lib.load().dg_cfl_dt(op, cfl, ctypes.byref(dt)), "dg_cfl_dt")
    return dt.value


def dg_lsrk_coefficients():
    a, b, c = np.empty(5), np.empty(5), np.empty(5)
    _lib.check(_lib.load().dg_lsrk_coefficients(_ptr(a), _ptr(b), _ptr(c)), "dg_lsrk_coefficients")
    return a, b, c


def dg_op_destroy(op):
    if op:
        _lib.load().dg_op_destroy(op)


# -------------------------------------------------------------- hot path
def dg_rhs(op, q, rhs, t=0.0, stream=None):
    _lib.check(_lib.load().dg_rhs(op, _dptr(q), _dptr(rhs), t, _stream_handle(stream)), "dg_rhs")


def dg_step(op, q, res, t0, dt, nsteps, stream=None):
    _lib.check(_lib.load().dg_step(op, _dptr(q), _dptr(res), t0, dt, nsteps,
                                   _stream_handle(stream)), "dg_step")


def dg_step_static(op, q, res, t0, dt, nsteps, stream=None):
    """dg_step with the library's fixed per-device scratch array instead of
    the operator's own buffer (allocates nothing)."""
    _lib.check(_lib.load().dg_step_static(op, _dptr(q), _dptr(res), t0, dt, nsteps,
                                          _stream_handle(stream)), "dg_step_static")


def dg_solve(op, q, res, T, dt=0.0, stream=None):
    n = ctypes.c_int32()
    t = ctypes.c_double()
    _lib.check(_lib.load().dg_solve(op, _dptr(q), _dptr(res), T, dt, ctypes.byref(n),
                                    ctypes.byref(t), _stream_handle(stream)), "dg_solve")
    return n.value, t.value


def dg_step_host(op, h_q, d_q, d_res, t0, dt, nsteps, stream=None):
    """h_q: host tensor (pinned recommended) or contiguous numpy array of
    3 * field_stride values."""
    hp = ctypes.c_void_p(h_q.data_ptr()) if hasattr(h_q, "data_ptr") else _ptr(h_q)
    _lib.check(_lib.load().dg_step_host(op, hp, _dptr(d_q), _dptr(d_res), t0, dt, nsteps,
                                        _stream_handle(stream)), "dg_step_host")


def dg_step_host_jobs_work_bytes(op):
    return int(_lib.load().dg_step_host_jobs_work_bytes(op))


def dg_step_host_jobs(op, h_qs, d_work, t0, dt, nsteps, stream=None):
    """h_qs: list of host tensors (pinned) or contiguous numpy arrays of
    3 * field_stride values each, one per job; d_work: device tensor of at
    least dg_step_host_jobs_work_bytes(op) bytes."""
    ptrs = (ctypes.c_void_p * max(len(h_qs), 1))(
        *[h.data_ptr() if hasattr(h, "data_ptr") else h.ctypes.data for h in h_qs])
    _lib.check(_lib.load().dg_step_host_jobs(op, len(h_qs), ptrs, _dptr(d_work), t0, dt, nsteps,
                                             _stream_handle(stream)), "dg_step_host_jobs")


def dg_test_fail_alloc(n):
    _lib.check(_lib.load().dg_test_fail_alloc(int(n)), "dg_test_fail_alloc")


def dg_test_fail_alloc_pending():
    return int(_lib.load().dg_test_fail_alloc_pending())


def dg_check_finite(op, q, stream=None):
    _lib.check(_lib.load().dg_check_finite(op, _dptr(q), _stream_handle(stream)), "dg_check_finite")


def dg_sync_check(op, stream=None):
    _lib.check(_lib.load().dg_sync_check(op, _stream_handle(stream)), "dg_sync_check")


def dg_test_wait_timeout(op, stream=None):
    _lib.check(_lib.load().dg_test_wait_timeout(op, _stream_handle(stream)), "dg_test_wait_timeout")


def dg_checkpoint_save(op, q, q_stride, t, step, path):
    """q: device tensor (field stride q_stride) or host numpy array / CPU
    tensor (DG_CKPT_HOST)."""
    host = not (hasattr(q, "is_cuda") and q.is_cuda)
    _lib.check(_lib.load().dg_checkpoint_save(op, _buf_ptr(q), q_stride,
                                              _lib.DG_CKPT_HOST if host else 0, t, step,
                                              str(path).encode()), "dg_checkpoint_save")


def dg_checkpoint_load(op, path, q, q_stride):
    """Fills q (device tensor or host array); returns (t, step)."""
    host = not (hasattr(q, "is_cuda") and q.is_cuda)
    t, step = ctypes.c_double(), ctypes.c_int64()
    _lib.check(_lib.load().dg_checkpoint_load(op, str(path).encode(), _buf_ptr(q), q_stride,
                                              _lib.DG_CKPT_HOST if host else 0, ctypes.byref(t),
                                              ctypes.byref(step)), "dg_checkpoint_load")
    return t.value, step.value


def dg_launch_count(op):
    return int(_lib.load().dg_launch_count(op))


def dg_last_error():
    m = _lib.load().dg_last_error()
    return m.decode() if m else ""


# --------------------------------------------------------------- batches
def dg_batch_create(capacity, flags=0):
    """capacity: 7 element counts (orders 1..7)."""
    c = np.ascontiguousarray(capacity, dtype=np.int64)
    if c.size != DG_N_MAX:
        raise ValueError("capacity needs %d entries" % DG_N_MAX)
    h = ctypes.c_void_p()
    _lib.check(_lib.load().dg_batch_create(_ptr(c), flags, ctypes.byref(h)), "dg_batch_create")
    return h.value


def dg_batch_destroy(batch):
    if batch:
        _lib.load().dg_batch_destroy(batch)


def dg_batch_add(batch, op, dt=0.0, source=None, stream=None):
    """source: None or (x, y, f, t0, amplitude) of a Ricker point source."""
    slot = ctypes.c_int32()
    src = None
    if source is not None:
        src = ctypes.byref(_lib.dg_point_source(*[float(v) for v in source]))
    _lib.check(_lib.load().dg_batch_add(batch, op, dt, src, _stream_handle(stream),
                                        ctypes.byref(slot)), "dg_batch_add")
    return slot.value


def dg_batch_remove(batch, slot):
    _lib.check(_lib.load().dg_batch_remove(batch, slot), "dg_batch_remove")


def dg_batch_info(batch, slot):
    N, K, dt, fs = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_int64()
    _lib.check(_lib.load().dg_batch_info(batch, slot, ctypes.byref(N), ctypes.byref(K),
                                         ctypes.byref(dt), ctypes.byref(fs)), "dg_batch_info")
    return N.value, K.value, dt.value, fs.value


def _buf_ptr(a):
    return ctypes.c_void_p(a.data_ptr()) if hasattr(a, "data_ptr") else _ptr(a)


def dg_batch_set_fields(batch, slot, src, stride, stream=None):
    """src: float32 host array / tensor or device tensor; field f at f * stride."""
    _lib.check(_lib.load().dg_batch_set_fields(batch, slot, _buf_ptr(src), stride,
                                               _stream_handle(stream)), "dg_batch_set_fields")


def dg_batch_get_fields(batch, slot, dst, stride, stream=None):
    _lib.check(_lib.load().dg_batch_get_fields(batch, slot, _buf_ptr(dst), stride,
                                               _stream_handle(stream)), "dg_batch_get_fields")


def dg_batch_step(batch, nsteps, stream=None):
    _lib.check(_lib.load().dg_batch_step(batch, nsteps, _stream_handle(stream)), "dg_batch_step")


def dg_batch_tune(batch, reps=5, stream=None):
    _lib.check(_lib.load().dg_batch_tune(batch, reps, _stream_handle(stream)), "dg_batch_tune")


def dg_batch_plan(batch):
    cta = np.zeros(DG_N_MAX, np.int32)
    nb = np.zeros(DG_N_MAX, np.int64)
    cost = np.zeros(DG_N_MAX, np.float64)
    _lib.check(_lib.load().dg_batch_plan(batch, _ptr(cta), _ptr(nb), _ptr(cost)), "dg_batch_plan")
    return cta, nb, cost


def dg_batch_plan_ctas(nblocks, cost, num_ctas):
    nb = np.ascontiguousarray(nblocks, dtype=np.int64)
    c = np.ascontiguousarray(cost, dtype=np.float64)
    out = np.zeros(DG_N_MAX, np.int32)
    _lib.check(_lib.load().dg_batch_plan_ctas(_ptr(nb), _ptr(c), num_ctas, _ptr(out)),
               "dg_batch_plan_ctas")
    return out


def dg_batch_launch_mode(batch):
    """("concurrent" | "split", tuned split ms, tuned concurrent ms)."""
    m, a, c = ctypes.c_int32(), ctypes.c_double(), ctypes.c_double()
    _lib.check(_lib.load().dg_batch_launch_mode(batch, ctypes.byref(m), ctypes.byref(a),
                                                ctypes.byref(c)), "dg_batch_launch_mode")
    return ("split" if m.value == _lib.DG_BATCH_MODE_SPLIT else "concurrent", a.value, c.value)


def dg_batch_set_block_elems(batch, N, elems):
    _lib.check(_lib.load().dg_batch_set_block_elems(batch, int(N), int(elems)),
               "dg_batch_set_block_elems")


def dg_batch_block_elems(batch):
    """(elements per block, tuned ms default, tuned ms alternative), 7 each."""
    e = np.zeros(DG_N_MAX, np.int32)
    md = np.zeros(DG_N_MAX, np.float64)
    ma = np.zeros(DG_N_MAX, np.float64)
    _lib.check(_lib.load().dg_batch_block_elems(batch, _ptr(e), _ptr(md), _ptr(ma)),
               "dg_batch_block_elems")
    return e, md, ma


def dg_batch_sync_check(batch, stream=None):
    _lib.check(_lib.load().dg_batch_sync_check(batch, _stream_handle(stream)), "dg_batch_sync_check")


def dg_batch_launch_count(batch):
    return int(_lib.load().dg_batch_launch_count(batch))


# --------------------------------------------------------------- serving
def dg_server_clock():
    return float(_lib.load().dg_server_clock())


def dg_server_create(capacity, sequential=False):
    c = np.ascontiguousarray(capacity, dtype=np.int64)
    if c.size != DG_N_MAX:
        raise ValueError("capacity needs %d entries" % DG_N_MAX)
    h = ctypes.c_void_p()
    _lib.check(_lib.load().dg_server_create(_ptr(c), _lib.DG_SERVER_SEQUENTIAL if sequential else 0,
                                            ctypes.byref(h)), "dg_server_create")
    return h.value


def dg_server_destroy(server):
    if server:
        _lib.load().dg_server_destroy(server)


def dg_server_submit(server, op, T, source=None, q0=None, out=None):
    """q0 / out: contiguous float32 host arrays of 3 * K * Np values (or
    None); they must stay alive until admission / completion."""
    rid = ctypes.c_int64()
    src = None
    if source is not None:
        src = ctypes.byref(_lib.dg_point_source(*[float(v) for v in source]))
    _lib.check(_lib.load().dg_server_submit(server, op, T, src,
                                            None if q0 is None else _buf_ptr(q0),
                                            None if out is None else _buf_ptr(out),
                                            ctypes.byref(rid)), "dg_server_submit")
    return rid.value


def _info_dict(i):
    return {"state": i.state, "status": i.status, "N": i.N, "K": i.K, "nsteps": i.nsteps,
            "dt": i.dt, "t_submit": i.t_submit, "t_admit": i.t_admit, "t_done": i.t_done,
            "t_retired": i.t_retired}


def dg_server_wait(server, request_id, timeout=-1.0):
    info = _lib.dg_request_info()
    _lib.check(_lib.load().dg_server_wait(server, request_id, timeout, ctypes.byref(info)),
               "dg_server_wait")
    return _info_dict(info)


def dg_server_info(server, request_id):
    info = _lib.dg_request_info()
    _lib.check(_lib.load().dg_server_info(server, request_id, ctypes.byref(info)), "dg_server_info")
    return _info_dict(info)


def dg_server_cancel(server, request_id):
    _lib.check(_lib.load().dg_server_cancel(server, request_id), "dg_server_cancel")


def dg_server_set_work_limit(server, max_nodes):
    _lib.check(_lib.load().dg_server_set_work_limit(server, int(max_nodes)),
               "dg_server_set_work_limit")


def dg_server_release(server, request_id):
    _lib.check(_lib.load().dg_server_release(server, request_id), "dg_server_release")


def dg_server_stats(server):
    v = [ctypes.c_int64() for _ in range(4)]
    _lib.check(_lib.load().dg_server_stats(server, *[ctypes.byref(x) for x in v]), "dg_server_stats")
    return {"completed": v[0].value, "failed": v[1].value, "steps": v[2].value,
            "launches": v[3].value}


# ------------------------------------------------------------ convenience
# FP32-field variants: name -> dg_operator_setup flags
_FP32_VARIANTS = {
    "fp32": 0,                              # per order: element threads at N <= 2, else 3xTF32
    "fp32tc": _lib.DG_SETUP_TC,             # 3xTF32 tensor-core products at every order
    "fp32simt": _lib.DG_SETUP_SIMT,         # CUDA-core FP32 products
    "fp32ept": _lib.DG_SETUP_ELEMENT_THREADS,  # CUDA cores, one thread per element (N <= 5)
    "tf32": _lib.DG_SETUP_TC_TF32,          # one TF32 product
    "bf16": _lib.DG_SETUP_TC_BF16,          # one BF16 product
    "bf16x3": _lib.DG_SETUP_TC_BF16X3,      # three BF16 products (hi/lo split)
}


# ------------------------------------------------------------ partitions
def dg_partition_create(op, P):
    h = ctypes.c_void_p()
    _lib.check(_lib.load().dg_partition_create(op, P, ctypes.byref(h)), "dg_partition_create")
    return h


def dg_partition_destroy(part):
    if part:
        _lib.load().dg_partition_destroy(part)


def dg_partition_info(part, p):
    """(K_p, G_p, n_recv_peers, n_send_peers, n_recv, n_send) of part p."""
    K, G, n_sends, n_recvs = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    rp, sp = ctypes.c_int32(), ctypes.c_int32()
    _lib.check(_lib.load().dg_partition_info(part, p, ctypes.byref(K), ctypes.byref(G),
                                             ctypes.byref(rp), ctypes.byref(sp),
                                             ctypes.byref(n_recvs), ctypes.byref(n_sends)),
               "dg_partition_info")
    return K.value, G.value, rp.value, sp.value, n_recvs.value, n_sends.value


def dg_partition_elements(part, p):
    K = dg_partition_info(part, p)[0]
    out = np.empty(K, np.int64)
    _lib.check(_lib.load().dg_partition_elements(part, p, _ptr(out)), "dg_partition_elements")
    return out


def dg_partition_ghosts(part, p):
    G = dg_partition_info(part, p)[1]
    out = np.empty(max(G, 1), np.int64)
    _lib.check(_lib.load().dg_partition_ghosts(part, p, _ptr(out)), "dg_partition_ghosts")
    return out[:G]


def dg_partition_conn(part, p):
    K = dg_partition_info(part, p)[0]
    out = np.empty((K, 3), np.int32)
    _lib.check(_lib.load().dg_partition_conn(part, p, _ptr(out)), "dg_partition_conn")
    return out


def dg_partition_exchange_plan(part, p):
    """{"send": [(peer, offsets)], "recv": [(peer, offsets)]} of part p."""
    _, _, rp, sp, nr, ns = dg_partition_info(part, p)
    send_peer, recv_peer = np.empty(max(sp, 1), np.int32), np.empty(max(rp, 1), np.int32)
    send_cnt, recv_cnt = np.empty(max(sp, 1), np.int64), np.empty(max(rp, 1), np.int64)
    send_off, recv_off = np.empty(max(ns, 1), np.int32), np.empty(max(nr, 1), np.int32)
    _lib.check(_lib.load().dg_partition_exchange_plan(
        part, p, _ptr(send_peer), _ptr(send_cnt), _ptr(send_off), _ptr(recv_peer),
        _ptr(recv_cnt), _ptr(recv_off)), "dg_partition_exchange_plan")

    def split(peers, counts, offs, n):
        out, o = [], 0
        for i in range(n):
            out.append((int(peers[i]), offs[o:o + counts[i]].copy()))
            o += counts[i]
        return out
    return {"send": split(send_peer, send_cnt, send_off, sp),
            "recv": split(recv_peer, recv_cnt, recv_off, rp)}


def dg_partition_set_fields(part, q, q_stride, stream=None):
    _lib.check(_lib.load().dg_partition_set_fields(part, _dptr(q), q_stride,
                                                   _stream_handle(stream)),
               "dg_partition_set_fields")


def dg_partition_get_fields(part, q, q_stride, stream=None):
    _lib.check(_lib.load().dg_partition_get_fields(part, _dptr(q), q_stride,
                                                   _stream_handle(stream)),
               "dg_partition_get_fields")


def dg_partition_exchange(part, stream=None):
    _lib.check(_lib.load().dg_partition_exchange(part, _stream_handle(stream)),
               "dg_partition_exchange")


def dg_partition_step(part, dt, nsteps, stream=None):
    _lib.check(_lib.load().dg_partition_step(part, dt, nsteps, _stream_handle(stream)),
               "dg_partition_step")


def dg_partition_sync_check(part, stream=None):
    _lib.check(_lib.load().dg_partition_sync_check(part, _stream_handle(stream)),
               "dg_partition_sync_check")


class Solver:
    """Owns a mesh + operator pair and the torch tensors that hold fields.

    Field tensors have shape (3, field_stride) on the operator's device, in
    the operator's precision; ``view(q)`` gives the (3, K, Np) window.
    ``precision``: "fp64", or an FP32-field variant: "fp32" (default:
    element threads at N <= 2, tensor cores (3xTF32) above), "fp32tc"
    (tensor cores at every order), "fp32simt", "fp32ept" (one thread per
    element on the CUDA cores, N <= 5), "tf32", "bf16", "bf16x3".
    ``eps``: per-element permittivity (K values; dg_operator_setup_media).
    """

    def __init__(self, VX, VY, EToV, N, precision="fp32", device=None, host_only=False,
                 simt=False, eps=None):
        import torch
        variant_flags = 0
        if precision in _FP32_VARIANTS:
            variant_flags = _FP32_VARIANTS[precision]
            precision = "fp32"
        elif precision not in ("fp64", DG_FP64, DG_FP32):
            raise ValueError("unknown precision %r" % (precision,))
        if simt:
            variant_flags |= _lib.DG_SETUP_SIMT
        self.precision = DG_FP32 if precision in ("fp32", DG_FP32) else DG_FP64
        self.dtype = torch.float32 if self.precision == DG_FP32 else torch.float64
        if device is not None and not host_only:
            torch.cuda.set_device(device)
        self.device = None if host_only else torch.device("cuda", torch.cuda.current_device())
        self.mesh = dg_mesh_create(VX, VY, EToV)
        try:
            flags = (DG_SETUP_HOST_ONLY if host_only else 0) | variant_flags
            if eps is None:
                self.op = dg_operator_setup(self.mesh, N, self.precision, flags)
            else:
                self.op = dg_operator_setup_media(self.mesh, N, eps, self.precision, flags)
        except Exception:
            dg_mesh_destroy(self.mesh)
            raise
        self.N = N
        self.Np, self.Nfp, self.K, self.fstride = dg_get_info(self.op)

    def close(self):
        dg_op_destroy(getattr(self, "op", None))
        dg_mesh_destroy(getattr(self, "mesh", None))
        self.op = self.mesh = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # fields
    def new_fields(self, zero=True):
        import torch
        f = torch.zeros if zero else torch.empty
        return f((3, self.fstride), dtype=self.dtype, device=self.device)

    def view(self, q):
        return q[:, : self.K * self.Np].view(3, self.K, self.Np)

    def from_numpy(self, q3):
        import torch
        q = self.new_fields()
        self.view(q).copy_(torch.as_tensor(np.asarray(q3), dtype=self.dtype))
        return q

    def to_numpy(self, q):
        return self.view(q).detach().to("cpu", dtype=__import__("torch").float64).numpy()

    # hot path
    def rhs(self, q, out=None, stream=None):
        out = self.new_fields(zero=False) if out is None else out
        dg_rhs(self.op, q, out, 0.0, stream)
        return out

    def step(self, q, res, dt, nsteps=1, t0=0.0, stream=None):
        dg_step(self.op, q, res, t0, dt, nsteps, stream)
        return q

    def solve(self, q, res, T, dt=0.0, stream=None):
        return dg_solve(self.op, q, res, T, dt, stream)

    def cfl_dt(self, cfl=1.0):
        return dg_cfl_dt(self.op, cfl)

    def save(self, q, path, t=0.0, step=0):
        """Checkpoint the fields q (a field tensor of this solver) with t, step."""
        dg_checkpoint_save(self.op, q, self.fstride, t, step, path)

    def load(self, path, q):
        """Resume: fill q from a checkpoint of this solver's mesh; returns (t, step)."""
        return dg_checkpoint_load(self.op, path, q, self.fstride)

    def tune(self, reps=5, stream=None):
        """Pick the fastest FP32 kernel and block size for this mesh (dg_operator_tune)."""
        return dg_operator_tune(self.op, reps, stream)

    def kernel(self):
        """(kernel, elements per block) the hot-path calls run."""
        return dg_operator_kernel(self.op)

    def nodes(self):
        return dg_get_nodes(self.op)


class Batch:
    """Many problems of mixed orders stepped together (dg_batch_*).

    ``capacity``: dict order -> element capacity, or 7 counts.  ``add``
    admits a Solver's operator (FP32) with its time step; fields move in and
    out as (3, K, Np) arrays.  ``split``: the split launch mode only
    (DG_BATCH_SPLIT); by default the orders' kernels run side by side.
    """

    def __init__(self, capacity, graph=True, adapt=True, device=None, split=False):
        import torch
        if device is not None:
            torch.cuda.set_device(device)
        if isinstance(capacity, dict):
            cap = [0] * DG_N_MAX
            for n, c in capacity.items():
                cap[n - 1] = int(c)
            capacity = cap
        flags = ((0 if graph else _lib.DG_BATCH_NO_GRAPH) | (0 if adapt else _lib.DG_BATCH_NO_ADAPT)
                 | (_lib.DG_BATCH_SPLIT if split else 0))
        self.batch = dg_batch_create(capacity, flags)

    def close(self):
        dg_batch_destroy(getattr(self, "batch", None))
        self.batch = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add(self, solver_or_op, dt=0.0, source=None, stream=None):
        """source: None or (x, y, f, t0, amplitude) of a Ricker point source."""
        op = solver_or_op.op if hasattr(solver_or_op, "op") else solver_or_op
        return dg_batch_add(self.batch, op, dt, source, stream)

    def remove(self, slot):
        dg_batch_remove(self.batch, slot)

    def info(self, slot):
        return dg_batch_info(self.batch, slot)

    def set_fields(self, slot, q3, stream=None):
        import torch
        q = np.ascontiguousarray(q3, dtype=np.float32)
        dg_batch_set_fields(self.batch, slot, q, q[0].size, stream)
        (stream or torch.cuda.current_stream()).synchronize()  # q is pageable and local

    def get_fields(self, slot, stream=None):
        import torch
        N, K, _, _ = self.info(slot)
        Np = (N + 1) * (N + 2) // 2
        out = np.empty((3, K, Np), np.float32)
        dg_batch_get_fields(self.batch, slot, out, K * Np, stream)
        (stream or torch.cuda.current_stream()).synchronize()
        return out

    def step(self, nsteps=1, stream=None):
        dg_batch_step(self.batch, nsteps, stream)

    def tune(self, reps=5, stream=None):
        dg_batch_tune(self.batch, reps, stream)

    def plan(self):
        return dg_batch_plan(self.batch)

    def launch_mode(self):
        return dg_batch_launch_mode(self.batch)

    def set_block_elems(self, N, elems):
        dg_batch_set_block_elems(self.batch, N, elems)

    def block_elems(self):
        return dg_batch_block_elems(self.batch)

    def sync_check(self, stream=None):
        dg_batch_sync_check(self.batch, stream)

    def launch_count(self):
        return dg_batch_launch_count(self.batch)


class Server:
    """Continuous-batching solve server (dg_server_*).

    ``capacity``: dict order -> element capacity, or 7 counts (the memory
    budget).  ``submit`` returns a request id at once; the result lands in
    the ``out`` array given to it once ``wait`` reports the request done.
    Operators, q0 and out arrays are kept alive here until ``release``.
    ``work_limit``: at most this many nodal values per field (sum of K * Np)
    stepped together, first come first served (dg_server_set_work_limit).
    """

    def __init__(self, capacity, sequential=False, device=None, work_limit=0):
        import torch
        if device is not None:
            torch.cuda.set_device(device)
        if isinstance(capacity, dict):
            cap = [0] * DG_N_MAX
            for n, c in capacity.items():
                cap[n - 1] = int(c)
            capacity = cap
        self.server = dg_server_create(capacity, sequential)
        self._keep = {}
        if work_limit:
            dg_server_set_work_limit(self.server, work_limit)

    def set_work_limit(self, max_nodes):
        dg_server_set_work_limit(self.server, max_nodes)

    def close(self):
        dg_server_destroy(getattr(self, "server", None))
        self.server = None
        self._keep = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, solver_or_op, T, source=None, q0=None, out=None):
        op = solver_or_op.op if hasattr(solver_or_op, "op") else solver_or_op
        if q0 is not None:
            q0 = np.ascontiguousarray(q0, dtype=np.float32)
        rid = dg_server_submit(self.server, op, T, source, q0, out)
        self._keep[rid] = (solver_or_op, q0, out)
        return rid

    def wait(self, rid, timeout=-1.0):
        return dg_server_wait(self.server, rid, timeout)

    def info(self, rid):
        return dg_server_info(self.server, rid)

    def release(self, rid):
        dg_server_release(self.server, rid)
        self._keep.pop(rid, None)

    def cancel(self, rid):
        dg_server_cancel(self.server, rid)

    def stats(self):
        return dg_server_stats(self.server)

    @staticmethod
    def clock():
        return dg_server_clock()


class Partition:
    """A Solver's mesh split into P parts stepped with one halo exchange per
    LSRK stage (dg_partition_*).  Fields move in and out as the Solver's
    (3, field_stride) tensors; ``plan(p)`` is part p's exchange lists."""

    def __init__(self, solver, P):
        self.solver = solver  # the operator must outlive the partition
        self.P = P
        self.part = dg_partition_create(solver.op, P)

    def close(self):
        dg_partition_destroy(getattr(self, "part", None))
        self.part = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self, p):
        return dg_partition_info(self.part, p)

    def elements(self, p):
        return dg_partition_elements(self.part, p)

    def ghosts(self, p):
        return dg_partition_ghosts(self.part, p)

    def conn(self, p):
        return dg_partition_conn(self.part, p)

    def plan(self, p):
        return dg_partition_exchange_plan(self.part, p)

    def set_fields(self, q, stream=None):
        dg_partition_set_fields(self.part, q, self.solver.fstride, stream)

    def get_fields(self, q, stream=None):
        dg_partition_get_fields(self.part, q, self.solver.fstride, stream)

    def exchange(self, stream=None):
        dg_partition_exchange(self.part, stream)

    def step(self, dt, nsteps=1, stream=None):
        dg_partition_step(self.part, dt, nsteps, stream)

    def sync_check(self, stream=None):
        dg_partition_sync_check(self.part, stream)
