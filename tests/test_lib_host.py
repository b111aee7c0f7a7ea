"""Host-side checks of libdgwave.so that need no GPU: the library loads and
exports every entry point of include/dgwave.h; its FP64 host set-up
(reference element, connectivity, geometry, trace maps, LSRK coefficients,
CFL step) agrees with the oracle; argument and mesh errors come back as
status codes; device entry points refuse a host-only operator."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
from synth import jittered_delaunay_mesh, square_grid_mesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dgw():
    from paper_1304_5546_gb300 import build as B
    B.build()
    import paper_1304_5546_gb300 as P
    return P


def test_exports_every_declared_symbol(dgw):
    header = open(os.path.join(ROOT, "include", "dgwave.h")).read()
    declared = set(re.findall(r"\b(dg_[a-z_0-9]+)\s*\(", header))
    assert len(declared) >= 20
    from paper_1304_5546_gb300 import _lib
    lib = _lib.load()
    for name in sorted(declared):
        assert hasattr(lib, name), name
    bound = {s[0] for s in _lib.SIGNATURES}
    assert declared == bound


@pytest.mark.parametrize("N", list(range(1, 8)))
def test_reference_element_matches_oracle(dgw, N):
    VX, VY, EToV = square_grid_mesh(1, 1)
    mesh = dgw.dg_mesh_create(VX, VY, EToV)
    op = dgw.dg_operator_setup(mesh, N, dgw.DG_FP64, dgw.DG_SETUP_HOST_ONLY)
    try:
        ref = dgw.dg_get_reference(op)
        R = O.ReferenceElement(N)
        assert np.abs(ref["r"] - R.r).max() < 1e-14
        assert np.abs(ref["s"] - R.s).max() < 1e-14
        scale = np.abs(R.Dr).max()
        assert np.abs(ref["Dr"] - R.Dr).max() < 1e-12 * scale
        assert np.abs(ref["Ds"] - R.Ds).max() < 1e-12 * scale
        assert np.abs(ref["LIFT"] - R.LIFT).max() < 1e-12 * np.abs(R.LIFT).max()
        assert np.array_equal(ref["Fmask"], R.Fmask)
    finally:
        dgw.dg_op_destroy(op)
        dgw.dg_mesh_destroy(mesh)


@pytest.mark.parametrize("N", [1, 3, 5, 7])
def test_mesh_geometry_maps_match_oracle(dgw, N):
    VX, VY, EToV = jittered_delaunay_mesh(7, seed=13)
    d = O.Discretization(VX, VY, EToV, N)
    mesh = dgw.dg_mesh_create(VX, VY, EToV)
    op = dgw.dg_operator_setup(mesh, N, dgw.DG_FP32, dgw.DG_SETUP_HOST_ONLY)
    try:
        EToE, EToF, EToVo = dgw.dg_mesh_connectivity(mesh)
        assert np.array_equal(EToE, d.EToE) and np.array_equal(EToF, d.EToF)
        assert np.array_equal(EToVo, d.EToV)
        K, nflip, nb = dgw.dg_mesh_info(mesh)
        assert (K, nflip, nb) == (d.K, 0, 4 * 7)
        Np, Nfp, K2, fstride = dgw.dg_get_info(op)
        assert (Np, Nfp, K2) == (d.Np, d.Nfp, d.K) and fstride >= K * Np and fstride % 64 == 0
        x, y = dgw.dg_get_nodes(op)
        assert np.abs(x - d.x).max() < 1e-14 and np.abs(y - d.y).max() < 1e-14
        g = dgw.dg_get_geometry(op)
        for name in ("rx", "ry", "sx", "sy", "J"):
            want = getattr(d, name)[:, 0]
            assert np.abs(g[name] - want).max() <= 1e-12 * np.abs(want).max(), name
        Fm = d.ref.Fmask
        for name in ("nx", "ny", "Fscale"):
            want = getattr(d, name).reshape(d.K, 3, d.Nfp)[:, :, 0]
            assert np.abs(g[name] - want).max() <= 1e-12 * np.abs(want).max(), name
        vM, vP = dgw.dg_get_maps(op)
        assert np.array_equal(vM, d.vmapM)
        assert np.array_equal(vP, d.vmapP)  # integer trace maps: bit-exact
        assert np.isclose(dgw.dg_cfl_dt(op, 1.0), O.cfl_dt(d), rtol=1e-13)
        del Fm
    finally:
        dgw.dg_op_destroy(op)
        dgw.dg_mesh_destroy(mesh)


def test_relabelled_mesh_maps_match_oracle(dgw):
    from synth import relabel_mesh
    VX, VY, EToV = jittered_delaunay_mesh(5, seed=17)
    E2, _, _ = relabel_mesh(EToV, seed=5)
    # flip a few to clockwise: both sides re-list them the same way
    E2[::7] = E2[::7][:, [0, 2, 1]]
    d = O.Discretization(VX, VY, E2, 4)
    mesh = dgw.dg_mesh_create(VX, VY, E2)
    op = dgw.dg_operator_setup(mesh, 4, dgw.DG_FP64, dgw.DG_SETUP_HOST_ONLY)
    try:
        assert dgw.dg_mesh_info(mesh)[1] == d.n_flipped > 0
        vM, vP = dgw.dg_get_maps(op)
        assert np.array_equal(vM, d.vmapM) and np.array_equal(vP, d.vmapP)
    finally:
        dgw.dg_op_destroy(op)
        dgw.dg_mesh_destroy(mesh)


def test_lsrk_coefficients_match_oracle(dgw):
    a, b, c = dgw.dg_lsrk_coefficients()
    assert np.array_equal(a, O.LSRK_A) and np.array_equal(b, O.LSRK_B)
    assert np.abs(c - O.LSRK_C).max() < 1e-15


def test_error_codes(dgw):
    from paper_1304_5546_gb300 import _lib
    VX, VY, EToV = square_grid_mesh(2, 2)
    # vertex index out of range
    bad = EToV.copy()
    bad[0, 0] = 99
    with pytest.raises(dgw.DGError) as ei:
        dgw.dg_mesh_create(VX, VY, bad)
    assert ei.value.status == _lib.DG_ERR_ARG
    # zero-area element
    with pytest.raises(dgw.DGError) as ei:
        dgw.dg_mesh_create(np.array([0.0, 1.0, 2.0]), np.zeros(3), np.array([[0, 1, 2]]))
    assert ei.value.status == _lib.DG_ERR_MESH_DEGENERATE
    # face shared by three elements
    VX3 = np.array([0.0, 1.0, 0.5, 0.5, 0.5])
    VY3 = np.array([0.0, 0.0, 1.0, -1.0, 2.0])
    with pytest.raises(dgw.DGError) as ei:
        dgw.dg_mesh_create(VX3, VY3, np.array([[0, 1, 2], [1, 0, 3], [0, 1, 4]]))
    assert ei.value.status == _lib.DG_ERR_MESH_NONCONFORMING
    mesh = dgw.dg_mesh_create(VX, VY, EToV)
    try:
        for N in (0, 8, -1):
            with pytest.raises(dgw.DGError) as ei:
                dgw.dg_operator_setup(mesh, N, dgw.DG_FP32, dgw.DG_SETUP_HOST_ONLY)
            assert ei.value.status == _lib.DG_ERR_ORDER
        with pytest.raises(dgw.DGError) as ei:
            dgw.dg_operator_setup(mesh, 3, 7, dgw.DG_SETUP_HOST_ONLY)
        assert ei.value.status == _lib.DG_ERR_ARG
        op = dgw.dg_operator_setup(mesh, 3, dgw.DG_FP32, dgw.DG_SETUP_HOST_ONLY)
        try:
            lib = _lib.load()
            # device entry points refuse a host-only operator (no GPU work)
            st = lib.dg_rhs(op, ctypes.c_void_p(16), ctypes.c_void_p(4096), 0.0, None)
            assert st == _lib.DG_ERR_NO_DEVICE
            assert "host-only" in dgw.dg_last_error()
            st = lib.dg_step(op, ctypes.c_void_p(16), ctypes.c_void_p(4096), 0.0, 0.1, 1, None)
            assert st == _lib.DG_ERR_NO_DEVICE
            assert lib.dg_launch_count(op) == 0
            # pipelined host jobs: three slots of two field buffers and one
            # shared residual; refused without a device
            Np, _, K, fstride = dgw.dg_get_info(op)
            assert lib.dg_step_host_jobs_work_bytes(op) == 7 * 3 * fstride * 4
            bufs = (ctypes.c_void_p * 1)(ctypes.c_void_p(4096))
            st = lib.dg_step_host_jobs(op, 1, bufs, ctypes.c_void_p(4096), 0.0, 0.1, 1, None)
            assert st == _lib.DG_ERR_NO_DEVICE
            st = lib.dg_cfl_dt(op, -1.0, ctypes.byref(ctypes.c_double()))
            assert st == _lib.DG_ERR_ARG
        finally:
            dgw.dg_op_destroy(op)
    finally:
        dgw.dg_mesh_destroy(mesh)
    assert _lib.load().dg_mesh_create(None, None, 0, None, 0, ctypes.byref(ctypes.c_void_p())) == _lib.DG_ERR_ARG


def test_element_thread_flag_checks(dgw):
    # DG_SETUP_ELEMENT_THREADS: FP32, N <= 5, no other kernel or product
    # flag; the kernel report of a host-only operator (no GPU work)
    from paper_1304_5546_gb300 import _lib
    VX, VY, EToV = square_grid_mesh(3, 3)
    mesh = dgw.dg_mesh_create(VX, VY, EToV)
    E, H = _lib.DG_SETUP_ELEMENT_THREADS, dgw.DG_SETUP_HOST_ONLY
    try:
        for N in range(1, 6):
            op = dgw.dg_operator_setup(mesh, N, dgw.DG_FP32, E | H)
            try:
                assert dgw.dg_operator_kernel(op) == ("element threads", 32)
                # 32 elements per block is the kernel's only size
                dgw.dg_operator_set_block_elems(op, 32)
                with pytest.raises(dgw.DGError) as ei:
                    dgw.dg_operator_set_block_elems(op, 40)
                assert ei.value.status == _lib.DG_ERR_ARG
            finally:
                dgw.dg_op_destroy(op)
        bad = [(6, dgw.DG_FP32, E), (7, dgw.DG_FP32, E), (3, dgw.DG_FP64, E),
               (3, dgw.DG_FP32, E | _lib.DG_SETUP_SIMT), (3, dgw.DG_FP32, E | _lib.DG_SETUP_TC),
               (3, dgw.DG_FP32, E | _lib.DG_SETUP_TC_BF16)]
        for N, prec, flags in bad:
            with pytest.raises(dgw.DGError) as ei:
                dgw.dg_operator_setup(mesh, N, prec, flags | H)
            assert ei.value.status == _lib.DG_ERR_ARG, (N, prec, flags)
        # a permittivity is allowed (the kernel's media variant)
        op = dgw.dg_operator_setup_media(mesh, 3, np.ones(EToV.shape[0]), dgw.DG_FP32, E | H)
        try:
            assert dgw.dg_operator_kernel(op) == ("element threads", 32)
        finally:
            dgw.dg_op_destroy(op)
        with pytest.raises(dgw.DGError) as ei:
            dgw.dg_operator_setup_media(mesh, 6, np.ones(EToV.shape[0]), dgw.DG_FP32, E | H)
        assert ei.value.status == _lib.DG_ERR_ARG
    finally:
        dgw.dg_mesh_destroy(mesh)


def test_default_fp32_kernel_per_order(dgw):
    # element threads at N <= 2, tensor cores above, with or without a
    # permittivity
    VX, VY, EToV = square_grid_mesh(3, 3)
    mesh = dgw.dg_mesh_create(VX, VY, EToV)
    eps = np.full(EToV.shape[0], 2.0)
    try:
        for N, want, want_media in ((1, "element threads", "element threads"),
                                    (2, "element threads", "element threads"),
                                    (3, "tensor cores", "tensor cores"),
                                    (5, "tensor cores", "tensor cores")):
            for media, w in ((False, want), (True, want_media)):
                op = (dgw.dg_operator_setup_media(mesh, N, eps, dgw.DG_FP32, dgw.DG_SETUP_HOST_ONLY)
                      if media else dgw.dg_operator_setup(mesh, N, dgw.DG_FP32, dgw.DG_SETUP_HOST_ONLY))
                try:
                    assert dgw.dg_operator_kernel(op)[0] == w, (N, media)
                finally:
                    dgw.dg_op_destroy(op)
    finally:
        dgw.dg_mesh_destroy(mesh)
