"""GPU parity against the FP64 oracle on meshes large enough that every CTA
of the persistent stage launches walks many element blocks.

The stage kernels run one CTA per SM (152 on a GB300) and walk blocks of E
elements with stride 152 E: E = 40 on the tensor cores from N = 4 on, 80 at
N <= 3 (two row tiles), 8 to 64 on the CUDA cores.  A CTA that handles
eight or more blocks goes round its ring of stage buffers (six deep on the
tensor cores, three on the CUDA cores) and flips every mbarrier phase more
than once.  It also reuses each double-buffered tensor-memory operand and
accumulator several times, hands a stage back for refilling after its
stores, and gathers neighbour traces one block ahead across many blocks.
The meshes here are

  n = 161: K = 51,842 elements, 1,297 blocks of 40 (8.5 per CTA), K % 40 = 2
  n = 225: K = 101,250 elements, 1,266 blocks of 80 (8.3 per CTA), K % 80 = 50

so the last block is ragged too, and blocks per CTA are not a whole number.

Each case checks, element by element, one right-hand side (Eq.
dg-strong-explicit) and two LSRK(5,4) steps on the same seeded input
against the oracle:

* FP32 fields: max nodal error <= 1e-5 relative to max |value|;
* FP64: <= 1e-12;
* the TF32 / BF16 product variants: the bound 32u that follows from their
  operand unit roundoff u (as in test_precision_gpu).

Inputs are seeded uniform random fields rounded to FP32 (both sides get the
values the FP32 solver holds), so every element and every node carries an
O(1) value: a misplaced block, a stale ring slot or a wrong neighbour shows
up as an O(1) error.
"""
import numpy as np
import pytest

import oracle as O
from synth import jittered_delaunay_mesh, random_fields, random_permittivity

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5, "fp32tc": 1e-5, "fp32simt": 1e-5, "fp32pairs": 1e-5,
       "fp32alt": 1e-5}
U = {"tf32": 2.0 ** -11, "bf16": 2.0 ** -8, "bf16x3": 2.0 ** -16}


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1304_5546_gb300 import build as B
    B.build()
    import paper_1304_5546_gb300 as P
    return P


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _n_for(N):
    # blocks of 80 elements at N <= 3 on the tensor cores, 40 above
    return 225 if N <= 3 else 161


class _Case:
    """One mesh and order, with the oracle's right-hand side and two LSRK
    steps of a seeded FP32-representable input, for a given right-hand side
    (uniform medium with flux parameter alpha, or a permittivity eps)."""

    def __init__(self, N, seed, alpha=1.0, eps_seed=None):
        self.N = N
        self.mesh = jittered_delaunay_mesh(_n_for(N), seed=seed)
        self.d = O.Discretization(*self.mesh, N)
        self.alpha = alpha
        self.eps = None if eps_seed is None else random_permittivity(self.d.K, seed=eps_seed)
        q = random_fields(self.d.K, self.d.Np, seed=seed + 1)
        self.q0 = q.astype(np.float32).astype(np.float64)
        self._want = None

    def rhs(self, u, t=0.0):
        if self.eps is None:
            return O.maxwell_rhs(self.d, u, alpha=self.alpha)
        return O.maxwell_rhs_media(self.d, u, self.eps)

    def solver(self, P, prec):
        # "fp32pairs": the tensor-core kernel with face pairs on; "fp32alt":
        # the tensor-core kernel in its alternative element-block size
        special = prec in ("fp32pairs", "fp32alt")
        s = P.Solver(*self.mesh, N=self.N, precision="fp32tc" if special else prec, eps=self.eps)
        if self.alpha != 1.0:
            P.dg_operator_set_alpha(s.op, self.alpha)
        if prec == "fp32pairs":
            P.dg_operator_set_face_pairs(s.op, 1)
        if prec == "fp32alt":
            alt = 40 if self.N <= 3 else 80
            P.dg_operator_set_block_elems(s.op, alt)
            assert s.kernel() == ("tensor cores", alt)
        return s

    def want(self, dt):
        if self._want is None or self._want[0] != dt:
            q = self.q0
            for n in range(2):
                q = O.lsrk_step(self.d, q, n * dt, dt, rhs=self.rhs)
            self._want = (dt, self.rhs(self.q0), q)
        return self._want[1], self._want[2]


_CACHE = {}


def _case(key, *args, **kw):
    # one oracle case alive at a time: the large Discretizations are big
    if key not in _CACHE:
        _CACHE.clear()
        _CACHE[key] = _Case(*args, **kw)
    return _CACHE[key]


def _run(P, case, prec):
    """GPU right-hand side and two steps; returns (rhs, q after 2 steps, dt)."""
    s = case.solver(P, prec)
    try:
        assert s.K == case.d.K
        dt = s.cfl_dt()
        q = s.from_numpy(case.q0)
        rhs = s.to_numpy(s.rhs(q))
        res = s.new_fields()
        s.step(q, res, dt, nsteps=2)
        got = s.to_numpy(q)
        P.dg_sync_check(s.op)
    finally:
        s.close()
    return rhs, got, dt


def _blocks_per_cta(K, E, ctas=152):
    return -(-K // E) / ctas


def test_mesh_sizes_walk_many_blocks_per_cta():
    # the sizes the docstring states (checked on the generator's output)
    for N, E in ((3, 80), (5, 40)):
        K = 2 * _n_for(N) ** 2
        assert _blocks_per_cta(K, E) >= 8.0 and K % E != 0, (N, K)


# the CUDA-core kernel serves every FP32 order with "fp32simt", N = 1 by
# default ("fp32"); "fp32tc" forces the tensor cores at every order
# ("fp32pairs": with face pairs, dg_operator_set_face_pairs; "fp32alt": in
# the alternative block size at N <= 4, dg_operator_set_block_elems); FP64
# (CUDA cores) at N = 3, 5, 7.  Ordered by N so that one oracle case serves
# all of an order's runs.
_UNIFORM = [(N, prec) for N in range(1, 8)
            for prec in ("fp32", "fp32tc", "fp32pairs", "fp32simt")
            + (("fp32alt",) if N <= 4 else ()) + (("fp64",) if N in (3, 5, 7) else ())]


@pytest.mark.parametrize("N,prec", _UNIFORM)
def test_large_uniform_rhs_and_two_steps(P, N, prec):
    case = _case(("uniform", N), N, seed=500 + N)
    rhs, got, dt = _run(P, case, prec)
    want_rhs, want_q = case.want(dt)
    assert _rel(rhs, want_rhs) <= TOL[prec], ("rhs", _rel(rhs, want_rhs))
    assert _rel(got, want_q) <= TOL[prec], ("2 steps", _rel(got, want_q))


_MEDIA = [(N, prec) for N in (3, 7)
          for prec in ("fp32", "fp32pairs") + (("fp32alt",) if N <= 4 else ())
          + ("fp32simt", "fp64")]


@pytest.mark.parametrize("N,prec", _MEDIA)
def test_large_media_rhs_and_two_steps(P, N, prec):
    case = _case(("media", N), N, seed=600 + N, eps_seed=700 + N)
    rhs, got, dt = _run(P, case, prec)
    want_rhs, want_q = case.want(dt)
    assert _rel(rhs, want_rhs) <= TOL[prec], ("rhs", _rel(rhs, want_rhs))
    assert _rel(got, want_q) <= TOL[prec], ("2 steps", _rel(got, want_q))


@pytest.mark.parametrize("prec", ["fp32", "fp32simt", "fp64"])
@pytest.mark.parametrize("N", [2, 5])
def test_large_central_flux_rhs_and_two_steps(P, N, prec):
    # alpha = 0 in Eq. max2d-numflux: the central flux
    case = _case(("alpha0", N), N, seed=800 + N, alpha=0.0)
    rhs, got, dt = _run(P, case, prec)
    want_rhs, want_q = case.want(dt)
    assert _rel(rhs, want_rhs) <= TOL[prec], ("rhs", _rel(rhs, want_rhs))
    assert _rel(got, want_q) <= TOL[prec], ("2 steps", _rel(got, want_q))


@pytest.mark.parametrize("variant", ["tf32", "bf16", "bf16x3"])
@pytest.mark.parametrize("N", [7, 3])
def test_large_precision_variants(P, N, variant):
    # N = 7: one row tile; N = 3: two row tiles (80-element blocks)
    case = _case(("uniform", N), N, seed=500 + N)
    rhs, got, dt = _run(P, case, variant)
    want_rhs, want_q = case.want(dt)
    assert np.isfinite(rhs).all() and np.isfinite(got).all()
    assert _rel(rhs, want_rhs) <= 32 * U[variant], ("rhs", _rel(rhs, want_rhs))
    assert _rel(got, want_q) <= 32 * U[variant], ("2 steps", _rel(got, want_q))


# ------------------------------------------------------------ batch, server
class _Problem:
    """A ~30k-element problem of a batch: media, own dt, optional source."""

    def __init__(self, P, n, N, seed, source=False):
        self.mesh = jittered_delaunay_mesh(n, seed=seed)
        self.N = N
        self.d = O.Discretization(*self.mesh, N)
        self.eps = random_permittivity(self.d.K, seed=seed + 1)
        self.solver = P.Solver(*self.mesh, N=N, precision="fp32", eps=self.eps, host_only=True)
        self.dt = 0.9 * self.solver.cfl_dt()
        self.q0 = random_fields(self.d.K, self.d.Np, seed=seed + 2).astype(np.float32)
        self.source = None
        if source:  # wavelet peak within the two steps
            f = 0.15 / self.dt
            self.source = (0.41, 0.57, f, 1.5 * self.dt, 2.0)

    def oracle(self, steps, dt=None):
        dt = self.dt if dt is None else dt
        if self.source is None:
            rhs = lambda u, t: O.maxwell_rhs_media(self.d, u, self.eps)  # noqa: E731
        else:
            xs, ys, f, t0, amp = self.source
            k, w = O.point_source_weights(self.d, xs, ys)

            def rhs(u, t):
                return (O.maxwell_rhs_media(self.d, u, self.eps)
                        + O.point_source_rhs(self.d, k, w, O.ricker(t, f, t0, amp)))
        q = self.q0.astype(np.float64)
        for n in range(steps):
            q = O.lsrk_step(self.d, q, n * dt, dt, rhs=rhs)
        return q


@pytest.mark.parametrize("split,alt3", [(True, False), (False, False), (False, True)])
def test_large_batch_of_three_orders(P, split, alt3):
    # split mode: n = 123, K = 30,258 per problem (ragged at E = 40 and 80);
    # the planner splits the 152 CTAs over N = 3, 5, 7, so each CTA walks
    # about ten blocks of its order.  Concurrent mode: every order's kernel
    # has 152 CTAs, so the problems are larger (n = 221: K = 97,682 at N = 3;
    # n = 156: K = 48,672 at N = 5, 7), again eight or more blocks per CTA
    sizes = (123, 123, 123) if split else (221, 156, 156)
    probs = [_Problem(P, sizes[0], 3, 11), _Problem(P, sizes[1], 5, 12, source=True),
             _Problem(P, sizes[2], 7, 13)]
    cap = [0] * 7
    for p in probs:
        cap[p.N - 1] += (p.d.K + 3) // 4 * 4
    b = P.Batch(cap, split=split)
    if alt3:  # N = 3 in 40-element blocks: 2,443 blocks, 16 per CTA
        b.set_block_elems(3, 40)
    slots = []
    for p in probs:
        slot = b.add(p.solver, p.dt, source=p.source)
        b.set_fields(slot, p.q0)
        slots.append(slot)
    b.step(2)
    b.sync_check()
    cta, nblk, _ = b.plan()
    got = [b.get_fields(s) for s in slots]
    b.close()
    for p in probs:
        assert nblk[p.N - 1] / max(cta[p.N - 1], 1) >= 8.0, (p.N, cta, nblk)
    for p, g in zip(probs, got):
        want = p.oracle(2)
        assert _rel(g.astype(np.float64), want) <= TOL["fp32"], (p.N, _rel(g, want))


def test_large_server_two_requests(P):
    # two ~30k-element requests with point sources, five steps each (a chunk
    # of four steps, then one), admitted together
    reqs = [_Problem(P, 123, 4, 21, source=True), _Problem(P, 123, 6, 22, source=True)]
    cap = [0] * 7
    for r in reqs:
        cap[r.N - 1] += (r.d.K + 3) // 4 * 4
    srv = P.Server(cap)
    outs, ids = [], []
    for r in reqs:
        r.T = 0.93 * 5 * r.solver.cfl_dt()  # -> 5 steps of T / 5
        o = np.zeros((3, r.d.K, r.d.Np), np.float32)
        outs.append(o)
        ids.append(srv.submit(r.solver, r.T, source=r.source, q0=r.q0, out=o))
    infos = [srv.wait(i, timeout=120.0) for i in ids]
    stats = srv.stats()
    srv.close()
    assert stats["completed"] == 2 and stats["failed"] == 0
    # the two were in the batch together
    assert infos[1]["t_admit"] < infos[0]["t_done"]
    for r, o, info in zip(reqs, outs, infos):
        assert info["state"] == 2 and info["nsteps"] == 5, info
        want = r.oracle(info["nsteps"], dt=info["dt"])
        assert _rel(o.astype(np.float64), want) <= TOL["fp32"], (r.N, _rel(o, want))
