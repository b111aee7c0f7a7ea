"""GPU checks of the solve server (dg_server_*): continuous batching of
requests with point sources on one GPU.

* every result equals, bit for bit, the same solve run alone in a batch of
  one (the result does not depend on the mix), and matches the FP64 oracle
  within the FP32 tolerance (1e-5 relative to max |q|);
* requests submitted while another runs are admitted before it finishes
  (continuous batching, not a queue);
* the memory budget holds: a request waits until its order's pool has room,
  and one that cannot fit even an empty pool fails with DG_ERR_OOM;
* the sequential mode runs one solve at a time and gives the same results.
"""
import time

import numpy as np
import pytest

import oracle as O
from synth import gaussian_pulse, jittered_delaunay_mesh

pytestmark = pytest.mark.gpu

TOL = 1e-5


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


class _Req:
    """A small solve: jittered mesh, order N, final time `nsteps` CFL steps,
    Ricker source, Gaussian start."""

    def __init__(self, P, n, N, seed, nsteps=6, source=True):
        self.mesh = jittered_delaunay_mesh(n, seed=seed)
        self.N = N
        self.solver = P.Solver(*self.mesh, N=N, precision="fp32", host_only=True)
        self.K, self.Np = self.solver.K, self.solver.Np
        self.T = 0.93 * nsteps * self.solver.cfl_dt()  # -> nsteps steps
        x, y = self.solver.nodes()
        self.q0 = np.stack(gaussian_pulse(x, y, 0.45, 0.55, 0.2)).astype(np.float32)
        self.source = None
        if source:
            dt = self.T / nsteps
            self.source = (0.4 + 0.02 * (seed % 5), 0.5, 0.15 / dt, 2.0 * dt, 1.3)

    def out(self):
        return np.zeros((3, self.K, self.Np), np.float32)

    def alone(self, P, dt, nsteps):
        b = P.Batch({self.N: (self.K + 3) // 4 * 4})
        s = b.add(self.solver, dt, source=self.source)
        b.set_fields(s, self.q0)
        b.step(nsteps)
        b.sync_check()
        q = b.get_fields(s)
        b.close()
        return q

    def oracle(self, dt, nsteps):
        d = O.Discretization(*self.mesh, self.N)
        if self.source is None:
            rhs = lambda u, t: O.maxwell_rhs(d, u)  # noqa: E731
        else:
            xs, ys, f, t0, amp = self.source
            k, w = O.point_source_weights(d, xs, ys)

            def rhs(u, t):
                return O.maxwell_rhs(d, u) + O.point_source_rhs(d, k, w, O.ricker(t, f, t0, amp))
        q = self.q0.astype(np.float64)
        for n in range(nsteps):
            q = O.lsrk_step(d, q, n * dt, dt, rhs=rhs)
        return q


@pytest.fixture(scope="module")
def reqs(P):
    return [_Req(P, 6, 3, 1), _Req(P, 7, 5, 2), _Req(P, 5, 7, 3), _Req(P, 6, 4, 4, source=False),
            _Req(P, 8, 5, 5, nsteps=9)]


def _capacity(rs):
    cap = [0] * 7
    for r in rs:
        cap[r.N - 1] += (r.K + 3) // 4 * 4
    return cap


@pytest.mark.parametrize("sequential", [False, True])
def test_results_equal_alone_and_oracle(P, reqs, sequential):
    srv = P.Server(_capacity(reqs), sequential=sequential)
    outs = [r.out() for r in reqs]
    ids = [srv.submit(r.solver, r.T, source=r.source, q0=r.q0, out=o) for r, o in zip(reqs, outs)]
    infos = [srv.wait(i, timeout=60.0) for i in ids]
    stats = srv.stats()
    srv.close()
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    for r, o, info in zip(reqs, outs, infos):
        assert info["state"] == 2, info
        alone = r.alone(P, info["dt"], info["nsteps"])
        assert np.array_equal(o, alone), (r.N, r.K)
        want = r.oracle(info["dt"], info["nsteps"])
        assert _rel(o.astype(np.float64), want) <= TOL, (r.N, _rel(o, want))
    if sequential:  # one at a time: each admission after the previous completion
        order = sorted(infos, key=lambda i: i["t_admit"])
        for a, b in zip(order, order[1:]):
            assert b["t_admit"] >= a["t_done"]


def test_requests_join_while_others_run(P, reqs):
    long = _Req(P, 9, 6, 21, nsteps=400, source=True)
    short = reqs[:3]
    srv = P.Server(_capacity([long] + short))
    lid = srv.submit(long.solver, long.T, source=long.source, q0=long.q0, out=long.out())
    # wait until the long solve is on the GPU, then submit the short ones
    t0 = time.time()
    while srv.info(lid)["state"] == 0 and time.time() - t0 < 10:
        time.sleep(0.001)
    sids = [srv.submit(r.solver, r.T, source=r.source, q0=r.q0, out=r.out()) for r in short]
    li = srv.wait(lid, timeout=120.0)
    sinfo = [srv.wait(i, timeout=60.0) for i in sids]
    srv.close()
    assert li["state"] == 2 and all(i["state"] == 2 for i in sinfo)
    # the short requests were admitted and finished while the long one ran
    for i in sinfo:
        assert i["t_admit"] < li["t_done"]
        assert i["t_done"] < li["t_done"]


def test_memory_budget_admission(P, reqs):
    a, b = reqs[1], reqs[4]  # both N = 5; the pool holds only the larger one
    cap = [0] * 7
    cap[4] = max((a.K + 3) // 4 * 4, (b.K + 3) // 4 * 4)
    srv = P.Server(cap)
    oa, ob = a.out(), b.out()
    ia = srv.submit(a.solver, a.T, source=a.source, q0=a.q0, out=oa)
    ib = srv.submit(b.solver, b.T, source=b.source, q0=b.q0, out=ob)
    inf_a, inf_b = srv.wait(ia, 60.0), srv.wait(ib, 60.0)
    too_big = _Req(P, 12, 5, 9)  # K = 288 > capacity
    ic = srv.submit(too_big.solver, too_big.T)
    inf_c = srv.wait(ic, 60.0)
    srv.close()
    assert inf_a["state"] == 2 and inf_b["state"] == 2
    assert inf_b["t_admit"] >= inf_a["t_admit"]
    assert inf_c["state"] == 3 and inf_c["status"] == 6  # DG_ERR_OOM
    assert np.array_equal(ob, b.alone(P, inf_b["dt"], inf_b["nsteps"]))


def test_concurrent_submitters(P, reqs):
    # four host threads submit and wait at once; every result equals the
    # request's solve alone
    import threading
    srv = P.Server(_capacity(reqs))
    outs = []  # (request, result, info) of every submission
    errors = []

    def client(k):
        try:
            for r in reqs[k % 2::2]:
                o = r.out()
                rid = srv.submit(r.solver, r.T, source=r.source, q0=r.q0, out=o)
                info = srv.wait(rid, timeout=60.0)
                outs.append((r, o, info))
        except Exception as ex:  # noqa: BLE001 (reported below)
            errors.append(ex)

    threads = [threading.Thread(target=client, args=(k,)) for k in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    srv.close()
    assert not errors, errors
    assert len(outs) == 2 * len(reqs)
    for r, o, info in outs:
        assert info["state"] == 2
        assert np.array_equal(o, r.alone(P, info["dt"], info["nsteps"]))


def test_cancel_queued_and_running(P, reqs):
    long = _Req(P, 9, 6, 22, nsteps=3000, source=True)
    cap = [0] * 7
    cap[5] = (long.K + 3) // 4 * 4  # room for one of the two N = 6 requests
    short = reqs[0]                 # N = 3
    cap[2] = (short.K + 3) // 4 * 4
    srv = P.Server(cap)
    out_long = long.out()
    lid = srv.submit(long.solver, long.T, source=long.source, q0=long.q0, out=out_long)
    t0 = time.time()
    while srv.info(lid)["state"] == 0 and time.time() - t0 < 10:
        time.sleep(0.001)
    qid = srv.submit(long.solver, long.T, source=long.source, q0=long.q0, out=long.out())
    assert srv.info(qid)["state"] == 0  # no room: queued
    srv.cancel(qid)
    srv.cancel(lid)
    sid = srv.submit(short.solver, short.T, source=short.source, q0=short.q0, out=short.out())
    qi, li, si = srv.wait(qid, 60.0), srv.wait(lid, 60.0), srv.wait(sid, 60.0)
    srv.close()
    assert qi["state"] == 4 and qi["t_admit"] == 0.0   # cancelled before admission
    assert li["state"] == 4 and np.all(out_long == 0)  # cancelled while running, no result
    assert si["state"] == 2


def test_work_limit_bounds_work_stepped_together(P, reqs):
    # limit = the largest request's nodal values: it runs alone, smaller ones
    # share the limit; admissions stay first come, first served
    nodes = [r.K * r.Np for r in reqs]
    limit = max(nodes)
    srv = P.Server(_capacity(reqs), work_limit=limit)
    with pytest.raises(P.DGError):
        srv.set_work_limit(-1)
    outs = [r.out() for r in reqs]
    ids = [srv.submit(r.solver, r.T, source=r.source, q0=r.q0, out=o) for r, o in zip(reqs, outs)]
    infos = [srv.wait(i, timeout=60.0) for i in ids]
    srv.close()
    assert all(i["state"] == 2 for i in infos)
    admits = [i["t_admit"] for i in infos]
    assert admits == sorted(admits)
    for a, (ia, na) in enumerate(zip(infos, nodes)):
        t = ia["t_admit"]
        others = [nb for b, (ib, nb) in enumerate(zip(infos, nodes))
                  if b != a and ib["t_admit"] <= t < ib["t_retired"]]
        assert not others or sum(others) + na <= limit, (a, others, na, limit)
    for r, o, info in zip(reqs, outs, infos):
        assert np.array_equal(o, r.alone(P, info["dt"], info["nsteps"]))
