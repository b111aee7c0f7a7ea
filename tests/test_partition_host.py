"""Host checks of mesh partitions (dg_partition_*; no GPU needed).

A partition splits an operator's elements into P parts; each part reads the
traces of its neighbours across a cut from ghost slots that one halo
exchange per stage fills (only face data crosses a cut).  Checked here on
plan-only partitions of host-only operators:

* every element belongs to exactly one part, parts hold K / P elements to
  within one, in increasing global order;
* each part's connection codes point at the same neighbour element, face
  and orientation as the global ones, through its own slot or a ghost slot
  holding that element;
* carrying out the exchange lists (numpy, one process) fills every node a
  cut face's flux reads with the neighbour's value, and nothing else;
* the same exchange between two gloo ranks on CPU, each holding one part
  and sending / receiving its lists with torch.distributed.
"""
import os
import socket
import sys

import numpy as np
import pytest

from synth import jittered_delaunay_mesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    from paper_1304_5546_gb300 import build as B
    B.build()
    import paper_1304_5546_gb300 as P
    return P


def _face_nodes(N, f):
    """Lattice numbers of face f's nodes (faces v1v2, v2v3, v3v1)."""
    idx = lambda row, col: row * (N + 1) - row * (row - 1) // 2 + col  # noqa: E731
    if f == 0:
        return [j for j in range(N + 1)]
    if f == 1:
        return [idx(j, N - j) for j in range(N + 1)]
    return [idx(j, 0) for j in range(N + 1)]


def _kpad(part, p, K_p):
    """Index of ghost slot 0 of part p: the smallest ghost code (every ghost
    slot is read by some face)."""
    codes = part.conn(p).ravel()
    codes = codes[codes >= 0] >> 3
    ghost = codes[codes >= K_p]
    return int(ghost.min()) if ghost.size else None


def _solver(P, n, N, seed):
    VX, VY, EToV = jittered_delaunay_mesh(n, seed=seed)
    return P.Solver(VX, VY, EToV, N=N, host_only=True)


CASES = [(6, 2, 1, 2), (10, 3, 2, 3), (9, 5, 3, 5), (12, 4, 4, 8), (7, 7, 5, 64)]


@pytest.mark.parametrize("n,N,seed,nparts", CASES)
def test_parts_cover_the_mesh(P, n, N, seed, nparts):
    s = _solver(P, n, N, seed)
    part = P.Partition(s, nparts)
    seen = np.zeros(s.K, np.int64)
    for p in range(nparts):
        el = part.elements(p)
        assert np.all(np.diff(el) > 0)
        assert abs(el.size - s.K / nparts) < 1.0
        seen[el] += 1
    assert np.all(seen == 1)


@pytest.mark.parametrize("n,N,seed,nparts", CASES)
def test_connection_codes_follow_the_global_mesh(P, n, N, seed, nparts):
    s = _solver(P, n, N, seed)
    EToE, EToF = P.dg_mesh_connectivity(s.mesh)[:2]
    part = P.Partition(s, nparts)
    for p in range(nparts):
        el, gh, conn = part.elements(p), part.ghosts(p), part.conn(p)
        K_p = el.size
        kpad = _kpad(part, p, K_p)
        if gh.size:
            assert kpad == (K_p + 1 + 63) // 64 * 64  # the single operator's padding
        local = {int(g): i for i, g in enumerate(el)}
        for e, k in enumerate(el):
            for f in range(3):
                code = conn[e, f]
                if EToE[k, f] == k:  # boundary face
                    assert code == -1
                    continue
                kP, fP = EToE[k, f], EToF[k, f]
                slot = code >> 3
                assert (code >> 1) & 3 == fP
                if int(kP) in local:
                    assert slot == local[int(kP)]
                else:
                    assert gh[slot - kpad] == kP
        # ghosts are distinct elements of other parts
        assert len(set(gh.tolist())) == gh.size
        assert not set(gh.tolist()) & set(local)


def _local_arrays(part, p, q, Np):
    """Part p's field array in its local layout: own elements from q, ghost
    slots NaN (q: (K, Np) of one field)."""
    el, gh = part.elements(p), part.ghosts(p)
    kpad = _kpad(part, p, el.size)
    size = (kpad if kpad is not None else el.size) + gh.size
    loc = np.full((size, Np), np.nan)
    loc[:el.size] = q[el]
    return loc.ravel(), kpad


def _check_ghosts(part, p, loc, kpad, q, N):
    """Every node the flux of a cut face reads holds the neighbour's value;
    ghost nodes no face reads stay NaN."""
    Np = q.shape[1]
    el, gh, conn = part.elements(p), part.ghosts(p), part.conn(p)
    read = np.zeros(loc.size, bool)
    for e in range(el.size):
        for f in range(3):
            code = conn[e, f]
            if code < 0 or (code >> 3) < el.size:
                continue
            slot, fP = code >> 3, (code >> 1) & 3
            for n in _face_nodes(N, fP):
                assert loc[slot * Np + n] == q[gh[slot - kpad], n]
                read[slot * Np + n] = True
    ghost_part = np.arange(loc.size) >= el.size * Np
    assert np.all(np.isnan(loc[ghost_part & ~read]))


@pytest.mark.parametrize("n,N,seed,nparts", CASES)
def test_exchange_lists_fill_the_ghosts(P, n, N, seed, nparts):
    s = _solver(P, n, N, seed)
    part = P.Partition(s, nparts)
    q = np.random.default_rng(seed).standard_normal((s.K, s.Np))
    locs = [_local_arrays(part, p, q, s.Np) for p in range(nparts)]
    plans = [part.plan(p) for p in range(nparts)]
    for p in range(nparts):
        for peer, off in plans[p]["send"]:
            # the receiver's list from p matches entry for entry
            (recv_off,) = [o for src, o in plans[peer]["recv"] if src == p]
            assert recv_off.size == off.size
            locs[peer][0][recv_off] = locs[p][0][off]
    for p in range(nparts):
        _check_ghosts(part, p, locs[p][0], locs[p][1], q, N)
    # message sizes: what p receives is what its peers send it
    for p in range(nparts):
        K_p, G_p, rp, sp, nr, ns = part.info(p)
        assert rp == len(plans[p]["recv"]) and sp == len(plans[p]["send"])
        assert nr == sum(o.size for _, o in plans[p]["recv"])
        assert ns == sum(o.size for _, o in plans[p]["send"])


def test_partition_rejects_bad_use(P):
    from paper_1304_5546_gb300 import DGError
    s = _solver(P, 3, 2, 1)
    for bad in (0, -1, 65, s.K + 1):
        with pytest.raises(DGError):
            P.Partition(s, bad)
    part = P.Partition(s, 2)
    with pytest.raises(DGError):
        part.info(2)
    with pytest.raises(DGError):  # plan only: no device state
        P.dg_partition_step(part.part, 0.1, 1, stream=0)


def _free_port():
    sock = socket.socket()
    sock.bind(("127.0.0.1", 0))
    port = sock.getsockname()[1]
    sock.close()
    return port


def _rank_main(rank, world, port, out_dir):
    """One part per rank: send the plan's outgoing traces to each peer with
    torch.distributed (gloo), receive into the ghost slots, check them."""
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import paper_1304_5546_gb300 as P
    from synth import jittered_delaunay_mesh as mesh

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        N = 4
        s = P.Solver(*mesh(11, seed=7), N=N, host_only=True)
        part = P.Partition(s, world)
        # the same global field on every rank (seeded); a rank keeps only its part
        q = np.random.default_rng(3).standard_normal((s.K, s.Np))
        loc, kpad = _local_arrays(part, rank, q, s.Np)
        plan = part.plan(rank)
        reqs = []
        for peer, off in plan["send"]:
            reqs.append(dist.isend(torch.from_numpy(loc[off].copy()), dst=peer))
        bufs = []
        for peer, off in plan["recv"]:
            buf = torch.empty(off.size, dtype=torch.float64)
            reqs.append(dist.irecv(buf, src=peer))
            bufs.append((off, buf))
        for r in reqs:
            r.wait()
        for off, buf in bufs:
            loc[off] = buf.numpy()
        _check_ghosts(part, rank, loc, kpad, q, N)
        n_recv = sum(o.size for o, _ in bufs)
        dist.barrier()
    finally:
        dist.destroy_process_group()
    with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as f:
        f.write("%d\n" % n_recv)


def test_exchange_between_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp

    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, str(tmp_path)))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
    for p in procs:
        if p.is_alive():
            p.kill()
            p.join()
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    for r in range(world):
        assert int(open(tmp_path / ("rank%d.txt" % r)).read()) > 0
