"""GPU checks of batches (dg_batch_*): many problems of mixed orders, sizes,
media and time steps stepped by one persistent launch per stage.

* every problem matches the FP64 oracle stepped alone with its own dt and
  permittivity (FP32 tolerance 1e-5 relative to max |q|, FP32-rounded start);
* a problem's result is bit-for-bit the same alone in a batch and in a mix
  (each element's arithmetic depends only on its own problem);
* graph replay and direct launches agree bit for bit, in both launch modes
  (concurrent: each order's kernel of its own, side by side; split: one
  launch per stage with the CTAs split among the orders), and the two modes
  agree with each other and the oracle;
* problems leave and join between steps (continuous batching): the others
  carry on unchanged and a newcomer in a freed range starts clean;
* the autotuner leaves the fields alone and produces a valid CTA split;
* Ricker point sources: each problem's wavelet runs on its own clock (time 0
  at its first step, stage times t_n + c_i dt), also for problems that join a
  batch that has already stepped.
"""
import numpy as np
import pytest

import oracle as O
from synth import gaussian_pulse, jittered_delaunay_mesh, random_permittivity

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


# (mesh n, N, seed): K = 2 n^2 = 98 (not a multiple of 4), 72, 128, 50, 162, 32
SPECS = [(7, 3, 1), (6, 5, 2), (8, 7, 3), (5, 1, 4), (9, 5, 5), (4, 2, 6)]


class _Problem:
    def __init__(self, P, n, N, seed, dt_scale=0.8, source=False):
        self.mesh = jittered_delaunay_mesh(n, seed=seed)
        self.N = N
        self.d = O.Discretization(*self.mesh, N)
        self.eps = random_permittivity(self.d.K, seed=seed + 100)
        self.solver = P.Solver(*self.mesh, N=N, precision="fp32", eps=self.eps, host_only=True)
        self.dt = dt_scale * self.solver.cfl_dt()
        x0, y0 = 0.3 + 0.05 * (seed % 5), 0.6 - 0.04 * (seed % 4)
        q = np.stack(gaussian_pulse(self.d.x, self.d.y, x0, y0, 0.2))
        self.q0 = q.astype(np.float32).astype(np.float64)
        self.source = None
        if source:
            # wavelet peak after 2.5 steps, a = pi f (t - t0) spanning about +-1.3
            f = 0.15 / self.dt
            self.source = (0.37 + 0.03 * (seed % 3), 0.52, f, 2.5 * self.dt, 1.7)

    def oracle(self, steps):
        if self.source is None:
            rhs = lambda u, t: O.maxwell_rhs_media(self.d, u, self.eps)  # noqa: E731
        else:
            xs, ys, f, t0, amp = self.source
            k, w = O.point_source_weights(self.d, xs, ys)

            def rhs(u, t):
                return (O.maxwell_rhs_media(self.d, u, self.eps)
                        + O.point_source_rhs(self.d, k, w, O.ricker(t, f, t0, amp)))
        q = self.q0
        for n in range(steps):
            q = O.lsrk_step(self.d, q, n * self.dt, self.dt, rhs=rhs)
        return q


def _oracle_without_source(p, steps):
    rhs = lambda u, t: O.maxwell_rhs_media(p.d, u, p.eps)  # noqa: E731
    q = p.q0
    for n in range(steps):
        q = O.lsrk_step(p.d, q, n * p.dt, p.dt, rhs=rhs)
    return q


_Problem.oracle_without_source = staticmethod(_oracle_without_source)


def _capacity(probs, extra=0):
    cap = [0] * 7
    for p in probs:
        cap[p.N - 1] += (p.d.K + 3) // 4 * 4 + extra
    return cap


@pytest.fixture(scope="module")
def problems(P):
    return [_Problem(P, *s) for s in SPECS]


def _run(P, probs, steps, graph=True, tune=False, adapt=True, split=False):
    b = P.Batch(_capacity(probs), graph=graph, adapt=adapt, split=split)
    slots = []
    for p in probs:
        slot = b.add(p.solver, p.dt, source=p.source)
        b.set_fields(slot, p.q0)
        slots.append(slot)
    if tune:
        b.tune(reps=2)
    b.step(steps)
    b.sync_check()
    out = [b.get_fields(s) for s in slots]
    assert b.launch_count() >= 5 * steps
    b.close()
    return out


def test_batch_matches_oracle(P, problems):
    steps = 3
    got = _run(P, problems, steps)
    for p, g in zip(problems, got):
        want = p.oracle(steps)
        assert _rel(g, want) <= TOL, (p.N, p.d.K, _rel(g, want))


def test_alone_equals_in_mix_bitwise(P, problems):
    steps = 2
    mix = _run(P, problems, steps)
    for i in (0, 2, 4):
        alone = _run(P, [problems[i]], steps)[0]
        assert np.array_equal(alone, mix[i]), i


@pytest.mark.parametrize("split", [False, True])
def test_graph_equals_direct_launches(P, problems, split):
    a = _run(P, problems[:4], 2, graph=True, split=split)
    b = _run(P, problems[:4], 2, graph=False, split=split)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_launch_modes_agree_and_match_oracle(P, problems):
    # concurrent (each order's kernel of its own, side by side) and split (one
    # launch per stage, CTAs split among the orders) run the same stage body
    steps = 3
    conc = _run(P, problems, steps, split=False)
    spl = _run(P, problems, steps, split=True)
    for p, x, y in zip(problems, conc, spl):
        want = p.oracle(steps)
        assert _rel(x, want) <= TOL and _rel(y, want) <= TOL
        assert _rel(x, y.astype(np.float64)) <= TOL


def test_leave_and_join_between_steps(P, problems):
    p0, p1, p2 = problems[0], problems[4], problems[1]  # N = 3, 5, 5
    cap = _capacity([p0, p1], extra=0)
    cap[4] = max(cap[4], (p2.d.K + 3) // 4 * 4)  # p2 fits where p1 was
    b = P.Batch(cap)
    s0 = b.add(p0.solver, p0.dt)
    b.set_fields(s0, p0.q0)
    s1 = b.add(p1.solver, p1.dt)
    b.set_fields(s1, p1.q0)
    b.step(2)
    got1 = b.get_fields(s1)
    b.remove(s1)
    s2 = b.add(p2.solver, p2.dt)  # reuses the freed range
    b.set_fields(s2, p2.q0)
    b.step(1)
    b.sync_check()
    got0 = b.get_fields(s0)
    got2 = b.get_fields(s2)
    b.close()
    assert _rel(got1, p1.oracle(2)) <= TOL
    assert _rel(got0, p0.oracle(3)) <= TOL
    assert _rel(got2, p2.oracle(1)) <= TOL


def test_tune_keeps_fields_and_plans_valid_split(P, problems):
    import torch
    b = P.Batch(_capacity(problems), split=True)
    slots = []
    for p in problems:
        s = b.add(p.solver, p.dt)
        b.set_fields(s, p.q0)
        slots.append(s)
    b.step(1)
    before = [b.get_fields(s) for s in slots]
    b.tune(reps=2)
    after = [b.get_fields(s) for s in slots]
    for x, y in zip(before, after):
        assert np.array_equal(x, y)
    cta, nblk, cost = b.plan()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert cta.sum() <= sms
    for g in range(7):
        assert (cta[g] >= 1) == (nblk[g] > 0)
        assert cta[g] <= max(nblk[g], 0) or nblk[g] == 0
        if nblk[g]:
            assert cost[g] > 0
    # stepping after the tune still matches the oracle
    b.step(1)
    b.sync_check()
    for p, s in zip(problems, slots):
        assert _rel(b.get_fields(s), p.oracle(2)) <= TOL
    b.close()


def test_batch_rejects_bad_use(P, problems):
    from paper_1304_5546_gb300 import DGError
    p = problems[0]  # N = 3
    b = P.Batch({5: 64})
    with pytest.raises(DGError):
        b.add(p.solver, p.dt)  # no capacity for N = 3
    small = P.Batch({3: 8})
    with pytest.raises(DGError):
        small.add(p.solver, p.dt)  # K = 98 > 8
    with pytest.raises(DGError):
        small.remove(0)
    b.close()
    small.close()


@pytest.fixture(scope="module")
def sourced(P):
    return [_Problem(P, n, N, seed, source=True) for n, N, seed in [(6, 3, 11), (7, 5, 12), (5, 7, 13)]]


def test_point_sources_match_oracle(P, sourced):
    steps = 5
    got = _run(P, sourced, steps)
    for p, g in zip(sourced, got):
        want = p.oracle(steps)
        # the source term must matter at this tolerance
        assert _rel(want, _Problem.oracle_without_source(p, steps)) > 1e-3
        assert _rel(g, want) <= TOL, (p.N, _rel(g, want))


def test_point_source_clock_starts_at_join(P, problems, sourced):
    # a sourced problem joins after the batch has stepped three times
    early, late = problems[1], sourced[1]
    b = P.Batch(_capacity([early, late]))
    s0 = b.add(early.solver, early.dt)
    b.set_fields(s0, early.q0)
    b.step(3)
    s1 = b.add(late.solver, late.dt, source=late.source)
    b.set_fields(s1, late.q0)
    b.step(4)
    b.sync_check()
    got0, got1 = b.get_fields(s0), b.get_fields(s1)
    b.close()
    assert _rel(got0, early.oracle(7)) <= TOL
    assert _rel(got1, late.oracle(4)) <= TOL
    # and bit for bit what it gives alone
    alone = _run(P, [late], 4)[0]
    assert np.array_equal(alone, got1)


def test_point_source_outside_mesh_is_rejected(P, sourced):
    from paper_1304_5546_gb300 import DGError
    p = sourced[0]
    b = P.Batch(_capacity([p]))
    with pytest.raises(DGError):
        b.add(p.solver, p.dt, source=(1.5, 0.5, 10.0, 0.12, 1.0))
    b.close()


def test_tune_picks_a_launch_mode_and_keeps_results(P, problems):
    # the tuner times the tuned split against the concurrent mode and keeps
    # the faster; either way the fields stay and the results match
    b = P.Batch(_capacity(problems))
    slots = []
    for p in problems:
        s = b.add(p.solver, p.dt)
        b.set_fields(s, p.q0)
        slots.append(s)
    assert b.launch_mode() == ("concurrent", 0.0, 0.0)  # the default, untuned
    b.tune(reps=2)
    mode, split_ms, conc_ms = b.launch_mode()
    assert split_ms > 0 and conc_ms > 0
    assert mode == ("concurrent" if conc_ms <= split_ms else "split")
    b.step(2)
    b.sync_check()
    for p, s in zip(problems, slots):
        assert _rel(b.get_fields(s), p.oracle(2)) <= TOL
    b.close()
    forced = P.Batch(_capacity(problems), split=True)
    assert forced.launch_mode()[0] == "split"
    forced.close()


def test_alternative_block_sizes_match_oracle(P, problems):
    # concurrent mode: N = 3 in 40-element blocks (default 80); the other
    # orders keep theirs; N = 5 has one size only
    steps = 3
    b = P.Batch(_capacity(problems))
    slots = []
    for p in problems:
        s = b.add(p.solver, p.dt)
        b.set_fields(s, p.q0)
        slots.append(s)
    b.set_block_elems(3, 40)
    with pytest.raises(P.DGError):
        b.set_block_elems(5, 80)
    e = b.block_elems()[0]
    assert e[2] == 40 and e[4] == 40 and e[6] == 40 and e[0] == 80
    b.step(steps)
    b.sync_check()
    for p, s in zip(problems, slots):
        assert _rel(b.get_fields(s), p.oracle(steps)) <= TOL, p.N
    b.set_block_elems(3, 0)
    assert b.block_elems()[0][2] == 80
    b.close()
    split = P.Batch(_capacity(problems), split=True)
    with pytest.raises(P.DGError):
        split.set_block_elems(3, 40)
    split.close()


def test_tune_records_block_sizes(P, problems):
    b = P.Batch(_capacity(problems))
    slots = []
    for p in problems:
        s = b.add(p.solver, p.dt)
        b.set_fields(s, p.q0)
        slots.append(s)
    b.tune(reps=2)
    elems, ms_def, ms_alt = b.block_elems()
    mode = b.launch_mode()[0]
    for N in range(1, 8):
        if elems[N - 1] == 0:
            continue
        sizes = {1: (80, 40), 2: (80, 40), 3: (80, 40), 4: (40, 80)}.get(N, (40,))
        assert elems[N - 1] in sizes
        if mode == "concurrent" and len(sizes) == 2:
            assert ms_def[N - 1] > 0 and ms_alt[N - 1] > 0
            assert elems[N - 1] == (sizes[1] if ms_alt[N - 1] < ms_def[N - 1] else sizes[0])
        if mode == "split":
            assert elems[N - 1] == sizes[0]
    b.step(2)
    b.sync_check()
    for p, s in zip(problems, slots):
        assert _rel(b.get_fields(s), p.oracle(2)) <= TOL
    b.close()


def test_online_split_adaptation_keeps_results(P, problems):
    # split mode, 20 steps: the split is re-planned from clock snapshots along
    # the way; which CTA computes a block never changes a result
    a = _run(P, problems, 20, adapt=True, split=True)
    b = _run(P, problems, 20, adapt=False, split=True)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
