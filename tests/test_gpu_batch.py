"""GPU batches (pdhg_batch): many 1D instances per launch.

A batched instance runs the same per-block code as a lone handle, so its
iterates equal the lone instance's bit for bit; against the oracle the
batched iterates meet the same bounds as single-instance parity; instances
leave the launches when they converge, after as many iterations as alone."""
import numpy as np
import pytest

import pdhg_workloads as W
from oracle import pdhg as opdhg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2207_07234_gb300 import binding
    binding.load()
    return binding


def steps(p, t, t0=0.1):
    return p.replace(tau_u=t, tau_phi=t, tau_u0=t0, tau_lambda=0.99)


def mixed():
    return [
        steps(W.advection_upwind_be(nx=256, nt=9), 0.6),
        steps(W.advection_upwind_be(nx=64, nt=5).replace(time="bdf2"), 0.4),
        steps(W.viscous_burgers(nx=512, nt=13, T=1.0, nu=0.01), 0.35),
        W.heat_table1(128, 11),
        W.burgers_dg_p2(ncell=128, nt=6, T=0.5, time="be").replace(c=0.5, tau_u=0.05, tau_u0=0.05, tau_phi=0.05),
        W.traffic_dg_p1(ncell=64, nt=7),
        steps(W.advection_upwind_be(nx=1024, nt=3).replace(alpha=-1.0, beta=1.0,
              u0=0.25 + 0.1 * np.sin(W.fd_nodes(1024, 2 * np.pi)), space="fd_lf", lf_a=0.5), 0.5),
    ]


FIELDS = ("u", "phi", "phit", "lambda", "lambdat")


LAUNCHES = [dict(persistent=True), dict(persistent=False),
            dict(persistent=True, blocks_per_sm=1, order=1, tiles=[3, 2, 4, 1, 2, 5, 1, 2])]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("launch", LAUNCHES, ids=["persistent", "per_stage", "persistent_order1_tiles"])
def test_batch_equals_lone_instances_bitwise(B, precision, launch):
    """The persistent launch (work queue, any tiles and blocks per multiprocessor) and the
    per-stage launches run the same per-block code: the iterates equal a lone handle's."""
    probs = mixed()
    with B.Batch(probs, precision=precision) as bt:
        bt.set_launch(**launch)
        bt.launches(reset=True)
        its, st = bt.iterate(20)
        assert bt.launches() == 20 * (1 if launch["persistent"] else 4)
        assert list(its) == [20] * len(probs) and list(st) == [0] * len(probs)
        got = [{f: bt.instance(i).get_host(f) for f in FIELDS} for i in range(len(probs))]
    for p, g in zip(probs, got):
        with B.Solver(p, precision=precision, path="plain") as s:
            s.iterate(20)
            for f in FIELDS:
                assert np.array_equal(s.get_host(f), g[f]), (p.name, f)


def test_batch_fixed_iterates_vs_oracle(B):
    probs = mixed()
    with B.Batch(probs, precision="fp64") as bt:
        bt.iterate(25)
        got = [(bt.instance(i).get_host("u"), bt.instance(i).get_host("phi")) for i in range(len(probs))]
    for p, (u, phi) in zip(probs, got):
        st = opdhg.initial_state(p)
        for _ in range(25):
            opdhg.step(p, st)
        tu = 1e-11 if p.nmodes == 2 else 1e-12
        assert np.max(np.abs(u - st["u"])) <= tu * np.max(np.abs(st["u"])), p.name
        assert np.max(np.abs(phi - st["phi"])) <= 10 * tu * np.max(np.abs(st["phi"])), p.name


def test_batch_convergence_masks_match_lone_counts(B):
    """Each instance stops at the check where it alone would stop; the others go on."""
    probs = [W.advection_upwind_be(nx=128, nt=64, tau=(1.4, 0.1, 0.35, 0.99)), W.heat_table1(64, 16),
             W.advection_upwind_be(nx=64, nt=16, cfl=1.0, tau=(0.5, 0.1, 0.5, 0.99)),
             W.traffic_dg_p1(ncell=32, nt=8)]
    with B.Batch(probs, precision="fp64") as bt:
        its, st = bt.iterate(20000, tol=1e-8, check_every=10)
    assert list(st) == [1] * len(probs)
    for p, n in zip(probs, its):
        with B.Solver(p, precision="fp64", path="plain") as s:
            assert s.iterate(20000, tol=1e-8, check_every=10) == n, p.name
    assert len(set(its)) > 1


@pytest.mark.parametrize("launch", LAUNCHES[:2], ids=["persistent", "per_stage"])
def test_batch_graph_replay_equals_launch_by_launch(B, launch):
    """Chunks of check_every iterations replayed from a CUDA graph (rebuilt whenever an
    instance leaves the active set) give the same counts, states and fields, bit for bit,
    as the same run launched kernel by kernel; 23 = 4 chunks of 5 plus a tail of 3."""
    probs = mixed()
    out = {}
    for graphs in (True, False):
        with B.Batch(probs, precision="fp64") as bt:
            bt.set_launch(**launch)
            bt.set_graphs(graphs)
            bt.launches(reset=True)
            its, st = bt.iterate(23, tol=0.3, check_every=5, relative=True)
            out[graphs] = (list(its), list(st), bt.launches(),
                           [{f: bt.instance(i).get_host(f) for f in FIELDS} for i in range(len(probs))])
    assert out[True][:3] == out[False][:3]
    for a, b in zip(out[True][3], out[False][3]):
        for f in FIELDS:
            assert np.array_equal(a[f], b[f]), f


def test_batch_isolates_a_diverging_instance(B):
    good = W.advection_upwind_be(nx=128, nt=16, tau=(0.5, 0.1, 0.5, 0.99))
    bad = good.replace(tau_u=40.0, tau_phi=40.0, tau_u0=40.0)
    with B.Batch([good, bad, good], precision="fp64") as bt:
        its, st = bt.iterate(20000, tol=1e-8, check_every=10)
        assert list(st) == [1, -1, 1]
        assert its[1] < its[0]
        assert np.all(np.isfinite(bt.instance(0).get_host("u")))


def test_batch_of_256_sampled(B):
    """The 256-instance workload (float32): a few iterations, then four instances
    (largest, smallest, median, smallest advection) against lone runs, bit for bit."""
    probs = W.batch_instances()
    with B.Batch(probs, precision="fp32") as bt:
        bt.iterate(5)
        cells = np.array([p.ndof * p.nt for p in probs])
        adv = [i for i, p in enumerate(probs) if p.space == "fd_upwind"]
        small_adv = min(adv, key=lambda i: cells[i])
        pick = [int(np.argmax(cells)), int(np.argmin(cells)), int(np.argsort(cells)[len(cells) // 2]), small_adv]
        got = {i: bt.instance(i).get_host("u") for i in pick}
        assert bt.launches() >= 5
    for i in pick:
        with B.Solver(probs[i], precision="fp32", path="plain") as s:
            s.iterate(5)
            assert np.array_equal(s.get_host("u"), got[i]), probs[i].name


def test_batch_instances_fp64_vs_oracle(B):
    """Instances drawn from the 256-instance distribution (the smallest advection and
    the smallest Burgers one, both with Bluestein lengths), batched in float64: 5
    iterations equal the oracle's within 1e-9.  These long-horizon instances (T up to
    ~12, CFL up to 8) lose digits to cancellation in J^T phit, whose low-frequency part
    the preconditioner makes large: in the oracle itself a 1e-15 relative change of u0
    moves u by 3e-11 relative after 5 iterations (advection 369 x 107), so rounding
    order alone accounts for differences of that size; in float32 the same cancellation
    costs about three digits, which is why the oracle comparison is made in float64 (the
    float32 batch is checked bit for bit against lone float32 runs above)."""
    probs = W.batch_instances()
    cells = np.array([p.ndof * p.nt for p in probs])
    pick = [min((i for i, p in enumerate(probs) if p.space == sp), key=lambda i: cells[i])
            for sp in ("fd_upwind", "fd_lf")]
    sub = [probs[i] for i in pick]
    with B.Batch(sub, precision="fp64") as bt:
        bt.iterate(5)
        got = [bt.instance(i).get_host("u") for i in range(len(sub))]
    for p, u in zip(sub, got):
        st = opdhg.initial_state(p)
        for _ in range(5):
            opdhg.step(p, st)
        assert np.max(np.abs(u - st["u"])) <= 1e-9 * np.max(np.abs(st["u"])), p.name


def test_batch_wait_budget_timeout_is_reported(B):
    """The bounded waits of the persistent iteration: with a zero budget the first wait
    gives up, the blocks leave, and the next residual check reports PDHG_ERR_TIMEOUT; the
    CUDA context stays usable and a new batch runs normally."""
    probs = mixed()
    with B.Batch(probs, precision="fp64") as bt:
        bt.set_launch(persistent=True)
        bt.set_wait_budget(0)
        with pytest.raises(B.PdhgError) as e:
            bt.iterate(2, tol=0.0, check_every=1)
        assert e.value.status == -6
    with B.Batch(probs, precision="fp64") as bt:
        bt.set_launch(persistent=True)
        its, st = bt.iterate(3, tol=0.0, check_every=1)
        assert list(its) == [3] * len(probs)
        assert all(np.all(np.isfinite(bt.instance(i).get_host("u"))) for i in range(len(probs)))
