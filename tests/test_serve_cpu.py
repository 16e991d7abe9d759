"""The serving loop's scheduling on the CPU, with the library calls replaced
by fakes (no GPU): admission by memory budget and (fifo policy) by the
resident-node cap in arrival order, the srpt policy advancing the least
remaining work first within the active-node cap, chunks that never run a
request past its step count, every request finishing once, and a failing
request reported without stopping the others."""
import numpy as np
import pytest

from paper_2108_07605_gb300 import lbm, serve


class FakeSolver:
    def __init__(self, rid, fail):
        self.h = rid
        self.fail = fail
        self.steps = 0

    def moments(self):
        if self.fail:
            raise lbm.LBMError(4, "temperature Newton did not converge")
        return {"steps": self.steps}

    def close(self):
        pass


def _stream(n, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):                      # all arrive at once
        nodes = int(rng.choice([64, 512, 4096]))
        out.append((0.0, {"P": np.zeros(nodes), "steps": int(rng.integers(3, 40)),
                          "lattice": ("D3Q27", "D2Q9")[k % 2], "bytes": nodes * 10}))
    return out


@pytest.fixture
def fakes(monkeypatch):
    import torch
    log = {"runs": [], "resident": []}
    plans = {}

    def create(handles):
        key = object()
        plans[key] = list(handles)
        return key

    def run(plan, n):
        log["runs"].append((tuple(plans[plan]), n))

    def destroy(plan):
        plans.pop(plan)

    monkeypatch.setattr(lbm, "lbm_batch_create", create)
    monkeypatch.setattr(lbm, "lbm_batch_run", run)
    monkeypatch.setattr(lbm, "lbm_batch_destroy", destroy)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)

    class NoFence:
        def __init__(self, device):
            pass

        def mark(self):
            pass

        def drain(self):
            pass
    monkeypatch.setattr(serve, "_TickFence", NoFence)
    monkeypatch.setattr(serve.Server, "_config_bytes", lambda self, r: r.w["bytes"])

    def admit(self, r, now):
        r.solver = FakeSolver(r.rid, r.w.get("fail", False))
        r.admitted = now
        self.used += r.bytes

    monkeypatch.setattr(serve.Server, "_admit", admit)
    log["plans"] = plans
    return log


def _run(srv, stream, log):
    done = srv.run(stream, on_tick=lambda now, act, pend, fin: log["resident"].append(
        (sum(r.bytes for r in act), sum(r.nodes for r in act), len(act))))
    return done


def test_every_request_finishes_once_within_the_budget(fakes):
    stream = _stream(12)
    budget = 2 * max(w["bytes"] for _a, w in stream)
    # the library's fixed lbm_step_noalloc scratch is taken off the budget
    srv = serve.Server(None, budget + lbm.NOALLOC_SCRATCH_BYTES, chunk=7)
    assert srv.budget == budget
    srv.mech = type("M", (), {"n_species": 9})()
    done = _run(srv, stream, fakes)
    assert sorted(r.rid for r in done) == list(range(12))
    assert all(r.remaining == 0 and r.error is None for r in done)
    assert max(b for b, _n, _k in fakes["resident"]) <= budget
    assert srv.used == 0 and not fakes["plans"]          # every plan destroyed
    # a plan replays at most the chunk and never past a member's step count
    steps = {}
    for members, n in fakes["runs"]:
        assert 1 <= n <= 7
        for m in members:
            steps[m] = steps.get(m, 0) + n
    assert steps == {k: w["steps"] for k, (_a, w) in enumerate(stream)}


def test_node_cap_admits_in_arrival_order(fakes):
    stream = _stream(12, seed=1)
    cap = 5000
    srv = serve.Server(None, 10 ** 12, chunk=5, max_nodes=cap, policy="fifo")
    srv.mech = type("M", (), {"n_species": 9})()
    done = _run(srv, stream, fakes)
    assert len(done) == 12
    assert all(nodes <= cap or k == 1 for _b, nodes, k in fakes["resident"])
    admitted = sorted(done, key=lambda r: (r.admitted, r.rid))
    assert [r.rid for r in admitted] == sorted(r.rid for r in done)   # first come, first admitted


def test_a_failing_request_is_reported_and_the_others_finish(fakes):
    stream = _stream(6, seed=2)
    stream[3][1]["fail"] = True
    srv = serve.Server(None, 10 ** 12, chunk=10)
    srv.mech = type("M", (), {"n_species": 9})()
    done = _run(srv, stream, fakes)
    out = serve.summarize(done, 1.0, 100)
    assert len(done) == 6
    assert [f["request"] for f in out["failed"]] == [3]
    assert "Newton" in out["failed"][0]["error"]
    assert all(r.error is None for r in done if r.rid != 3)


def test_srpt_advances_least_remaining_work_first(fakes):
    """A long request that arrived first and a short one that arrived later,
    both resident, with room to advance only one at a time: the short one
    runs first and finishes first; the long one then runs to its end."""
    stream = [(0.0, {"P": np.zeros(4096), "steps": 40, "lattice": "D3Q27", "bytes": 10}),
              (0.0, {"P": np.zeros(4096), "steps": 5, "lattice": "D3Q27", "bytes": 10})]
    srv = serve.Server(None, 10 ** 12, chunk=10, policy="srpt", active_nodes=5000)
    srv.mech = type("M", (), {"n_species": 9})()
    done = _run(srv, stream, fakes)
    assert [r.rid for r in done] == [1, 0]
    assert all(len(members) == 1 for members, _n in fakes["runs"])
    assert fakes["runs"][0] == ((1,), 5)
    assert sum(n for members, n in fakes["runs"] if members == (0,)) == 40


def test_srpt_keeps_the_advanced_nodes_within_the_cap(fakes):
    stream = _stream(12, seed=4)
    cap = 5000
    srv = serve.Server(None, 10 ** 12, chunk=6, policy="srpt", active_nodes=cap)
    srv.mech = type("M", (), {"n_species": 9})()
    done = _run(srv, stream, fakes)
    assert sorted(r.rid for r in done) == list(range(12))
    nodes = {k: int(w["P"].size) for k, (_a, w) in enumerate(stream)}
    for members, n in fakes["runs"]:
        assert sum(nodes[m] for m in members) <= cap or len(members) == 1
        assert 1 <= n <= 6
