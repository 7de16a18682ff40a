"""Host logic of the continuous-batching server, on the CPU: the GPU objects
(lattices, batches) are replaced by fakes that advance a simulated clock by the
predicted GPU time of what they run, so admission, the memory budget, the
per-tick selection and the scheduling policies are checked without a GPU."""
import numpy as np
import pytest

from paper_1112_4533_gb300 import serve


class Sim:
    def __init__(self):
        self.t = 0.0
        self.resident = 0
        self.max_resident_bytes = 0
        self.selections = []

    def clock(self):
        return self.t


@pytest.fixture
def sim(monkeypatch):
    S = Sim()

    class FakeLattice:
        def __init__(self, nc, dims, beta, hot_start=True, seed=1, precision=32, graph_sweeps=1):
            self.nc, self.dims, self.seed = nc, dims, seed
            S.resident += 1

        def close(self):
            S.resident -= 1

    class FakeBatch:
        def __init__(self, lats, use_graphs=True):
            self.lats = lats

        def run(self, k, n_hb, n_or):
            cost = sum(serve.sweep_cost_ms(serve.Request(0, L.nc, L.dims[0], 1.0, 1, 0, 0.0)) for L in self.lats)
            S.selections.append((len(self.lats), k, cost))
            S.t += k * cost / 1e3
            # fake observables: the chain's seed, so histories can be told apart
            return (np.tile([float(L.seed) for L in self.lats], (k, 1)),
                    np.tile([complex(L.seed, 0) for L in self.lats], (k, 1)))

        def close(self):
            pass

    monkeypatch.setattr(serve.sun, "Lattice", FakeLattice)
    monkeypatch.setattr(serve.sun, "Batch", FakeBatch)
    monkeypatch.setattr(serve, "footprint", lambda r, precision=32: r.nc * r.nc * r.L ** 4 * 100)
    monkeypatch.setattr(serve.time, "sleep", lambda dt: setattr(S, "t", S.t + dt))
    return S


def big_and_small():
    # one SU(6) 24^4 request (about 1.4 s of GPU time per 10 sweeps), then small ones arriving just after
    reqs = [serve.Request(0, 6, 24, 25.0, 100, 10, 0.0)]
    reqs += [serve.Request(i, 2, 8, 2.3, 50, 10 + i, 0.01 * i) for i in range(1, 9)]
    return reqs


def test_every_request_completes_with_its_own_history(sim):
    out = serve.Server(1 << 40, clock=sim.clock).run(big_and_small())
    for r in out:
        assert len(r.plaquette) == r.n_sweeps
        assert np.all(r.plaquette == r.seed)
        assert r.t_done >= r.t_admit >= r.arrival
    assert sim.resident == 0


def test_srpt_lets_small_requests_finish_before_the_large_one(sim):
    out = serve.Server(1 << 40, clock=sim.clock, policy="srpt").run(big_and_small())
    big = out[0]
    assert all(r.t_done < big.t_done for r in out[1:])


def test_fifo_holds_small_requests_behind_the_large_one(sim):
    out = serve.Server(1 << 40, clock=sim.clock, policy="fifo", work_cap_ms=1.0).run(big_and_small())
    big = out[0]
    assert all(r.t_done >= big.t_done for r in out[1:])


def test_selection_respects_the_work_cap(sim):
    cap = 0.5
    serve.Server(1 << 40, clock=sim.clock, work_cap_ms=cap).run(big_and_small())
    for n, k, cost in sim.selections:
        assert n == 1 or cost <= cap + 1e-12


def test_memory_budget_bounds_the_resident_chains(sim):
    reqs = [serve.Request(i, 3, 8, 6.0, 20, i, 0.0) for i in range(6)]
    one = serve.footprint(reqs[0])
    srv = serve.Server(int(2.5 * one), clock=sim.clock)
    peak = []
    orig = serve.sun.Batch.run

    def run(self, k, a, b):
        peak.append(sim.resident)
        return orig(self, k, a, b)

    serve.sun.Batch.run = run
    out = srv.run(reqs)
    assert max(peak) <= 2
    assert all(len(r.plaquette) == 20 for r in out)


def test_request_larger_than_the_budget_is_refused(sim):
    r = serve.Request(0, 6, 24, 25.0, 10, 1, 0.0)
    with pytest.raises(RuntimeError):
        serve.Server(serve.footprint(r) // 2, clock=sim.clock).run([r])
