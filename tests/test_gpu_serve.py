"""GPU tests of the continuous-batching server: every request's plaquette and
Polyakov history is bitwise the same served alone and served in a mix of
concurrent requests of other Nc, sizes and lengths; the memory budget is
respected; the plain path gives the same results."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def serve():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1112_4533_gb300 import build as b
    b.build()
    from paper_1112_4533_gb300 import serve as s
    return s


def small_trace(s):
    # short chains on small lattices, arrivals spread over 0.3 s
    reqs = s.poisson_trace(12, rate=40.0, seed=3, ncs=(2, 3, 4, 6), Ls=(4, 6, 8), sweeps=(3, 9))
    return reqs


def test_each_request_is_the_same_alone_and_in_the_mix(serve):
    trace = small_trace(serve)
    srv = serve.Server(hbm_budget=2 << 30, sweeps_per_tick=2)
    mixed = srv.run(trace)
    assert srv.ticks > 1
    overlapped = [r for r in mixed if any(q is not r and q.t_admit < r.t_done and r.t_admit < q.t_done for q in mixed)]
    assert overlapped, "the trace must put requests on the GPU together"
    for r in mixed[:6]:
        solo_trace = [serve.Request(r.rid, r.nc, r.L, r.beta, r.n_sweeps, r.seed, 0.0)]
        solo = serve.Server(hbm_budget=2 << 30, sweeps_per_tick=3).run(solo_trace)[0]
        assert len(r.plaquette) == r.n_sweeps
        assert np.array_equal(solo.plaquette, r.plaquette), r.rid
        assert np.array_equal(solo.polyakov, r.polyakov), r.rid


def test_plain_path_gives_the_same_chains(serve):
    trace = small_trace(serve)[:5]
    mixed = serve.Server(hbm_budget=2 << 30).run(trace)
    plain, _, _ = serve.serve_plain(trace)
    for a, b in zip(sorted(mixed, key=lambda r: r.rid), sorted(plain, key=lambda r: r.rid)):
        assert np.abs(a.plaquette - b.plaquette).max() < 1e-12
        assert np.abs(a.polyakov - b.polyakov).max() < 1e-12


def test_memory_budget_limits_admission(serve):
    trace = [serve.Request(i, 3, 8, 6.0, 4, 50 + i, 0.0) for i in range(4)]
    one = serve.footprint(trace[0])
    srv = serve.Server(hbm_budget=int(1.5 * one), sweeps_per_tick=2)
    out = srv.run(trace)
    # at most one chain fits at a time: admissions follow completions
    spans = sorted((r.t_admit, r.t_done) for r in out)
    for (a0, d0), (a1, d1) in zip(spans, spans[1:]):
        assert a1 >= d0
    with pytest.raises(RuntimeError):
        serve.Server(hbm_budget=one // 2).run(trace[:1])
