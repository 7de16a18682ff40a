"""GPU tests of the autotuner (sun_autotune, sun_autotune_batch): it returns a
configuration the library accepts, the configuration it picks keeps the
update within the FP32 tolerance of the oracle, repeated calls come from the
cache, and a batch built with the tuned options still evolves every chain
exactly as alone."""

import numpy as np
import pytest

import oracle as orc
from tests.inputs import random_gauge_config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sunlib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1112_4533_gb300 import build as b
    b.build()
    import paper_1112_4533_gb300 as p
    p.load_library()
    return p


def lattice_kwargs(t):
    return {k: t[k] for k in ("storage", "block_threads", "variant", "reunit_mode", "graph_sweeps")}


def test_autotune_su3_picks_a_valid_configuration(sunlib):
    dims = (8, 8, 8, 8)
    t = sunlib.autotune(3, dims, 6.0, 1, 2, tune_storage=True, tune_reunit_mode=True)
    assert t["storage"] in (12, 18)
    assert t["block_threads"] in (64, 128, 256)
    assert t["variant"] & ~(1 | 8) == 0  # no two-row staple unless asked for
    assert t["reunit_mode"] in (0, 1, 2)
    assert t["graph_sweeps"] in (1, 4, 16)
    assert t["ms_per_sweep"] > 0.0
    # the tuned lattice follows the oracle through one overrelaxation pass
    U0 = random_gauge_config(3, dims, 90)
    with sunlib.Lattice(3, dims, 6.0, seed=4, **lattice_kwargs(t)) as L:
        L.import_links(U0)
        L.update_pass(sunlib.OVERRELAX, 2, 1)
        got = L.export_links()
    want = U0.copy()
    orc.update_pass(want, 6.0, orc.OVERRELAX, 2, 1, 0, 4)
    assert np.abs(got - want).max() < 1e-5


def test_autotune_is_cached(sunlib):
    dims = (6, 6, 6, 6)
    a = sunlib.autotune(2, dims, 2.3, 1, 1)
    b = sunlib.autotune(2, dims, 2.3, 1, 1)
    # ms_per_sweep included: a new measurement would not repeat the first one's time
    assert a == b


@pytest.mark.parametrize("nc", [4, 6])
def test_autotune_large_nc_choices(sunlib, nc):
    t = sunlib.autotune(nc, (4, 4, 4, 8), 0.7 * nc * nc, 1, 1, tune_storage=False)
    assert t["storage"] == 2 * nc * nc
    assert t["variant"] & ~(4 | 8) == 0
    with sunlib.Lattice(nc, (4, 4, 4, 8), 0.7 * nc * nc, hot_start=True, **lattice_kwargs(t)) as L:
        L.run(1, 1, 1)


def test_autotuned_batch_keeps_chains_exact(sunlib):
    chains = [(3, (4, 4, 4, 4), 5.8), (3, (6, 6, 6, 6), 6.1), (3, (8, 8, 8, 8), 6.3)]
    t = sunlib.autotune_batch(chains, 1, 2)
    kw = lattice_kwargs(t)
    alone = []
    for i, (nc, dims, beta) in enumerate(chains):
        with sunlib.Lattice(nc, dims, beta, hot_start=True, seed=50 + i, **kw) as L:
            p, l = L.run(2, 1, 2)
            alone.append((L.export_links(), p))
    lats = [sunlib.Lattice(nc, dims, beta, hot_start=True, seed=50 + i, **kw)
            for i, (nc, dims, beta) in enumerate(chains)]
    with sunlib.Batch(lats) as B:
        plaq, _ = B.run(2, 1, 2)
    for i, L in enumerate(lats):
        assert np.array_equal(L.export_links(), alone[i][0])
        assert np.abs(plaq[:, i] - alone[i][1]).max() < 1e-12
        L.close()


def test_autotune_cache_file_persists_across_processes(tmp_path):
    """SUN_TUNE_CACHE: a second process finds the first one's result in the file."""
    import os
    import subprocess
    import sys
    path = tmp_path / "tune.txt"
    code = ("import paper_1112_4533_gb300 as p; "
            "r = p.autotune(3, (6, 6, 6, 6), 6.0, 1, 1); print(r['variant'], r['block_threads'], r['storage'], "
            "repr(r['ms_per_sweep']))")
    env = dict(os.environ, SUN_TUNE_CACHE=str(path))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    first = subprocess.run([sys.executable, "-c", code], env=env, cwd=root, capture_output=True, text=True, timeout=300)
    assert first.returncode == 0, first.stderr
    lines = path.read_text().splitlines()
    assert len(lines) == 1 and "\t" in lines[0]
    second = subprocess.run([sys.executable, "-c", code], env=env, cwd=root, capture_output=True, text=True, timeout=300)
    assert second.returncode == 0, second.stderr
    a, b = first.stdout.split(), second.stdout.split()
    assert a[:3] == b[:3]
    # served from the file: the stored time (written with 6 decimals), not a new measurement
    assert float(b[3]) == round(float(a[3]), 6)
    assert len(path.read_text().splitlines()) == 1
