"""GPU tests of configuration files (sun_save_config / sun_load_config): a
chain saved mid-run and loaded into a fresh lattice (created with another seed,
beta and a cold start) continues bitwise as the uninterrupted chain, for every
storage format; the file's links are the lattice's exported links; mismatched
or damaged files are refused and leave the lattice unchanged."""
import numpy as np
import pytest

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


CASES = [(2, 4, 32), (2, 8, 64), (3, 12, 32), (3, 18, 32), (3, 12, 64), (4, 32, 32), (6, 72, 32)]


def beta_for(nc):
    return 2.3 if nc == 2 else (6.0 if nc == 3 else 0.7 * nc * nc)


@pytest.mark.parametrize("nc,st,prec", CASES)
def test_save_load_resumes_bitwise(sunlib, tmp_path, nc, st, prec):
    dims = (4, 4, 6, 4)
    kw = dict(storage=st, precision=prec, reunit_every=2)
    with sunlib.Lattice(nc, dims, beta_for(nc), hot_start=True, seed=21, **kw) as A:
        ref_p, ref_l = A.run(5, 1, 2)
        ref = A.export_links()
    path = tmp_path / "chain.cfg"
    with sunlib.Lattice(nc, dims, beta_for(nc), hot_start=True, seed=21, **kw) as B:
        B.run(3, 1, 2)  # an odd sweep count: the re-unitarization cadence must resume too
        B.save(path)
        saved = B.export_links()
    h = sunlib.read_config_header(path)
    assert (h["nc"], h["storage"], h["precision"], h["seed"], h["heatbath_step"], h["sweeps_done"]) == \
        (nc, st, prec, 21, 3, 3)
    with sunlib.Lattice(nc, dims, 1.0, hot_start=False, seed=99, **kw) as C:
        C.load(path)
        assert np.array_equal(C.export_links(), saved)
        assert C.heatbath_step == 3
        p, l = C.run(2, 1, 2)
        assert np.array_equal(C.export_links(), ref)
        assert np.array_equal(p, ref_p[3:]) and np.array_equal(l, ref_l[3:])


def test_mismatched_lattice_is_refused_and_unchanged(sunlib, tmp_path):
    path = tmp_path / "a.cfg"
    with sunlib.Lattice(3, (4, 4, 4, 4), 6.0, hot_start=True, seed=3) as A:
        A.save(path)
    for kw in (dict(dims=(4, 4, 4, 6)), dict(storage=18), dict(precision=64), dict(nc=2, storage=4)):
        args = dict(nc=3, dims=(4, 4, 4, 4), storage=12, precision=32)
        args.update(kw)
        with sunlib.Lattice(args["nc"], args["dims"], 6.0, hot_start=True, seed=4, storage=args["storage"],
                            precision=args["precision"]) as B:
            before = B.export_links()
            with pytest.raises(sunlib.SunError):
                B.load(path)
            assert np.array_equal(B.export_links(), before)


def test_damaged_file_leaves_the_lattice_unchanged(sunlib, tmp_path):
    path = tmp_path / "b.cfg"
    with sunlib.Lattice(3, (4, 4, 4, 4), 6.0, hot_start=True, seed=5) as A:
        A.save(path)
    data = bytearray(open(path, "rb").read())
    data[200] ^= 0x40  # one bit of the payload
    open(path, "wb").write(bytes(data))
    with sunlib.Lattice(3, (4, 4, 4, 4), 6.0, hot_start=True, seed=6) as B:
        before = B.export_links()
        step = B.heatbath_step
        with pytest.raises(sunlib.SunError):
            B.load(path)
        assert np.array_equal(B.export_links(), before) and B.heatbath_step == step


@pytest.mark.parametrize("nc,st,prec", CASES)
def test_compact_host_format(sunlib, nc, st, prec):
    """sun_export_stored: the stored rows of the canonical export in the storage
    precision; pinned and pageable buffers agree, in both formats (pinned memory
    is read and written in place, pageable memory read in place where the device
    reaches it through the host's page tables and written through the staging
    buffer); the round trips are exact."""
    import torch
    dims = (4, 4, 4, 6)
    rows = st // (2 * nc)
    with sunlib.Lattice(nc, dims, beta_for(nc), hot_start=True, seed=8, storage=st, precision=prec) as L:
        L.run(1, 1, 1)
        U = L.export_links()
        raw = L.export_stored()
        vals = raw.view(np.float32 if prec == 32 else np.float64).reshape(4, dims[3], dims[2], dims[1], dims[0],
                                                                          rows, nc, 2)
        want = np.stack([U[..., :rows, :].real, U[..., :rows, :].imag], axis=-1)
        assert np.array_equal(vals, want.astype(vals.dtype))
        pinned = torch.empty(raw.nbytes, dtype=torch.uint8).pin_memory()
        L.export_stored_raw(pinned.data_ptr(), raw.nbytes)
        assert np.array_equal(pinned.numpy(), raw)
        L.run(1, 1, 1)  # move away, then restore from each buffer
        L.import_stored(raw)
        assert np.array_equal(L.export_links(), U)
        L.run(1, 1, 1)
        L.import_stored_raw(pinned.data_ptr(), raw.nbytes)
        assert np.array_equal(L.export_links(), U)
        canon = torch.empty(U.nbytes, dtype=torch.uint8).pin_memory()
        L.export_links_raw(canon.data_ptr(), 2 * U.size)
        assert np.array_equal(canon.numpy().view(np.complex128).reshape(U.shape), U)
        L.run(1, 1, 1)
        L.import_links_raw(canon.data_ptr(), 2 * U.size)
        assert np.array_equal(L.export_links(), U)
        L.run(1, 1, 1)
        L.import_links(U)
        assert np.array_equal(L.export_links(), U)


@pytest.mark.parametrize("nc,st,prec", [(3, 12, 64), (3, 18, 64), (2, 4, 64), (4, 32, 64), (3, 12, 32),
                                        (2, 4, 32)])
def test_loaded_configuration_follows_the_oracle(sunlib, tmp_path, nc, st, prec):
    """A file written from the oracle's links (loaded into a lattice with
    heatbath step 3) holds exactly those links (rounded to FP32 for FP32
    lattices) in the rows the storage keeps; loaded into a fresh lattice of
    another seed, beta and start, the chain continues as the oracle does from
    the same links and state: FP64, one sweep of 1 heatbath + 2
    overrelaxation steps with the re-unitarization, links to 1e-11; FP32, one
    overrelaxation pass (1e-5) and, from the file again, one heatbath pass
    (1e-5 where the accept branch agrees, no flips at this size)."""
    import oracle as orc
    from tests.oracle_configs import cold_thermal
    dims = (4, 4, 6, 4)
    beta, seed, step = beta_for(nc), 21, 3
    U = cold_thermal(nc, dims, beta)
    path = tmp_path / "oracle.cfg"
    with sunlib.Lattice(nc, dims, beta, seed=seed, storage=st, precision=prec) as A:
        A.import_links(U)
        A.heatbath_step = step
        A.save(path)
    rows = st // (2 * nc)
    payload = np.fromfile(str(path), dtype=np.uint8)[128:].view(np.complex128 if prec == 64 else np.complex64)
    want_rows = U[..., :rows, :].astype(np.complex128 if prec == 64 else np.complex64)
    assert np.array_equal(payload, want_rows.ravel())
    with sunlib.Lattice(nc, dims, 1.0, hot_start=False, seed=99, storage=st, precision=prec) as C:
        C.load(path)
        assert C.heatbath_step == step
        if prec == 64:
            C.sweep(1, 2)
            got = C.export_links()
            want = U.copy()
            orc.sweep(want, beta, 1, 2, True, seed, step)
            assert np.abs(got - want).max() < 1e-11
        else:
            C.update_pass(sunlib.OVERRELAX, 1, 0)
            got = C.export_links()
            want = U.copy()
            orc.update_pass(want, beta, orc.OVERRELAX, 1, 0, step, seed)
            assert np.abs(got - want).max() < 1e-5
            C.load(path)
            C.update_pass(sunlib.HEATBATH, 2, 1)
            got = C.export_links()
            want = U.copy()
            orc.update_pass(want, beta, orc.HEATBATH, 2, 1, step, seed)
            assert np.abs(got - want).max() < 1e-5
