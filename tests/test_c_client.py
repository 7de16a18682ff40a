"""The C ABI used from a plain C program (tests/c_client/sweep_client.c): no
Python, no PyTorch on its path.  On the CPU the public header compiles as
strict C11 and as C++ and the client links against libsun.so; on the GPU the
client's plaquette and Polyakov histories and final links are bitwise those of
the Python binding for the same seed (library-owned memory and stream against
caller-owned ones)."""
import os
import shutil
import subprocess

import numpy as np
import pytest


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CLIENT = os.path.join(ROOT, "tests", "c_client", "sweep_client.c")
INCLUDE = os.path.join(ROOT, "include")


def _cc():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    return cc


def build_client(out_dir):
    from paper_1112_4533_gb300 import build as b
    lib = b.build()
    libdir = os.path.dirname(lib)
    exe = os.path.join(str(out_dir), "sweep_client")
    cmd = [_cc(), "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic", "-O1", "-I" + INCLUDE, CLIENT,
           "-L" + libdir, "-lsun", "-Wl,-rpath," + libdir, "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_header_compiles_as_c_and_cxx(tmp_path):
    src = tmp_path / "h.c"
    src.write_text('#include "sun.h"\nint main(void) { sun_options o; sun_options_init(&o); return o.variant; }\n')
    for cc, std in ((_cc(), "-std=c99"), (shutil.which("g++") or "g++", "-std=c++11")):
        lang = ["-x", "c++"] if "++" in cc else []
        r = subprocess.run([cc] + lang + [std, "-Wall", "-Wextra", "-Werror", "-pedantic", "-fsyntax-only",
                                          "-I" + INCLUDE, str(src)], capture_output=True, text=True)
        assert r.returncode == 0, (cc, r.stderr)


def test_client_compiles_and_links(tmp_path):
    exe = build_client(tmp_path)
    assert os.access(exe, os.X_OK)


def test_client_usage_error_without_gpu_work(tmp_path):
    exe = build_client(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 1 and "usage" in r.stderr


@pytest.mark.gpu
@pytest.mark.parametrize("nc,dims,beta,seed", [
    (3, (8, 6, 4, 6), 6.0, 31),
    (2, (6, 6, 6, 8), 2.3, 7),
    (4, (4, 4, 4, 6), 11.0, 3),
])
def test_client_matches_the_python_binding(tmp_path, nc, dims, beta, seed):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    exe = build_client(tmp_path)
    sweeps, n_hb, n_or = 3, 1, 3
    out = tmp_path / "out.bin"
    r = subprocess.run([exe, str(nc)] + [str(d) for d in dims] +
                       [repr(beta), str(seed), str(sweeps), str(n_hb), str(n_or), str(out)],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    raw = np.fromfile(str(out), dtype=np.float64)
    nx, ny, nz, nt = dims
    n_links = 8 * nc * nc * nx * ny * nz * nt
    assert raw.size == 3 * sweeps + n_links
    plaq_c, poly_c = raw[:sweeps], raw[sweeps:3 * sweeps]
    links_c = raw[3 * sweeps:].view(np.complex128).reshape(4, nt, nz, ny, nx, nc, nc)

    import paper_1112_4533_gb300 as p
    p.load_library()
    with p.Lattice(nc, dims, beta, hot_start=True, seed=seed) as L:
        plaq, poly = L.run(sweeps, n_hb, n_or)
        links = L.export_links()
    assert np.array_equal(plaq_c, plaq)
    assert np.array_equal(poly_c[0::2], poly.real) and np.array_equal(poly_c[1::2], poly.imag)
    assert np.array_equal(links_c, links)
