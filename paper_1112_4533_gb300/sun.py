"""Python binding of the SU(Nc) link-sweep C ABI (include/sun.h).

Argument marshalling only: every step of the sweep runs in libsun.so's CUDA
kernels.  PyTorch supplies the device memory (one uint8 tensor per lattice,
passed as the caller-owned device buffer) and the CUDA stream.  There is no CPU
fallback: if libsun.so is missing, importing the library raises.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libsun.so")

HEATBATH = 0
OVERRELAX = 1

OK = 0
_STATUS = {0: "ok", 1: "invalid argument", 2: "out of device memory", 3: "CUDA error",
           4: "device wait timed out", 5: "unsupported combination", 6: "invalid state"}


class SunError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("storage", ctypes.c_int), ("reunit_every", ctypes.c_int),
                ("block_threads", ctypes.c_int), ("stream", ctypes.c_void_p), ("device_buf", ctypes.c_void_p),
                ("device_buf_bytes", ctypes.c_size_t), ("use_graphs", ctypes.c_int), ("variant", ctypes.c_int),
                ("reunit_mode", ctypes.c_int), ("wave_lag", ctypes.c_int), ("wave_skip_units", ctypes.c_int),
                ("graph_sweeps", ctypes.c_int)]


class LatticeInfo(ctypes.Structure):
    _fields_ = [("nc", ctypes.c_int), ("precision", ctypes.c_int), ("storage", ctypes.c_int),
                ("reserved", ctypes.c_int), ("dims", ctypes.c_int * 4), ("beta", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("link_bytes", ctypes.c_size_t), ("links_bytes", ctypes.c_size_t),
                ("footprint", ctypes.c_size_t), ("links", ctypes.c_void_p), ("stream", ctypes.c_void_p)]


_lib = None

# every entry point of include/sun.h: (name, restype, argtypes)
_P = ctypes.c_void_p
_I4 = ctypes.POINTER(ctypes.c_int)
_D = ctypes.POINTER(ctypes.c_double)
class ConfigHeader(ctypes.Structure):
    _fields_ = [("version", ctypes.c_uint32), ("nc", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("storage", ctypes.c_int32), ("dims", ctypes.c_int32 * 4), ("beta", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("heatbath_step", ctypes.c_uint64), ("sweeps_done", ctypes.c_uint64),
                ("payload_bytes", ctypes.c_uint64), ("checksum", ctypes.c_uint64), ("reserved", ctypes.c_uint8 * 40)]


SIGNATURES = [
    ("sun_abi_version", ctypes.c_int, []),
    ("sun_options_init", None, [ctypes.POINTER(Options)]),
    ("sun_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("sun_last_error", ctypes.c_char_p, []),
    ("sun_footprint_bytes", ctypes.c_size_t, [ctypes.c_int, _I4, ctypes.POINTER(Options)]),
    ("sun_lattice_create", ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, _I4, ctypes.c_double, ctypes.c_int,
                                          ctypes.c_uint64, ctypes.POINTER(Options)]),
    ("sun_lattice_destroy", None, [_P]),
    ("sun_update_pass", ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    ("sun_update_pass_reunit", ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    ("sun_sweep", ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
    ("sun_run", ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D]),
    ("sun_reunitarize", ctypes.c_int, [_P]),
    ("sun_plaquette", ctypes.c_int, [_P, _D]),
    ("sun_polyakov_loop", ctypes.c_int, [_P, _D, _D]),
    ("sun_export_links", ctypes.c_int, [_P, _D, ctypes.c_size_t]),
    ("sun_import_links", ctypes.c_int, [_P, _D, ctypes.c_size_t]),
    ("sun_get_heatbath_step", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64)]),
    ("sun_set_heatbath_step", ctypes.c_int, [_P, ctypes.c_uint64]),
    ("sun_set_beta", ctypes.c_int, [_P, ctypes.c_double]),
    ("sun_synchronize", ctypes.c_int, [_P]),
    ("sun_get_info", ctypes.c_int, [_P, ctypes.POINTER(LatticeInfo)]),
    ("sun_plaquette_noalloc", ctypes.c_int, [_P, ctypes.c_int, _I4, ctypes.c_int, ctypes.c_int, _D, _P]),
    ("sun_selftest_conversions", ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]),
    ("sun_batch_create", ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.c_int, _P, ctypes.c_int]),
    ("sun_batch_run", ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D]),
    ("sun_batch_destroy", None, [_P]),
    ("sun_check_links", ctypes.c_int, [_P, _D, _D, ctypes.POINTER(ctypes.c_uint64)]),
    ("sun_export_stored", ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    ("sun_import_stored", ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    ("sun_save_config", ctypes.c_int, [_P, ctypes.c_char_p]),
    ("sun_load_config", ctypes.c_int, [_P, ctypes.c_char_p]),
    ("sun_read_config_header", ctypes.c_int, [ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(ConfigHeader)]),
    ("sun_slabs_create", ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, _I4, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(Options)]),
    ("sun_slabs_destroy", None, [_P]),
    ("sun_slabs_run", ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D]),
    ("sun_slabs_export_links", ctypes.c_int, [_P, _D, ctypes.c_size_t]),
    ("sun_slabs_import_links", ctypes.c_int, [_P, _D, ctypes.c_size_t]),
    ("sun_autotune", ctypes.c_int, [ctypes.c_int, _I4, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(Options), _D]),
    ("sun_autotune_batch", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                          _D, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Options),
                                          _D]),
]

TUNE_STORAGE, TUNE_REUNIT_MODE, TUNE_TWO_ROW = 1, 2, 4


def load_library(path=None):
    """Load libsun.so (raises OSError if it was not built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise OSError(f"{p} not found: build it with paper_1112_4533_gb300.build.build()")
    L = ctypes.CDLL(p)
    for name, res, args in SIGNATURES:
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = L
    return L


def _check(status):
    if status != OK:
        msg = load_library().sun_last_error()
        raise SunError(status, msg.decode() if msg else "")


def _dims(dims):
    if len(dims) != 4:
        raise ValueError("dims must be (Nx, Ny, Nz, Nt)")
    return (ctypes.c_int * 4)(*[int(d) for d in dims])


def _options(precision=32, storage=0, reunit_every=1, block_threads=0, stream=None, device_buf=None,
             device_buf_bytes=0, use_graphs=True, variant=0, reunit_mode=0, wave_lag=0, wave_skip_units=0,
             graph_sweeps=0):
    o = Options()
    load_library().sun_options_init(ctypes.byref(o))
    o.precision = int(precision)
    o.storage = int(storage)
    o.reunit_every = int(reunit_every)
    o.block_threads = int(block_threads)
    o.stream = stream
    o.device_buf = device_buf
    o.device_buf_bytes = int(device_buf_bytes)
    o.use_graphs = 1 if use_graphs else 0
    o.variant = int(variant)
    o.reunit_mode = int(reunit_mode)
    o.wave_lag = int(wave_lag)
    o.wave_skip_units = int(wave_skip_units)
    o.graph_sweeps = int(graph_sweeps)
    return o


def _tuned(o, ms):
    return {"storage": o.storage, "block_threads": o.block_threads, "variant": o.variant,
            "reunit_mode": o.reunit_mode, "graph_sweeps": o.graph_sweeps, "ms_per_sweep": ms.value}


def autotune(nc, dims, beta, n_heatbath=1, n_overrelax=4, precision=32, storage=0, reunit_mode=0,
             tune_storage=True, tune_reunit_mode=False, two_row=False, use_graphs=True):
    """Measured kernel configuration for one lattice (sun_autotune): a dict of
    Lattice keyword arguments (storage, block_threads, variant, reunit_mode)
    plus ms_per_sweep of the winner."""
    flags = (TUNE_STORAGE if tune_storage else 0) | (TUNE_REUNIT_MODE if tune_reunit_mode else 0) | \
        (TUNE_TWO_ROW if two_row else 0)
    o = _options(precision, storage, use_graphs=use_graphs, reunit_mode=reunit_mode)
    ms = ctypes.c_double(0.0)
    _check(load_library().sun_autotune(int(nc), _dims(dims), float(beta), int(n_heatbath), int(n_overrelax), flags,
                                       ctypes.byref(o), ctypes.byref(ms)))
    return _tuned(o, ms)


def autotune_batch(chains, n_heatbath=1, n_overrelax=4, precision=32, storage=0, reunit_mode=0,
                   tune_storage=True, tune_reunit_mode=False, two_row=False, use_graphs=True):
    """Measured configuration shared by a batch (sun_autotune_batch); chains is a
    list of (nc, dims, beta).  Returns the dict of autotune()."""
    n = len(chains)
    ncs = (ctypes.c_int * n)(*[int(c[0]) for c in chains])
    dims = (ctypes.c_int * (4 * n))(*[int(d) for c in chains for d in c[1]])
    betas = np.array([float(c[2]) for c in chains], dtype=np.float64)
    flags = (TUNE_STORAGE if tune_storage else 0) | (TUNE_REUNIT_MODE if tune_reunit_mode else 0) | \
        (TUNE_TWO_ROW if two_row else 0)
    o = _options(precision, storage, use_graphs=use_graphs, reunit_mode=reunit_mode)
    ms = ctypes.c_double(0.0)
    _check(load_library().sun_autotune_batch(n, ncs, dims, _dptr(betas), int(n_heatbath), int(n_overrelax), flags,
                                             ctypes.byref(o), ctypes.byref(ms)))
    return _tuned(o, ms)


def read_config_header(path, verify=True):
    """Header of a configuration file (sun_read_config_header) as a dict; with
    verify the payload size and checksum are checked too.  Needs no GPU."""
    h = ConfigHeader()
    _check(load_library().sun_read_config_header(os.fsencode(path), int(bool(verify)), ctypes.byref(h)))
    return {"version": h.version, "nc": h.nc, "precision": h.precision, "storage": h.storage,
            "dims": tuple(h.dims), "beta": h.beta, "seed": h.seed, "heatbath_step": h.heatbath_step,
            "sweeps_done": h.sweeps_done, "payload_bytes": h.payload_bytes, "checksum": h.checksum}


def footprint_bytes(nc, dims, precision=32, storage=0):
    """Device bytes a lattice needs (0 if the arguments are invalid)."""
    o = _options(precision, storage)
    return int(load_library().sun_footprint_bytes(int(nc), _dims(dims), ctypes.byref(o)))


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Lattice:
    """One SU(Nc) gauge configuration resident on the GPU.

    Device memory is a torch uint8 tensor owned by this object; work is
    enqueued on `stream` (a torch.cuda.Stream; a new one by default).
    """

    def __init__(self, nc, dims, beta, hot_start=False, seed=1, precision=32, storage=0, reunit_every=1,
                 block_threads=0, stream=None, use_graphs=True, device=None, variant=0, reunit_mode=0,
                 wave_lag=0, wave_skip_units=0, graph_sweeps=0):
        import torch  # device memory and streams only

        self.nc = int(nc)
        self.dims = tuple(int(d) for d in dims)
        self._lib = load_library()
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=dev)
        nbytes = footprint_bytes(nc, dims, precision, storage)
        if nbytes == 0:
            # let the library report what is wrong
            o = _options(precision, storage, reunit_every, block_threads)
            h = ctypes.c_void_p()
            _check(self._lib.sun_lattice_create(ctypes.byref(h), int(nc), _dims(dims), float(beta),
                                                int(bool(hot_start)), int(seed), ctypes.byref(o)))
            raise SunError(1, "invalid lattice arguments")
        with torch.cuda.device(dev):
            self._buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        base = self._buf.data_ptr()
        aligned = (base + 255) // 256 * 256
        o = _options(precision, storage, reunit_every, block_threads, ctypes.c_void_p(self.stream.cuda_stream),
                     ctypes.c_void_p(aligned), nbytes, use_graphs, variant, reunit_mode, wave_lag,
                     wave_skip_units, graph_sweeps)
        # the tensor's memory must be usable on our stream
        self.stream.wait_stream(torch.cuda.current_stream(dev))
        h = ctypes.c_void_p()
        with torch.cuda.device(dev):
            _check(self._lib.sun_lattice_create(ctypes.byref(h), int(nc), _dims(dims), float(beta),
                                                int(bool(hot_start)), int(seed), ctypes.byref(o)))
        self._h = h
        info = self.info()
        self.precision = info.precision
        self.storage = info.storage
        self.footprint = info.footprint
        self.links_bytes = info.links_bytes
        self.link_bytes = info.link_bytes
        self.volume = self.dims[0] * self.dims[1] * self.dims[2] * self.dims[3]

    # -- lifecycle
    def close(self):
        if getattr(self, "_h", None):
            self._lib.sun_lattice_destroy(self._h)
            self._h = None
            self._buf = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        if not self._h:
            raise SunError(6, "lattice is closed")
        return self._h

    # -- the method
    def update_pass(self, mode, mu, parity):
        _check(self._lib.sun_update_pass(self.handle, int(mode), int(mu), int(parity)))

    def update_pass_reunit(self, mode, mu, parity):
        """update_pass with each updated link re-unitarized in FP64 inside the kernel."""
        _check(self._lib.sun_update_pass_reunit(self.handle, int(mode), int(mu), int(parity)))

    def sweep(self, n_heatbath=1, n_overrelax=4):
        _check(self._lib.sun_sweep(self.handle, int(n_heatbath), int(n_overrelax)))

    def run(self, n_sweeps, n_heatbath=1, n_overrelax=4, plaquette=True, polyakov=True):
        """n_sweeps sweeps with the observables measured after each; returns
        (plaquette history, complex Polyakov history) as numpy arrays (None if not asked)."""
        n = int(n_sweeps)
        ph = np.zeros(n) if plaquette else None
        lh = np.zeros(2 * n) if polyakov else None
        _check(self._lib.sun_run(self.handle, n, int(n_heatbath), int(n_overrelax),
                                 _dptr(ph) if ph is not None else None, _dptr(lh) if lh is not None else None))
        poly = lh[0::2] + 1j * lh[1::2] if lh is not None else None
        return ph, poly

    def reunitarize(self):
        _check(self._lib.sun_reunitarize(self.handle))

    def plaquette(self):
        v = ctypes.c_double()
        _check(self._lib.sun_plaquette(self.handle, ctypes.byref(v)))
        return v.value

    def polyakov_loop(self):
        re, im = ctypes.c_double(), ctypes.c_double()
        _check(self._lib.sun_polyakov_loop(self.handle, ctypes.byref(re), ctypes.byref(im)))
        return complex(re.value, im.value)

    # -- state
    def export_links(self, out=None):
        """Links in canonical order as complex128 (4, Nt, Nz, Ny, Nx, nc, nc)."""
        nx, ny, nz, nt = self.dims
        shape = (4, nt, nz, ny, nx, self.nc, self.nc)
        if out is None:
            out = np.empty(shape, dtype=np.complex128)
        assert out.dtype == np.complex128 and out.flags.c_contiguous and out.shape == shape
        flat = out.view(np.float64).reshape(-1)
        _check(self._lib.sun_export_links(self.handle, _dptr(flat), flat.size))
        return out

    def import_links(self, U):
        a = np.ascontiguousarray(U, dtype=np.complex128)
        flat = a.view(np.float64).reshape(-1)
        _check(self._lib.sun_import_links(self.handle, _dptr(flat), flat.size))

    def export_links_raw(self, host_ptr, n_doubles):
        """Export into caller memory given as an address (e.g. a pinned torch tensor)."""
        _check(self._lib.sun_export_links(self.handle, ctypes.cast(host_ptr, _D), int(n_doubles)))

    def import_links_raw(self, host_ptr, n_doubles):
        _check(self._lib.sun_import_links(self.handle, ctypes.cast(host_ptr, _D), int(n_doubles)))

    @property
    def heatbath_step(self):
        v = ctypes.c_uint64()
        _check(self._lib.sun_get_heatbath_step(self.handle, ctypes.byref(v)))
        return v.value

    @heatbath_step.setter
    def heatbath_step(self, step):
        _check(self._lib.sun_set_heatbath_step(self.handle, int(step)))

    def check_links(self):
        """(max |U U^+ - 1|, max |det U - 1|, non-finite link count) over all links (sun_check_links)."""
        dev, det = ctypes.c_double(), ctypes.c_double()
        bad = ctypes.c_uint64()
        _check(self._lib.sun_check_links(self.handle, ctypes.byref(dev), ctypes.byref(det), ctypes.byref(bad)))
        return dev.value, det.value, int(bad.value)

    def export_stored(self, out=None):
        """The compact host format (sun_export_stored): a uint8 array of links_bytes."""
        if out is None:
            out = np.empty(self.links_bytes, dtype=np.uint8)
        assert out.flags.c_contiguous and out.nbytes == self.links_bytes
        _check(self._lib.sun_export_stored(self.handle, out.ctypes.data_as(ctypes.c_void_p), out.nbytes))
        return out

    def import_stored(self, buf):
        a = np.ascontiguousarray(buf).view(np.uint8).reshape(-1)
        _check(self._lib.sun_import_stored(self.handle, a.ctypes.data_as(ctypes.c_void_p), a.nbytes))

    def export_stored_raw(self, host_ptr, nbytes):
        _check(self._lib.sun_export_stored(self.handle, ctypes.c_void_p(host_ptr), int(nbytes)))

    def import_stored_raw(self, host_ptr, nbytes):
        _check(self._lib.sun_import_stored(self.handle, ctypes.c_void_p(host_ptr), int(nbytes)))

    def save(self, path):
        """Write links and chain state to a configuration file (sun_save_config)."""
        _check(self._lib.sun_save_config(self.handle, os.fsencode(path)))

    def load(self, path):
        """Resume the chain stored in a configuration file (sun_load_config)."""
        _check(self._lib.sun_load_config(self.handle, os.fsencode(path)))

    def set_beta(self, beta):
        _check(self._lib.sun_set_beta(self.handle, float(beta)))

    def synchronize(self):
        _check(self._lib.sun_synchronize(self.handle))

    def info(self):
        i = LatticeInfo()
        _check(self._lib.sun_get_info(self.handle, ctypes.byref(i)))
        return i


def lattice_create(nc, dims, beta, hot_start=False, seed=1, **kw):
    """Same as sun_lattice_create: returns a Lattice."""
    return Lattice(nc, dims, beta, hot_start=hot_start, seed=seed, **kw)


class Batch:
    """Independent lattices swept together (sun_batch_*): one kernel launch per
    pass for all chains of equal (Nc, storage, precision), groups overlapping on
    their own streams.  The lattices must stay open while the batch lives."""

    def __init__(self, lattices, stream=None, use_graphs=True):
        self._lib = load_library()
        self.lattices = list(lattices)
        arr = (ctypes.c_void_p * len(self.lattices))(*[L.handle.value for L in self.lattices])
        h = ctypes.c_void_p()
        s = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
        _check(self._lib.sun_batch_create(ctypes.byref(h), arr, len(self.lattices), s, 1 if use_graphs else 0))
        self._h = h

    @property
    def n(self):
        return len(self.lattices)

    def run(self, n_sweeps, n_heatbath=1, n_overrelax=4, plaquette=True, polyakov=True):
        """Returns (plaquette [n_sweeps, n], Polyakov [n_sweeps, n] complex), None if not asked."""
        ns, n = int(n_sweeps), self.n
        ph = np.zeros((ns, n)) if plaquette else None
        lh = np.zeros((ns, n, 2)) if polyakov else None
        _check(self._lib.sun_batch_run(self._h, ns, int(n_heatbath), int(n_overrelax),
                                       _dptr(ph) if ph is not None else None,
                                       _dptr(lh) if lh is not None else None))
        return ph, (lh[..., 0] + 1j * lh[..., 1] if lh is not None else None)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sun_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Slabs:
    """A lattice cut into n_slabs t-slabs with halo exchange after every pass
    (sun_slabs_*): the same chain as one Lattice with the same seed."""

    def __init__(self, nc, dims, n_slabs, beta, hot_start=False, seed=1, precision=32, storage=0, reunit_every=1,
                 block_threads=0, use_graphs=True, variant=0, reunit_mode=0):
        import torch  # streams only
        self.nc = int(nc)
        self.dims = tuple(int(d) for d in dims)
        self.n_slabs = int(n_slabs)
        self._lib = load_library()
        self.stream = torch.cuda.Stream()
        o = _options(precision, storage, reunit_every, block_threads, ctypes.c_void_p(self.stream.cuda_stream),
                     None, 0, use_graphs, variant, reunit_mode)
        h = ctypes.c_void_p()
        _check(self._lib.sun_slabs_create(ctypes.byref(h), self.nc, _dims(dims), self.n_slabs, float(beta),
                                          int(bool(hot_start)), int(seed), ctypes.byref(o)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sun_slabs_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def run(self, n_sweeps, n_heatbath=1, n_overrelax=4, plaquette=True, polyakov=True):
        plaq = np.zeros(n_sweeps) if plaquette else None
        poly = np.zeros(2 * n_sweeps) if polyakov else None
        _check(self._lib.sun_slabs_run(self._h, int(n_sweeps), int(n_heatbath), int(n_overrelax),
                                       _dptr(plaq) if plaquette else None, _dptr(poly) if polyakov else None))
        return plaq, (poly[0::2] + 1j * poly[1::2]) if polyakov else None

    def export_links(self):
        nx, ny, nz, nt = self.dims
        out = np.empty((4, nt, nz, ny, nx, self.nc, self.nc), dtype=np.complex128)
        flat = out.view(np.float64).reshape(-1)
        _check(self._lib.sun_slabs_export_links(self._h, _dptr(flat), flat.size))
        return out

    def import_links(self, U):
        a = np.ascontiguousarray(U, dtype=np.complex128)
        flat = a.view(np.float64).reshape(-1)
        _check(self._lib.sun_slabs_import_links(self._h, _dptr(flat), flat.size))
