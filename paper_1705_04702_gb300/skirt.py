"""Thin ctypes binding of libskirt (include/skirt.h).

Argument marshalling only: every step of the photon-packet life cycle runs in
the library's CUDA kernels.  PyTorch provides device memory and streams.
Importing this module loads ``lib/libskirt.so`` and raises ImportError if it
has not been built -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libskirt.so")

# status codes
OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_EVENT_CAP, ERR_NONFINITE, ERR_SOURCE, ERR_NO_DEVICE = range(8)
SRC_POINT, SRC_DISK, SRC_BEAM, SRC_DUST = range(4)
PREC_FP64, PREC_MIXED = 0, 1
SCHED_PER_LAMBDA, SCHED_PERSISTENT = 0, 1
REC_FIELDS = 8

_dp = ctypes.POINTER(ctypes.c_double)


class skirt_source(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("pos", ctypes.c_double * 3), ("dir", ctypes.c_double * 3),
                ("h_R", ctypes.c_double), ("h_z", ctypes.c_double), ("emission", ctypes.c_void_p)]


class skirt_wavelengths(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("kscale", _dp), ("albedo", _dp), ("g", _dp), ("lsrc", _dp)]


class skirt_instrument(ctypes.Structure):
    _fields_ = [("distance", ctypes.c_double), ("inclination_deg", ctypes.c_double),
                ("azimuth_deg", ctypes.c_double), ("fov", ctypes.c_double), ("npx", ctypes.c_int)]


class skirt_trace_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("schedule", ctypes.c_int), ("w_min", ctypes.c_double),
                ("max_events", ctypes.c_int), ("peel", ctypes.c_int), ("accumulate", ctypes.c_int),
                ("block", ctypes.c_int), ("chunk", ctypes.c_int), ("blocks_per_sm", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("step_min", ctypes.c_int), ("phase", ctypes.c_uint32),
                ("nrec", ctypes.c_int),
                ("records", ctypes.c_void_p),
                ("first_packet", ctypes.POINTER(ctypes.c_uint64)),
                ("total_packets", ctypes.POINTER(ctypes.c_uint64))]


TUNE_MAX_POINTS = 256


class skirt_tune_point(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int), ("chunk", ctypes.c_int), ("blocks_per_sm", ctypes.c_int),
                ("step_min", ctypes.c_int), ("ms", ctypes.c_float), ("ms_confirm", ctypes.c_float)]


class skirt_tune_report(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("chosen", ctypes.c_int), ("repeats", ctypes.c_int),
                ("sample_packets", ctypes.c_ulonglong), ("confirm_packets", ctypes.c_ulonglong),
                ("points", skirt_tune_point * TUNE_MAX_POINTS)]

    def as_dict(self):
        pts = [{k: getattr(self.points[i], k) for k, _ in skirt_tune_point._fields_} for i in range(self.n)]
        return {"n": self.n, "chosen": self.chosen, "repeats": self.repeats, "sample_packets": self.sample_packets,
                "confirm_packets": self.confirm_packets, "points": pts}


class skirt_ledger(ctypes.Structure):
    _fields_ = [("emitted", ctypes.c_double), ("absorbed", ctypes.c_double), ("escaped", ctypes.c_double),
                ("residual", ctypes.c_double), ("scatterings", ctypes.c_double),
                ("deposit_steps", ctypes.c_double), ("locate_steps", ctypes.c_double),
                ("peel_steps", ctypes.c_double), ("status_bits", ctypes.c_int), ("kernel_ms", ctypes.c_float)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libskirt.so is not built ({LIB_PATH}); run paper_1705_04702_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64
    L.skirt_last_error.restype = ctypes.c_char_p
    L.skirt_last_error.argtypes = []
    L.skirt_version.restype = ctypes.c_char_p
    L.skirt_version.argtypes = []
    L.skirt_trace_opts_default.argtypes = [ctypes.POINTER(skirt_trace_opts)]
    L.skirt_trace_opts_default.restype = i
    L.skirt_grid_create.argtypes = [ctypes.POINTER(vp), i, i, i, _dp, vp]
    L.skirt_grid_create.restype = i
    L.skirt_octree_create.argtypes = [ctypes.POINTER(vp), i, _dp, ctypes.c_longlong, vp, vp]
    L.skirt_octree_create.restype = i
    L.skirt_grid_destroy.argtypes = [vp]
    L.skirt_grid_destroy.restype = i
    L.skirt_trace.argtypes = [vp, ctypes.POINTER(skirt_source), ctypes.POINTER(skirt_wavelengths),
                              ctypes.POINTER(u64), u64, ctypes.POINTER(skirt_instrument), i,
                              ctypes.POINTER(skirt_trace_opts), vp, vp, vp, ctypes.POINTER(skirt_ledger),
                              _dp, vp]
    L.skirt_trace.restype = i
    L.skirt_autotune.argtypes = [vp, ctypes.POINTER(skirt_source), ctypes.POINTER(skirt_wavelengths),
                                 ctypes.POINTER(u64), u64, ctypes.POINTER(skirt_instrument), i,
                                 ctypes.POINTER(skirt_trace_opts), ctypes.c_double, i, vp, vp, vp,
                                 ctypes.POINTER(skirt_tune_report), vp]
    L.skirt_autotune.restype = i
    L.skirt_microbench.argtypes = [i, ctypes.c_longlong, _dp, ctypes.POINTER(ctypes.c_float)]
    L.skirt_philox4x32_10.argtypes = [vp, vp, vp, i]
    L.skirt_philox4x32_10.restype = i
    L.skirt_microbench.restype = i
    return L


lib = _load()


class SkirtError(RuntimeError):
    def __init__(self, code, where):
        msg = lib.skirt_last_error().decode(errors="replace")
        super().__init__(f"{where} failed with status {code}: {msg}")
        self.code = code


def _check(code, where, allow=()):
    if code != OK and code not in allow:
        raise SkirtError(code, where)
    return code


def _ptr(x):
    """Address of a torch tensor / numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    return ctypes.c_void_p(x.ctypes.data)


# --------------------------------------------------------------------- C names
def skirt_version() -> str:
    return lib.skirt_version().decode()


def skirt_trace_opts_default() -> skirt_trace_opts:
    o = skirt_trace_opts()
    _check(lib.skirt_trace_opts_default(ctypes.byref(o)), "skirt_trace_opts_default")
    return o


def skirt_grid_create(nx, ny, nz, bbox, kr):
    """kr: float32 torch tensor (CUDA or CPU) or numpy array of nx*ny*nz values."""
    h = ctypes.c_void_p()
    bb = (ctypes.c_double * 6)(*[float(v) for v in bbox])
    _check(lib.skirt_grid_create(ctypes.byref(h), int(nx), int(ny), int(nz), bb, _ptr(kr)), "skirt_grid_create")
    return h


def skirt_octree_create(max_level, bbox, leaves, kr):
    """leaves: int32 numpy array [nleaf, 4] (level, ix, iy, iz); kr: float32
    torch tensor (CUDA or CPU) or numpy array of nleaf values."""
    h = ctypes.c_void_p()
    bb = (ctypes.c_double * 6)(*[float(v) for v in bbox])
    lv = np.ascontiguousarray(leaves, dtype=np.int32)
    _check(lib.skirt_octree_create(ctypes.byref(h), int(max_level), bb, int(lv.shape[0]), _ptr(lv), _ptr(kr)),
           "skirt_octree_create")
    return h


def skirt_grid_destroy(h):
    _check(lib.skirt_grid_destroy(h), "skirt_grid_destroy")


def skirt_trace(grid, src: skirt_source, wl: skirt_wavelengths, npackets, seed, instruments, opts,
                absorbed, images, sed, stream=None, allow=(ERR_EVENT_CAP,)):
    """Marshals to skirt_trace; returns (status, ledger dict, per-wavelength
    ledger [n, 4])."""
    npk = np.ascontiguousarray(npackets, dtype=np.uint64)
    n = wl.n
    ins_arr = (skirt_instrument * max(len(instruments), 1))(*instruments)
    led = skirt_ledger()
    per = np.zeros((n, 4))
    st = None if stream is None else ctypes.c_void_p(int(stream))
    code = lib.skirt_trace(grid, ctypes.byref(src), ctypes.byref(wl),
                           npk.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), int(seed) & (2 ** 64 - 1),
                           ins_arr, len(instruments), ctypes.byref(opts), _ptr(absorbed), _ptr(images), _ptr(sed),
                           ctypes.byref(led), per.ctypes.data_as(_dp), st)
    _check(code, "skirt_trace", allow)
    return code, led.as_dict(), per


def skirt_autotune(grid, src, wl, npackets, seed, instruments, opts, sample_fraction, absorbed, images, sed,
                   stream=None, repeats=0):
    """Writes the tuned schedule into opts; returns the sweep report (dict)."""
    npk = np.ascontiguousarray(npackets, dtype=np.uint64)
    ins_arr = (skirt_instrument * max(len(instruments), 1))(*instruments)
    st = None if stream is None else ctypes.c_void_p(int(stream))
    rep = skirt_tune_report()
    code = lib.skirt_autotune(grid, ctypes.byref(src), ctypes.byref(wl),
                              npk.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), int(seed) & (2 ** 64 - 1),
                              ins_arr, len(instruments), ctypes.byref(opts), float(sample_fraction), int(repeats),
                              _ptr(absorbed), _ptr(images), _ptr(sed), ctypes.byref(rep), st)
    _check(code, "skirt_autotune", (ERR_EVENT_CAP,))
    return rep.as_dict()


def skirt_philox4x32_10(ctr, key):
    """ctr: uint32 [n, 4], key: uint32 [n, 2] -> the device generator's
    output blocks, uint32 [n, 4]."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, dtype=np.uint32).reshape(-1, 2)
    if c.shape[0] != k.shape[0]:
        raise ValueError("ctr and key must have the same number of rows")
    out = np.zeros_like(c)
    _check(lib.skirt_philox4x32_10(_ptr(c), _ptr(k), _ptr(out), int(c.shape[0])), "skirt_philox4x32_10")
    return out


def skirt_microbench(kind, size=0):
    """Returns (operations per second, kernel ms) of microbenchmark `kind`."""
    rate = ctypes.c_double()
    ms = ctypes.c_float()
    _check(lib.skirt_microbench(int(kind), int(size), ctypes.byref(rate), ctypes.byref(ms)), "skirt_microbench")
    return rate.value, ms.value


# ------------------------------------------------------- problem marshalling
class Tables:
    """Keeps the host arrays a skirt_wavelengths points into alive."""

    def __init__(self, wl):
        self.kscale = np.ascontiguousarray(wl.kscale, dtype=np.float64)
        self.albedo = np.ascontiguousarray(wl.albedo, dtype=np.float64)
        self.g = np.ascontiguousarray(wl.g, dtype=np.float64)
        self.lsrc = None if wl.lsrc is None else np.ascontiguousarray(wl.lsrc, dtype=np.float64)
        self.c = skirt_wavelengths(wl.n, self.kscale.ctypes.data_as(_dp), self.albedo.ctypes.data_as(_dp),
                                   self.g.ctypes.data_as(_dp),
                                   None if self.lsrc is None else self.lsrc.ctypes.data_as(_dp))


def make_source(s, emission=None) -> skirt_source:
    return skirt_source(int(s.kind), (ctypes.c_double * 3)(*s.pos), (ctypes.c_double * 3)(*s.dir),
                        float(s.h_R), float(s.h_z), None if emission is None else emission.data_ptr())


def make_instruments(instruments):
    return [skirt_instrument(float(i.distance), float(i.inclination), float(i.azimuth), float(i.fov), int(i.npx))
            for i in instruments]


class Grid:
    """Owns a skirt grid handle built from a workloads.Grid (or any object with
    nx, ny, nz, bbox, kr) or a workloads.Octree (max_level, bbox, leaves, kr)."""

    def __init__(self, grid, kr=None):
        import torch
        self.nx, self.ny, self.nz = grid.nx, grid.ny, grid.nz
        self.bbox = tuple(grid.bbox)
        self.octree = getattr(grid, "leaves", None) is not None
        self.ncell = grid.ncell if self.octree else grid.nx * grid.ny * grid.nz
        if kr is None:
            kr = torch.from_numpy(np.ascontiguousarray(grid.kr, dtype=np.float32).ravel())
        if self.octree:
            self.h = skirt_octree_create(grid.max_level, self.bbox, grid.leaves, kr)
        else:
            self.h = skirt_grid_create(self.nx, self.ny, self.nz, self.bbox, kr)

    def close(self):
        if self.h is not None and self.h.value:
            skirt_grid_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def packet_range_arrays(first_packet, total_packets):
    """uint64 arrays for skirt_trace_opts.first_packet / total_packets (None stays None)."""
    f = None if first_packet is None else np.ascontiguousarray(first_packet, dtype=np.uint64)
    t = None if total_packets is None else np.ascontiguousarray(total_packets, dtype=np.uint64)
    return f, t


def _u64p(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def run_problem(prob, grid: Grid | None = None, precision=PREC_MIXED, schedule=SCHED_PERSISTENT, nrec=0,
                use_graph=False, peel=True, block=0, chunk=0, blocks_per_sm=0, step_min=0, outputs=None, emission=None,
                device="cuda", stream=None, accumulate=False, first_packet=None, total_packets=None):
    """Traces a workloads.Problem on the GPU; returns a dict of torch tensors
    (absorbed [ncell, n], images list [npx, npx, n], sed [ninstr, n], records)
    plus ledger information.  first_packet / total_packets (per wavelength)
    select a packet range of the run, as in skirt_trace_opts."""
    import torch
    own = grid is None
    if own:
        grid = Grid(prob.grid)
    n = prob.wl.n
    tables = Tables(prob.wl)
    ins = make_instruments(prob.instruments)
    img_elems = sum(i.npx * i.npx for i in prob.instruments) * n
    if outputs is None:
        absorbed = torch.zeros((grid.ncell, n), dtype=torch.float64, device=device)
        images = torch.zeros(max(img_elems, 1), dtype=torch.float64, device=device)
        sed = torch.zeros((max(len(ins), 1), n), dtype=torch.float64, device=device)
    else:
        absorbed, images, sed = outputs
    records = torch.zeros((n, max(nrec, 1), REC_FIELDS), dtype=torch.float64, device=device) if nrec else None
    o = skirt_trace_opts_default()
    o.precision = precision
    o.schedule = schedule
    o.w_min = prob.w_min
    o.max_events = prob.max_events
    o.peel = 1 if peel else 0
    o.accumulate = 1 if accumulate else 0
    o.block = block
    o.chunk = chunk
    o.blocks_per_sm = blocks_per_sm
    o.step_min = step_min
    o.use_graph = 1 if use_graph else 0
    o.phase = prob.phase
    o.nrec = nrec
    o.records = records.data_ptr() if records is not None else None
    fp, tp = packet_range_arrays(first_packet, total_packets)
    o.first_packet = _u64p(fp)
    o.total_packets = _u64p(tp)
    src = make_source(prob.source, emission)
    code, led, per = skirt_trace(grid.h, src, tables.c, prob.npk, prob.seed, ins, o, absorbed, images, sed,
                                 stream=stream)
    imgs, off = [], 0
    for i in prob.instruments:
        k = i.npx * i.npx * n
        imgs.append(images[off:off + k].view(i.npx, i.npx, n))
        off += k
    out = {"absorbed": absorbed, "images": imgs, "images_flat": images[:off], "sed": sed[:len(ins)],
           "records": records[:, :nrec] if records is not None else None, "ledger": led,
           "ledger_per_lambda": per, "status": code}
    if own:
        grid.close()
    return out


# ------------------------------------------------------------ dust emission
EMIT_EXACT, EMIT_SURROGATE = 0, 1
NBANDS, NEMIT, MLP_HIDDEN = 32, 100, 128
MLP_NPARAM = 128 * 32 + 128 + 128 * 128 + 128 + 100 * 128 + 100


class skirt_mlp_train_opts(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int), ("batch", ctypes.c_int), ("lr", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("seed", ctypes.c_uint64), ("guard_quantile", ctypes.c_float)]


class skirt_emission_stats(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_ulonglong), ("n_fallback", ctypes.c_ulonglong),
                ("ms_features", ctypes.c_float), ("ms_surrogate", ctypes.c_float), ("ms_exact", ctypes.c_float)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


def _bind_emission(L):
    vp, i, ll, fp = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.POINTER(ctypes.c_float)
    L.skirt_emission_grid.argtypes = [_dp, _dp]
    L.skirt_dust_mass.argtypes = [vp, vp, vp]
    L.skirt_band_features.argtypes = [vp, ll, i, _dp, vp, vp, vp, vp]
    L.skirt_mlp_create.argtypes = [ctypes.POINTER(vp), ctypes.c_uint64]
    L.skirt_mlp_destroy.argtypes = [vp]
    L.skirt_mlp_set_params.argtypes = [vp, fp, fp, fp, fp, fp]
    L.skirt_mlp_get_params.argtypes = [vp, fp, fp, fp, fp, fp]
    L.skirt_mlp_set_guard.argtypes = [vp, ctypes.c_float]
    L.skirt_mlp_get_guard.argtypes = [vp, fp]
    L.skirt_mlp_train_opts_default.argtypes = [ctypes.POINTER(skirt_mlp_train_opts)]
    L.skirt_mlp_train.argtypes = [vp, vp, vp, ll, ctypes.POINTER(skirt_mlp_train_opts), fp, vp]
    L.skirt_mlp_grad.argtypes = [vp, vp, vp, i, fp, fp, vp]
    L.skirt_mlp_forward.argtypes = [vp, vp, vp, ll, vp, vp, vp]
    L.skirt_dust_emission.argtypes = [vp, ll, i, _dp, vp, i, vp, vp, vp, ctypes.POINTER(skirt_emission_stats), vp]
    L.skirt_dust_emission_exact_static.argtypes = [vp, ll, i, _dp, vp, vp, vp, vp]
    L.skirt_dust_emission_pair.argtypes = [vp, ll, i, _dp, vp, i, _dp, vp, vp, vp, vp]
    L.skirt_emission_totals.argtypes = [vp, vp, i, _dp, vp]
    for name in ("skirt_emission_grid", "skirt_dust_mass", "skirt_band_features", "skirt_mlp_create",
                 "skirt_mlp_destroy", "skirt_mlp_set_params", "skirt_mlp_get_params", "skirt_mlp_set_guard",
                 "skirt_mlp_get_guard", "skirt_mlp_train_opts_default",
                 "skirt_mlp_train", "skirt_mlp_grad", "skirt_mlp_forward", "skirt_dust_emission",
                 "skirt_dust_emission_exact_static", "skirt_dust_emission_pair", "skirt_emission_totals"):
        getattr(L, name).restype = i


_bind_emission(lib)


def _st(stream):
    return None if stream is None else ctypes.c_void_p(int(stream))


def _fp(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float32).ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def skirt_emission_grid():
    lam = np.zeros(NEMIT)
    W = np.zeros(NEMIT)
    _check(lib.skirt_emission_grid(lam.ctypes.data_as(_dp), W.ctypes.data_as(_dp)), "skirt_emission_grid")
    return lam, W


def skirt_dust_mass(grid, mass, stream=None):
    _check(lib.skirt_dust_mass(grid, _ptr(mass), _st(stream)), "skirt_dust_mass")


def skirt_band_features(absorbed, ncell, n_in, lambda_in, mass, features, total, stream=None):
    lam = np.ascontiguousarray(lambda_in, dtype=np.float64)
    _check(lib.skirt_band_features(_ptr(absorbed), int(ncell), int(n_in), lam.ctypes.data_as(_dp), _ptr(mass),
                                   _ptr(features), _ptr(total), _st(stream)), "skirt_band_features")


def skirt_dust_emission(absorbed, ncell, n_in, lambda_in, mass, mode, net, emission, temperature=None, stream=None):
    lam = np.ascontiguousarray(lambda_in, dtype=np.float64)
    st = skirt_emission_stats()
    _check(lib.skirt_dust_emission(_ptr(absorbed), int(ncell), int(n_in), lam.ctypes.data_as(_dp), _ptr(mass),
                                   int(mode), None if net is None else net.h, _ptr(emission), _ptr(temperature),
                                   ctypes.byref(st), _st(stream)), "skirt_dust_emission")
    return st.as_dict()


def skirt_emission_totals(grid, emission, nlambda, stream=None):
    """Per-wavelength column sums (FP64, host) of a device emission table [ncell][nlambda]."""
    t = np.zeros(int(nlambda))
    _check(lib.skirt_emission_totals(grid, _ptr(emission), int(nlambda), t.ctypes.data_as(_dp), _st(stream)),
           "skirt_emission_totals")
    return t


def skirt_dust_emission_pair(absorbed_a, ncell, lambda_a, absorbed_b, lambda_b, mass, emission, temperature=None,
                             stream=None):
    """Exact emission from two absorbed tables (absorbed_b / lambda_b may be None)."""
    la = np.ascontiguousarray(lambda_a, dtype=np.float64)
    lb = None if lambda_b is None else np.ascontiguousarray(lambda_b, dtype=np.float64)
    _check(lib.skirt_dust_emission_pair(_ptr(absorbed_a), int(ncell), la.size, la.ctypes.data_as(_dp),
                                        _ptr(absorbed_b), 0 if lb is None else lb.size,
                                        None if lb is None else lb.ctypes.data_as(_dp), _ptr(mass), _ptr(emission),
                                        _ptr(temperature), _st(stream)), "skirt_dust_emission_pair")


def skirt_dust_emission_exact_static(absorbed, ncell, n_in, lambda_in, mass, emission, temperature=None, stream=None):
    """Exact emission that allocates no device memory (fixed 4096-wavelength working table)."""
    lam = np.ascontiguousarray(lambda_in, dtype=np.float64)
    _check(lib.skirt_dust_emission_exact_static(_ptr(absorbed), int(ncell), int(n_in), lam.ctypes.data_as(_dp),
                                                _ptr(mass), _ptr(emission), _ptr(temperature), _st(stream)),
           "skirt_dust_emission_exact_static")


class MLP:
    """Owns a skirt_mlp_t (the emission surrogate network)."""

    def __init__(self, seed=1):
        self.h = ctypes.c_void_p()
        _check(lib.skirt_mlp_create(ctypes.byref(self.h), int(seed)), "skirt_mlp_create")

    def close(self):
        if self.h is not None and self.h.value:
            lib.skirt_mlp_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params=None, x_mean=None, x_std=None, hull_lo=None, hull_hi=None):
        keep = [None if a is None else np.ascontiguousarray(a, dtype=np.float32)
                for a in (params, x_mean, x_std, hull_lo, hull_hi)]
        ptrs = [None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) for a in keep]
        _check(lib.skirt_mlp_set_params(self.h, *ptrs), "skirt_mlp_set_params")

    def get_params(self):
        out = [np.zeros(MLP_NPARAM, np.float32)] + [np.zeros(NBANDS, np.float32) for _ in range(4)]
        _check(lib.skirt_mlp_get_params(self.h, *[a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) for a in out]),
               "skirt_mlp_get_params")
        return out  # params, mean, std, lo, hi

    def set_guard(self, share_max):
        _check(lib.skirt_mlp_set_guard(self.h, float(share_max)), "skirt_mlp_set_guard")

    def get_guard(self):
        v = ctypes.c_float()
        _check(lib.skirt_mlp_get_guard(self.h, ctypes.byref(v)), "skirt_mlp_get_guard")
        return v.value

    def train(self, features, emission, n, epochs=None, batch=None, lr=None, seed=None, stream=None,
              guard_quantile=None):
        """features: device float [n, 32]; emission: device double [n, 100]
        (target rows, normalised on the device)."""
        target = emission
        o = skirt_mlp_train_opts()
        _check(lib.skirt_mlp_train_opts_default(ctypes.byref(o)), "skirt_mlp_train_opts_default")
        if epochs is not None:
            o.epochs = int(epochs)
        if batch is not None:
            o.batch = int(batch)
        if lr is not None:
            o.lr = float(lr)
        if seed is not None:
            o.seed = int(seed)
        if guard_quantile is not None:
            o.guard_quantile = float(guard_quantile)
        hist = np.zeros(o.epochs, np.float32)
        _check(lib.skirt_mlp_train(self.h, _ptr(features), _ptr(target), int(n), ctypes.byref(o),
                                   hist.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _st(stream)), "skirt_mlp_train")
        return hist

    def grad(self, x_std, target, n, stream=None):
        g = np.zeros(MLP_NPARAM, np.float32)
        loss = ctypes.c_float()
        _check(lib.skirt_mlp_grad(self.h, _ptr(x_std), _ptr(target), int(n),
                                  g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(loss), _st(stream)),
               "skirt_mlp_grad")
        return g, loss.value

    def forward(self, features, total, n, emission, flags=None, stream=None):
        _check(lib.skirt_mlp_forward(self.h, _ptr(features), _ptr(total), int(n), _ptr(emission), _ptr(flags),
                                     _st(stream)), "skirt_mlp_forward")


def unpack_params(p):
    """Packed FP32 parameter vector -> dict W1 b1 W2 b2 W3 b3 (float64)."""
    p = np.asarray(p, dtype=np.float64)
    o = 0
    out = {}
    for name, shape in (("W1", (128, 32)), ("b1", (128,)), ("W2", (128, 128)), ("b2", (128,)), ("W3", (100, 128)),
                        ("b3", (100,))):
        k = int(np.prod(shape))
        out[name] = p[o:o + k].reshape(shape)
        o += k
    return out


def pack_params(d):
    return np.concatenate([np.asarray(d[k], dtype=np.float32).ravel() for k in ("W1", "b1", "W2", "b2", "W3", "b3")])
