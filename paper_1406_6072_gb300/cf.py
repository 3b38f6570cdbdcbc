"""Thin Python binding of the C ABI in ``include/cf.h`` (``libcf.so``).

Argument marshalling only: every function has the name of its C entry point,
takes torch CUDA tensors (or raw integer device pointers) for device arrays
and a stream (default: torch's current stream), and raises :class:`CfError`
on a non-OK status.  All computation happens in the CUDA library; if the
library has not been built this module fails on import.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# CF_LIBRARY may name another build of the same library (e.g. a tuning variant)
LIB_PATH = os.environ.get("CF_LIBRARY") or os.path.join(_HERE, "libcf.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libcf.so is not built (run __graft_entry__.build() or "
                      "python -m paper_1406_6072_gb300._build): " + LIB_PATH)

_lib = C.CDLL(LIB_PATH)

# ----------------------------------------------------------------- constants
CF_OK, CF_ERR_ARG, CF_ERR_NOT_PSD, CF_ERR_NOMEM, CF_ERR_UNSUPPORTED, CF_ERR_CUDA = 0, 1, 2, 3, 4, 5
CF_ERR_TIMEOUT, CF_ERR_BUSY, CF_ERR_NOT_FOUND = 6, 7, 8
STATUS_NAMES = {0: "CF_OK", 1: "CF_ERR_ARG", 2: "CF_ERR_NOT_PSD", 3: "CF_ERR_NOMEM",
                4: "CF_ERR_UNSUPPORTED", 5: "CF_ERR_CUDA", 6: "CF_ERR_TIMEOUT", 7: "CF_ERR_BUSY",
                8: "CF_ERR_NOT_FOUND"}
CF_F64, CF_F32, CF_BF16_TC, CF_F16_TC = 0, 1, 2, 3
CF_XI_GAUSSIAN, CF_XI_GEN_CAUCHY, CF_XI_EXPONENTIAL, CF_XI_TABLE = 0, 1, 2, 3
CF_EMBED_CLAMP, CF_EMBED_SKIP_ERROR, CF_EMBED_LOG1P, CF_EMBED_DF = 1, 2, 4, 8
CF_BINS_LINEAR, CF_BINS_LOG, CF_BINS_EDGES = 0, 1, 2


class CfError(RuntimeError):
    def __init__(self, status, func, message):
        self.status = status
        super().__init__("%s returned %s: %s" % (func, STATUS_NAMES.get(status, status), message))


# ----------------------------------------------------------------- structs
class cf_grid(C.Structure):
    _fields_ = [("ndim", C.c_int32), ("embed_factor", C.c_int32), ("n", C.c_int64 * 3), ("cell", C.c_double * 3)]


class cf_xi(C.Structure):
    _fields_ = [("kind", C.c_int32), ("table_on_device", C.c_int32), ("amp", C.c_double),
                ("scale", C.c_double), ("beta", C.c_double), ("table", C.c_void_p)]


class cf_embed_report(C.Structure):
    _fields_ = [("lambda_min", C.c_double), ("lambda_max", C.c_double), ("tau", C.c_double),
                ("neg_mass", C.c_double), ("cov_error", C.c_double), ("n_negative", C.c_int64),
                ("n_zeroed", C.c_int64), ("clamped", C.c_int32), ("exact", C.c_int32)]

    def asdict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class cf_lp_params(C.Structure):
    _fields_ = [("sigma2", C.c_double), ("nbar", C.c_double), ("f", C.c_void_p), ("seed", C.c_uint64),
                ("delta_out", C.c_void_p), ("counts_out", C.c_void_p)]


class cf_bins(C.Structure):
    _fields_ = [("nbins", C.c_int32), ("kind", C.c_int32), ("kmin", C.c_double), ("kmax", C.c_double),
                ("edges", C.c_void_p)]


class cf_serve_cfg(C.Structure):
    _fields_ = [("device", C.c_int32), ("max_inflight", C.c_int32), ("queue_capacity", C.c_int32),
                ("cache_entries", C.c_int32), ("max_batch_realizations", C.c_int32),
                ("small_request_cells", C.c_int32), ("hbm_budget", C.c_size_t)]


class cf_request(C.Structure):
    _fields_ = [("grid", cf_grid), ("xi", cf_xi), ("embed_flags", C.c_uint32), ("want_counts", C.c_int32),
                ("seed", C.c_uint64), ("r0", C.c_uint64), ("R", C.c_int32), ("pad_", C.c_int32),
                ("sigma2", C.c_double), ("nbar", C.c_double), ("lp_seed", C.c_uint64),
                ("host_fields", C.c_void_p), ("host_counts", C.c_void_p)]


class cf_result(C.Structure):
    _fields_ = [("status", C.c_int), ("cache_hit", C.c_int32), ("queue_ms", C.c_double), ("run_ms", C.c_double),
                ("latency_ms", C.c_double), ("dev_fields", C.c_void_p), ("dev_counts", C.c_void_p),
                ("embed", cf_embed_report)]

    def asdict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "embed"}
        d["embed"] = self.embed.asdict()
        return d


class cf_serve_statistics(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("failed", C.c_uint64),
                ("rejected", C.c_uint64), ("queued", C.c_int64), ("inflight", C.c_int64),
                ("cache_hits", C.c_uint64), ("cache_misses", C.c_uint64), ("cache_evictions", C.c_uint64),
                ("batches", C.c_uint64), ("batched_requests", C.c_uint64), ("realizations", C.c_uint64),
                ("bytes_in_use", C.c_size_t), ("bytes_peak", C.c_size_t), ("budget", C.c_size_t),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("mean_ms", C.c_double),
                ("realizations_per_s", C.c_double)]

    def asdict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = C.c_void_p
_S = C.c_void_p  # cudaStream_t
_sigs = {
    "cf_embed": [C.POINTER(cf_grid), C.POINTER(cf_xi), C.c_uint32, _S, C.POINTER(_P), C.POINTER(cf_embed_report)],
    "cf_embed_from_lambda": [C.POINTER(cf_grid), _P, C.c_uint32, _S, C.POINTER(_P), C.POINTER(cf_embed_report)],
    "cf_embedding_free": [_P],
    "cf_embedding_lambda": [_P, _P, _S],
    "cf_embedding_sqrt_lambda": [_P, _P, _S],
    "cf_embedding_info": [_P, C.POINTER(cf_grid), C.POINTER(cf_embed_report)],
    "cf_draw_noise": [C.c_uint64, C.c_uint64, C.c_int32, C.c_int64, C.c_int64, C.c_int32, _P, _S],
    "cf_noise_selfcheck": [C.POINTER(C.c_uint64), C.POINTER(C.c_uint32)],
    "cf_sample_workspace_size": [_P, C.c_int32, C.c_int32, C.POINTER(C.c_size_t)],
    "cf_sample": [_P, C.c_uint64, C.c_uint64, C.c_int32, C.c_int32, _P, _P, C.c_size_t, _S],
    "cf_sample_lp": [_P, C.c_uint64, C.c_uint64, C.c_int32, C.c_int32, _P, C.POINTER(cf_lp_params), _P,
                     C.c_size_t, _S],
    "cf_sample_noalloc": [_P, C.c_uint64, C.c_uint64, C.c_int32, _P, _S],
    "cf_tc_faults": [_S, C.POINTER(C.c_uint32)],
    "cf_embed_periodic": [_P, _P, C.c_int32, C.c_int32, C.c_int32, C.c_uint32, _S, C.POINTER(_P), _P],
    "cf_copy_corner": [_P, C.c_int32, _P, _P, C.c_int64, _P, _S],
    "cf_mean_cov": [_P, C.c_int64, C.c_int32, _P, _P, _S],
    "cf_cic_histogram": [_P, C.c_int64, C.c_int64, _P, C.c_int32, _P, _P, _P, _S],
    "cf_cic_prediction": [C.c_double, C.c_double, _P, C.c_int64, C.c_int32, _P, _S],
    "cf_astar": [_P, _P, C.c_int64, C.c_int64, C.c_double, C.c_double, _P, _S],
    "cf_cumulative_information": [_P, _P, C.c_int32, _P, _P, C.c_size_t, _S],
    "cf_plan_create": [_P, C.c_uint64, C.c_uint64, C.c_int32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _S,
                       C.POINTER(_P)],
    "cf_plan_launch": [_P, _S],
    "cf_plan_seek": [_P, C.c_uint64, _S],
    "cf_plan_destroy": [_P],
    "cf_tune_sample": [_P, C.c_int32, C.c_int32, _P, C.c_size_t, _P, _S, C.POINTER(C.c_int32),
                       C.POINTER(C.c_double)],
    "cf_tune_info": [_P, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                     C.POINTER(C.c_int32)],
    "cf_tune_set": [_P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32],
    "cf_lognormal_poisson": [_P, C.c_int32, C.c_int64, C.c_int64, C.c_double, C.c_double, _P, C.c_uint64,
                             C.c_uint64, _P, _P, _S],
    "cf_power_spectrum_workspace_size": [C.POINTER(cf_grid), C.c_int64, C.POINTER(cf_bins), C.c_int32,
                                         C.POINTER(C.c_size_t)],
    "cf_power_spectrum": [_P, C.c_int32, C.POINTER(cf_grid), C.c_int64, C.POINTER(cf_bins), _P, _P, _P, _P, _P,
                          C.c_size_t, _S],
    "cf_power_spectrum_counts": [_P, _P, C.POINTER(cf_grid), C.c_int64, C.POINTER(cf_bins), _P, _P, _P, _P, _P,
                                 C.c_size_t, _S],
    "cf_sample_spectra_workspace_size": [_P, C.c_int32, C.POINTER(cf_bins), C.POINTER(C.c_size_t)],
    "cf_sample_spectra": [_P, C.c_uint64, C.c_uint64, C.c_int32, _P, _P, C.POINTER(cf_bins), _P, _P, _P, _P, _P,
                          C.c_size_t, _P, C.c_size_t, _P, _S],
    "cf_serve_create": [C.POINTER(cf_serve_cfg), C.POINTER(_P)],
    "cf_serve_submit": [_P, C.POINTER(cf_request), C.POINTER(C.c_uint64)],
    "cf_serve_poll": [_P, C.c_uint64, C.POINTER(cf_result)],
    "cf_serve_wait": [_P, C.c_uint64, C.c_int64, C.POINTER(cf_result)],
    "cf_serve_release": [_P, C.c_uint64],
    "cf_serve_stats": [_P, C.POINTER(cf_serve_statistics)],
    "cf_serve_destroy": [_P],
}
for _name, _args in _sigs.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = C.c_int
_lib.cf_kernel_timing.argtypes = [C.c_int32]
_lib.cf_kernel_timing.restype = C.c_int
_lib.cf_kernel_timing_read.argtypes = [C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)]
_lib.cf_kernel_timing_read.restype = C.c_int
_lib.cf_last_error.restype = C.c_char_p
_lib.cf_last_error.argtypes = []
_lib.cf_version.restype = C.c_char_p
_lib.cf_version.argtypes = []


def _check(status, func):
    if status != CF_OK:
        raise CfError(status, func, _lib.cf_last_error().decode(errors="replace"))


def _ptr(x):
    """Device (or host) address of a tensor / integer / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError("cannot take the address of %r" % type(x))


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def make_grid(n, cell=None, factor=2):
    """Survey grid of n cells per axis; the embedding grid has factor * n
    points per axis (2, 4 or 8)."""
    g = cf_grid()
    n = list(n)
    g.ndim = len(n)
    g.embed_factor = int(factor)
    for a in range(3):
        g.n[a] = int(n[a]) if a < len(n) else 1
        g.cell[a] = float(cell[a]) if cell is not None and a < len(cell) else 1.0
    return g


def make_xi(kind, amp=1.0, scale=1.0, beta=0.0, table=None, table_on_device=None):
    x = cf_xi()
    x.kind = int(kind)
    x.amp, x.scale, x.beta = float(amp), float(scale), float(beta)
    if table is not None:
        x.table = _ptr(table)
        x.table_on_device = int(table_on_device if table_on_device is not None
                                else getattr(table, "is_cuda", False))
    return x


def make_bins(nbins, kind=CF_BINS_LINEAR, kmin=0.0, kmax=0.0, edges=None):
    b = cf_bins()
    b.nbins, b.kind, b.kmin, b.kmax = int(nbins), int(kind), float(kmin), float(kmax)
    b._edges_keep = None
    if edges is not None:
        arr = np.ascontiguousarray(edges, dtype=np.float64)
        b._edges_keep = arr
        b.edges = arr.ctypes.data
    return b


# ----------------------------------------------------------------- entry points
class Embedding:
    """Owns a cf_embedding handle (freed on close/garbage collection)."""

    def __init__(self, handle, report):
        self.handle = handle
        self.report = report

    def close(self):
        if self.handle:
            _lib.cf_embedding_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cf_embed(grid, xi, flags=0, stream=None):
    h = _P()
    rep = cf_embed_report()
    st = _lib.cf_embed(C.byref(grid), C.byref(xi), flags, _stream(stream), C.byref(h), C.byref(rep))
    if st == CF_ERR_NOT_PSD:
        err = CfError(st, "cf_embed", _lib.cf_last_error().decode())
        err.report = rep.asdict()
        raise err
    _check(st, "cf_embed")
    return Embedding(h.value, rep.asdict())


def cf_embed_periodic(grid, xi, box_factor, extent=2, resolution=4, flags=0, stream=None):
    """Periodic-box (k-space) sampler embedding; see include/cf.h."""
    h = _P()
    rep = cf_embed_report()
    _check(_lib.cf_embed_periodic(C.byref(grid), C.byref(xi), box_factor, extent, resolution, flags, _stream(stream),
                                  C.byref(h), C.byref(rep)), "cf_embed_periodic")
    return Embedding(h.value, rep.asdict())


def cf_mean_cov(x, nrows, ncols, mean=None, cov=None, stream=None):
    _check(_lib.cf_mean_cov(_ptr(x), nrows, ncols, _ptr(mean), _ptr(cov), _stream(stream)), "cf_mean_cov")


def cf_copy_corner(inp, dtype, grid_in, grid_out, nfields, out, stream=None):
    _check(_lib.cf_copy_corner(_ptr(inp), dtype, C.byref(grid_in), C.byref(grid_out), nfields, _ptr(out),
                               _stream(stream)), "cf_copy_corner")


def cf_embed_from_lambda(grid, lam, flags=0, stream=None):
    h = _P()
    rep = cf_embed_report()
    st = _lib.cf_embed_from_lambda(C.byref(grid), _ptr(lam), flags, _stream(stream), C.byref(h), C.byref(rep))
    if st == CF_ERR_NOT_PSD:
        err = CfError(st, "cf_embed_from_lambda", _lib.cf_last_error().decode())
        err.report = rep.asdict()
        raise err
    _check(st, "cf_embed_from_lambda")
    return Embedding(h.value, rep.asdict())


def cf_embedding_free(emb):
    emb.close()


def cf_embedding_lambda(emb, dst, stream=None):
    _check(_lib.cf_embedding_lambda(emb.handle, _ptr(dst), _stream(stream)), "cf_embedding_lambda")


def cf_embedding_sqrt_lambda(emb, dst, stream=None):
    _check(_lib.cf_embedding_sqrt_lambda(emb.handle, _ptr(dst), _stream(stream)), "cf_embedding_sqrt_lambda")


def cf_embedding_info(emb):
    g = cf_grid()
    rep = cf_embed_report()
    _check(_lib.cf_embedding_info(emb.handle, C.byref(g), C.byref(rep)), "cf_embedding_info")
    return g, rep.asdict()


def cf_draw_noise(seed, r0, R, ncells, m_last, dtype, out, stream=None):
    _check(_lib.cf_draw_noise(seed, r0, R, ncells, m_last, dtype, _ptr(out), _stream(stream)), "cf_draw_noise")


def cf_noise_selfcheck():
    """Mismatches of the noise's quotient and square-root sequences against
    the IEEE operations over their whole input domains, and the first
    mismatching inputs' bit patterns: ((nq, ns), (mq, xs))."""
    mism = (C.c_uint64 * 2)()
    ex = (C.c_uint32 * 2)()
    _check(_lib.cf_noise_selfcheck(mism, ex), "cf_noise_selfcheck")
    return (int(mism[0]), int(mism[1])), (int(ex[0]), int(ex[1]))


def cf_sample_workspace_size(emb, R, dtype):
    n = C.c_size_t()
    _check(_lib.cf_sample_workspace_size(emb.handle, R, dtype, C.byref(n)), "cf_sample_workspace_size")
    return n.value


def cf_sample(emb, seed, r0, R, dtype, fields_out, ws, ws_bytes, stream=None):
    _check(_lib.cf_sample(emb.handle, seed, r0, R, dtype, _ptr(fields_out), _ptr(ws), ws_bytes, _stream(stream)),
           "cf_sample")


def cf_sample_noalloc(emb, seed, r0, R, fields_out, stream=None):
    """Binary32 sampler with its intermediate in the library's static array
    (no device allocation).  Calls share that array; the first call on a
    device synchronises it for a one-time set-up, so make it before any
    capture.  When another thread captures a CUDA graph in global mode, pass a
    stream created non-blocking (torch.cuda.Stream() is): the legacy default
    stream synchronises with the capturing stream and breaks the capture."""
    _check(_lib.cf_sample_noalloc(emb.handle, seed, r0, R, _ptr(fields_out), _stream(stream)), "cf_sample_noalloc")


def cf_tune_sample(emb, dtype, R, ws, ws_bytes, fields_scratch, stream=None):
    """Times the candidate chunk schedules; returns (chunk, ms per realization)."""
    c = C.c_int32()
    ms = C.c_double()
    _check(_lib.cf_tune_sample(emb.handle, dtype, R, _ptr(ws), ws_bytes, _ptr(fields_scratch), _stream(stream),
                               C.byref(c), C.byref(ms)), "cf_tune_sample")
    return c.value, ms.value


def cf_tune_info(emb, dtype):
    """The recorded sampler schedule: (chunk, rows_shape, cols_shape, persistent)."""
    c, r, k, p = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
    _check(_lib.cf_tune_info(emb.handle, dtype, C.byref(c), C.byref(r), C.byref(k), C.byref(p)), "cf_tune_info")
    return c.value, r.value, k.value, p.value


def cf_tune_set(emb, dtype, chunk=0, rows_shape=0, cols_shape=0, persistent=0):
    _check(_lib.cf_tune_set(emb.handle, dtype, chunk, rows_shape, cols_shape, persistent), "cf_tune_set")


def cf_cic_histogram(counts, cells, nfields, f, nbins, hist_out, mean=None, cov=None, stream=None):
    _check(_lib.cf_cic_histogram(_ptr(counts), cells, nfields, _ptr(f), nbins, _ptr(hist_out), _ptr(mean), _ptr(cov),
                                 _stream(stream)), "cf_cic_histogram")


def cf_cic_prediction(sigma2_A, nbar, f, cells, nbins, pred_out, stream=None):
    _check(_lib.cf_cic_prediction(sigma2_A, nbar, _ptr(f), cells, nbins, _ptr(pred_out), _stream(stream)),
           "cf_cic_prediction")


def cf_astar(counts, f, cells, nfields, nbar, sigma2_A, out, stream=None):
    _check(_lib.cf_astar(_ptr(counts), _ptr(f), cells, nfields, nbar, sigma2_A, _ptr(out), _stream(stream)),
           "cf_astar")


class Plan:
    """A captured graph of the binary32 per-realization path (cf_plan_*)."""

    def __init__(self, emb, seed, r0, R, fields, lp=None, bins=None, pk=None, nmodes=None, mean=None, cov=None,
                 pk_counts=None, mean_counts=None, cov_counts=None, stream=None):
        h = _P()
        lpp = C.byref(lp) if lp is not None else None
        bp = C.byref(bins) if bins is not None else None
        _check(_lib.cf_plan_create(emb.handle, seed, r0, R, lpp, bp, _ptr(fields), _ptr(pk), _ptr(nmodes), _ptr(mean),
                                   _ptr(cov), _ptr(pk_counts), _ptr(mean_counts), _ptr(cov_counts), _stream(stream),
                                   C.byref(h)), "cf_plan_create")
        self.handle = h
        self._keep = (emb, lp, bins)

    def launch(self, stream=None):
        _check(_lib.cf_plan_launch(self.handle, _stream(stream)), "cf_plan_launch")

    def seek(self, r0, stream=None):
        _check(_lib.cf_plan_seek(self.handle, r0, _stream(stream)), "cf_plan_seek")

    def close(self):
        if self.handle:
            _lib.cf_plan_destroy(self.handle)
            self.handle = None


def cumulative_information_workspace_size(nbins):
    return 8 * (nbins * nbins + nbins) + 4 * nbins


def cf_cumulative_information(mean, cov, nbins, info_out, ws, ws_bytes, stream=None):
    _check(_lib.cf_cumulative_information(_ptr(mean), _ptr(cov), nbins, _ptr(info_out), _ptr(ws), ws_bytes,
                                          _stream(stream)), "cf_cumulative_information")


def cf_tc_faults(stream=None):
    """Tensor-core waits that ran out of time since the last call (0 = all good)."""
    c = C.c_uint32()
    _check(_lib.cf_tc_faults(_stream(stream), C.byref(c)), "cf_tc_faults")
    return c.value


def make_lp(sigma2, nbar, counts_out, seed, f=None, delta_out=None):
    p = cf_lp_params()
    p.sigma2, p.nbar, p.seed = float(sigma2), float(nbar), int(seed)
    p.f, p.delta_out, p.counts_out = _ptr(f), _ptr(delta_out), _ptr(counts_out)
    return p


def cf_sample_lp(emb, seed, r0, R, dtype, fields_out, lp, ws, ws_bytes, stream=None):
    _check(_lib.cf_sample_lp(emb.handle, seed, r0, R, dtype, _ptr(fields_out), C.byref(lp), _ptr(ws), ws_bytes,
                             _stream(stream)), "cf_sample_lp")


def cf_lognormal_poisson(G, dtype, cells_per_field, nfields, sigma2, nbar, f, seed, field0, delta_out, counts_out,
                         stream=None):
    _check(_lib.cf_lognormal_poisson(_ptr(G), dtype, cells_per_field, nfields, sigma2, nbar, _ptr(f), seed, field0,
                                     _ptr(delta_out), _ptr(counts_out), _stream(stream)), "cf_lognormal_poisson")


def cf_power_spectrum_workspace_size(grid, nfields, bins, dtype):
    n = C.c_size_t()
    _check(_lib.cf_power_spectrum_workspace_size(C.byref(grid), nfields, C.byref(bins), dtype, C.byref(n)),
           "cf_power_spectrum_workspace_size")
    return n.value


def cf_sample_spectra_workspace_size(emb, R, bins):
    n = C.c_size_t()
    _check(_lib.cf_sample_spectra_workspace_size(emb.handle, R, C.byref(bins), C.byref(n)),
           "cf_sample_spectra_workspace_size")
    return n.value


def cf_sample_spectra(emb, seed, r0, R, fields_out, lp, bins, pk_out, nmodes_out, mean=None, cov=None, ws=None,
                      ws_bytes=0, pk_ws=None, pk_ws_bytes=0, sampled_event=None, stream=None):
    """cf_sample / cf_sample_lp (lp may be None) fused with cf_power_spectrum
    of the fields; sampled_event (torch.cuda.Event) is recorded once the
    fields and counts are complete."""
    ev = None
    if sampled_event is not None:
        h = sampled_event.cuda_event if hasattr(sampled_event, "cuda_event") else int(sampled_event)
        if not h:
            raise ValueError("sampled_event has no CUDA event yet (record it once first)")
        ev = C.c_void_p(h)
    _check(_lib.cf_sample_spectra(emb.handle, seed, r0, R, _ptr(fields_out), C.byref(lp) if lp is not None else None,
                                  C.byref(bins), _ptr(pk_out), _ptr(nmodes_out), _ptr(mean), _ptr(cov), _ptr(ws),
                                  ws_bytes, _ptr(pk_ws), pk_ws_bytes, ev, _stream(stream)), "cf_sample_spectra")


def cf_power_spectrum(fields, dtype, grid, nfields, bins, pk_out, nmodes_out, mean=None, cov=None, ws=None,
                      ws_bytes=0, stream=None):
    _check(_lib.cf_power_spectrum(_ptr(fields), dtype, C.byref(grid), nfields, C.byref(bins), _ptr(pk_out),
                                  _ptr(nmodes_out), _ptr(mean), _ptr(cov), _ptr(ws), ws_bytes, _stream(stream)),
           "cf_power_spectrum")


def cf_power_spectrum_counts(counts, f, grid, nfields, bins, pk_out, nmodes_out, mean=None, cov=None, ws=None,
                             ws_bytes=0, stream=None):
    _check(_lib.cf_power_spectrum_counts(_ptr(counts), _ptr(f), C.byref(grid), nfields, C.byref(bins),
                                         _ptr(pk_out), _ptr(nmodes_out), _ptr(mean), _ptr(cov), _ptr(ws), ws_bytes,
                                         _stream(stream)), "cf_power_spectrum_counts")


# ----------------------------------------------------------------- serving
def make_serve_cfg(device=0, max_inflight=4, queue_capacity=100000, cache_entries=64, max_batch_realizations=256,
                   hbm_budget=32 << 30, small_request_cells=0):
    c = cf_serve_cfg()
    c.small_request_cells = int(small_request_cells)
    c.device, c.max_inflight, c.queue_capacity = device, max_inflight, queue_capacity
    c.cache_entries, c.max_batch_realizations, c.hbm_budget = cache_entries, max_batch_realizations, hbm_budget
    return c


def make_request(n, kind, amp, scale, beta=0.0, seed=0, r0=0, R=1, embed_flags=CF_EMBED_CLAMP, want_counts=False,
                 sigma2=0.0, nbar=0.0, lp_seed=0, host_fields=None, host_counts=None, cell=None, factor=2):
    r = cf_request()
    r.grid = make_grid(n, cell, factor)
    r.xi = make_xi(kind, amp, scale, beta)
    r.embed_flags, r.want_counts = embed_flags, int(bool(want_counts))
    r.seed, r.r0, r.R = seed, r0, R
    r.sigma2, r.nbar, r.lp_seed = sigma2, nbar, lp_seed
    r.host_fields, r.host_counts = _ptr(host_fields), _ptr(host_counts)
    return r


class Server:
    """Owns a cf_server handle."""

    def __init__(self, handle):
        self.handle = handle

    def close(self):
        if self.handle:
            _lib.cf_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cf_serve_create(cfg):
    h = _P()
    _check(_lib.cf_serve_create(C.byref(cfg), C.byref(h)), "cf_serve_create")
    return Server(h.value)


def cf_serve_submit(sv, req):
    t = C.c_uint64()
    _check(_lib.cf_serve_submit(sv.handle, C.byref(req), C.byref(t)), "cf_serve_submit")
    return t.value


def cf_serve_poll(sv, ticket):
    """Result dict when finished, None while queued or running."""
    r = cf_result()
    st = _lib.cf_serve_poll(sv.handle, ticket, C.byref(r))
    if st == CF_ERR_BUSY:
        return None
    _check(st, "cf_serve_poll")
    return r.asdict()


def cf_serve_wait(sv, ticket, timeout_us=-1):
    r = cf_result()
    _check(_lib.cf_serve_wait(sv.handle, ticket, timeout_us, C.byref(r)), "cf_serve_wait")
    return r.asdict()


def cf_serve_release(sv, ticket):
    _check(_lib.cf_serve_release(sv.handle, ticket), "cf_serve_release")


def cf_serve_stats(sv):
    s = cf_serve_statistics()
    _check(_lib.cf_serve_stats(sv.handle, C.byref(s)), "cf_serve_stats")
    return s.asdict()


def cf_serve_destroy(sv):
    sv.close()


def cf_kernel_timing(enable):
    _check(_lib.cf_kernel_timing(int(bool(enable))), "cf_kernel_timing")


def cf_kernel_timing_read():
    """{kernel: (launches, total_ms)} accumulated since cf_kernel_timing(1)."""
    import json
    need = C.c_size_t()
    _lib.cf_kernel_timing_read(None, 0, C.byref(need))
    buf = C.create_string_buffer(need.value + 64)
    _check(_lib.cf_kernel_timing_read(buf, len(buf), C.byref(need)), "cf_kernel_timing_read")
    return {k: (int(v[0]), float(v[1])) for k, v in json.loads(buf.value.decode()).items()}


def cf_last_error():
    return _lib.cf_last_error().decode(errors="replace")


def cf_version():
    return _lib.cf_version().decode()


def raw_lib():
    """The loaded ctypes library (for ABI tests)."""
    return _lib
