"""One pass of the whole hot path over a workload, through the C ABI.

A step is: embed (a1-a3) -> sample with the fused lognormal/Poisson epilogue
(b1-b4, c1-c2) -> power spectra of the Gaussian fields and of the count maps
with mean and covariance (d1).  Device buffers are allocated once with torch;
every computation is a call into libcf.so on one stream.
"""
from __future__ import annotations

import torch

from . import cf
from .workloads import Workload


class FieldPipeline:
    """Buffers and calls of one step.  With `embed_stream`, embeddings run on
    that stream: the embedding of the next step (a binary64 job) then overlaps
    the sampler and spectra of the current one, which stay on `stream`; an
    embedding is released in stream order after its last use, so replacing it
    while its sampler is still queued is safe."""

    def __init__(self, wl: Workload, device="cuda:0", stream=None, R=None, with_pk=True, embed_stream=None,
                 fused=False, embed_df=False):
        self.wl = wl
        self.dev = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.dev)
        self.embed_stream = embed_stream if embed_stream is not None else self.stream
        self.R = wl.R if R is None else R
        self.dtype = cf.CF_F32 if wl.dtype == "f32" else cf.CF_F64
        self.tdtype = torch.float32 if wl.dtype == "f32" else torch.float64
        self.grid = cf.make_grid(wl.n, wl.cell[: wl.ndim], wl.factor)
        self.xi = cf.make_xi(wl.xi_kind, wl.amp, wl.scale, wl.beta)
        self.flags = (cf.CF_EMBED_CLAMP if wl.clamp else 0) | (cf.CF_EMBED_DF if embed_df else 0)
        self.with_lp = wl.nbar is not None and self.dtype == cf.CF_F32
        self.with_pk = with_pk and wl.nbins is not None
        F = 2 * self.R
        shape = (self.R, 2) + tuple(wl.n)
        self.fields = torch.empty(shape, dtype=self.tdtype, device=self.dev)
        self.counts = torch.empty(shape, dtype=torch.int32, device=self.dev) if self.with_lp else None
        self.emb = None
        self.ws = None
        self.ws_bytes = 0
        if self.with_pk:
            self.bins = cf.make_bins(wl.nbins)
            self.pk_ws_bytes = cf.cf_power_spectrum_workspace_size(self.grid, F, self.bins, self.dtype)
            self.pk_ws = torch.empty(self.pk_ws_bytes, dtype=torch.uint8, device=self.dev)
            self.pk = torch.empty((F, wl.nbins), dtype=torch.float64, device=self.dev)
            self.nmodes = torch.empty(wl.nbins, dtype=torch.int64, device=self.dev)
            self.mean = torch.empty(wl.nbins, dtype=torch.float64, device=self.dev)
            self.cov = torch.empty((wl.nbins, wl.nbins), dtype=torch.float64, device=self.dev)
            if self.with_lp:
                self.pkg = torch.empty_like(self.pk)
                self.meang = torch.empty_like(self.mean)
                self.covg = torch.empty_like(self.cov)
                # the count maps' spectra run beside the fields' on a second
                # stream, with their own workspace and mode counts
                self.pk_ws_g = torch.empty(self.pk_ws_bytes, dtype=torch.uint8, device=self.dev)
                self.nmodes_g = torch.empty_like(self.nmodes)
                self.stream_g = torch.cuda.Stream(self.dev)
                self.ev_sampled = torch.cuda.Event()
                self.ev_counts_done = torch.cuda.Event()
                self.ev_sampled.record(self.stream)  # creates the CUDA event (the fused call records it)
        # fused=True on square 2D grids: the sampler's last pass also runs the
        # first axis of the fields' spectra (cf_sample_spectra; measured no
        # faster on the 512^2 workload, where the two spectra run concurrently)
        self.fused = (fused and self.with_pk and self.dtype == cf.CF_F32 and wl.ndim == 2 and wl.n[0] == wl.n[1]
                      and wl.factor == 2 and 128 <= wl.n[0] <= 2048)
        if self.fused:
            self.fused_ws_bytes = None
            self.fused_ws = None

    def embed(self, xi=None):
        if self.emb is not None:
            self.emb.close()
        self.emb = cf.cf_embed(self.grid, xi or self.xi, self.flags, self.embed_stream)
        need = cf.cf_sample_workspace_size(self.emb, self.R, self.dtype)
        if self.ws is None or need > self.ws_bytes:
            self.ws_bytes = need
            self.ws = torch.empty(max(need, 1), dtype=torch.uint8, device=self.dev)
        return self.emb.report

    def tune(self):
        """Times the sampler's chunk schedules on this workload's grid (the
        pipeline's field buffer serves as scratch) and keeps the fastest for
        later calls; returns (chunk, ms per realization)."""
        per = cf.cf_sample_workspace_size(self.emb, 1, self.dtype)
        cap = per * self.R
        ws = torch.empty(max(cap, 1), dtype=torch.uint8, device=self.dev)
        chunk, ms = cf.cf_tune_sample(self.emb, self.dtype, self.R, ws, cap, self.fields, self.stream)
        del ws
        self.ws_bytes = cf.cf_sample_workspace_size(self.emb, self.R, self.dtype)
        self.ws = torch.empty(max(self.ws_bytes, 1), dtype=torch.uint8, device=self.dev)
        return chunk, ms

    def sample(self, r0=0):
        wl = self.wl
        if self.fused:
            need = cf.cf_sample_spectra_workspace_size(self.emb, self.R, self.bins)
            if self.fused_ws is None or need > self.fused_ws_bytes:
                self.fused_ws_bytes = need
                self.fused_ws = torch.empty(need, dtype=torch.uint8, device=self.dev)
            lp = cf.make_lp(wl.sigma2, wl.nbar, self.counts, wl.seed + 1000) if self.with_lp else None
            cf.cf_sample_spectra(self.emb, wl.seed, r0, self.R, self.fields, lp, self.bins, self.pk, self.nmodes,
                                 self.mean, self.cov, self.ws, self.ws_bytes, self.fused_ws, self.fused_ws_bytes,
                                 self.ev_sampled if self.with_lp else None, self.stream)
            return
        if self.with_lp:
            lp = cf.make_lp(wl.sigma2, wl.nbar, self.counts, wl.seed + 1000)
            cf.cf_sample_lp(self.emb, wl.seed, r0, self.R, self.dtype, self.fields, lp, self.ws, self.ws_bytes,
                            self.stream)
        else:
            cf.cf_sample(self.emb, wl.seed, r0, self.R, self.dtype, self.fields, self.ws, self.ws_bytes, self.stream)

    def spectra(self):
        if not self.with_pk:
            return
        F = 2 * self.R
        if self.with_lp:
            if not self.fused:
                self.ev_sampled.record(self.stream)
            self.stream_g.wait_event(self.ev_sampled)
            cf.cf_power_spectrum_counts(self.counts, None, self.grid, F, self.bins, self.pkg, self.nmodes_g,
                                        self.meang, self.covg, self.pk_ws_g, self.pk_ws_bytes, self.stream_g)
            self.ev_counts_done.record(self.stream_g)
        if not self.fused:  # the fused call computed the fields' spectra
            cf.cf_power_spectrum(self.fields, self.dtype, self.grid, F, self.bins, self.pk, self.nmodes, self.mean,
                                 self.cov, self.pk_ws, self.pk_ws_bytes, self.stream)
        if self.with_lp:
            # the step ends on the main stream once both spectra are done (the
            # next sampling overwrites the count maps)
            self.stream.wait_event(self.ev_counts_done)

    def step(self, r0=0):
        """Embed + sample (+ lognormal/Poisson) + spectra for realizations [r0, r0+R)."""
        self.embed()
        self.sample(r0)
        self.spectra()

    @property
    def cells_per_step(self):
        return 2 * self.R * self.wl.cells_per_field

    def close(self):
        if self.emb is not None:
            self.emb.close()
            self.emb = None
