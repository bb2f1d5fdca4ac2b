"""Pairwise line-of-sight power-spectrum and correlation-function multipoles on GB300.

Thin ctypes binding of the C ABI in ``include/bym.h`` (library ``libbym.so``,
built in-tree by ``paper_2102_08384_gb300.build``).  This module only
marshals arguments: every step of the estimators runs in the library's CUDA
kernels.  Catalogs are (n, 4) float32 arrays of x, y, z, w -- numpy arrays
(host memory) or CUDA torch tensors (device memory) -- with optional float32
nbar arrays.

Estimators (Philcox & Slepian, arXiv:2102.08384):
  los="yamamoto"  Sec. 2, eq. Yamamoto-estimator / eq. 2pcf-yama
  los="midpoint"  Secs. 3-4, eq. FFT-midpoint / eq. xi-parity-all-estimator
  los="bisector"  Secs. 5-6, eq. bisector-pk-fft / the Sec. 6 estimator
  los="midpoint_even"  the parity-even midpoint forms, Secs. 3.3 and 4.3 (order <= 4)
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbym.so")

LOS = {"yamamoto": 0, "midpoint": 1, "bisector": 2, "midpoint_even": 3}

BYM_OK = 0
ERRORS = {-1: "INVAL", -2: "OUT_OF_BOX", -3: "NOMEM", -4: "CUDA", -5: "TIMEOUT", -6: "UNSUPPORTED",
          -7: "BUSY"}


class BymError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"bym error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class Catalog(ctypes.Structure):
    _fields_ = [("xyzw", ctypes.c_void_p), ("nbar", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("on_device", ctypes.c_int)]


class Params(ctypes.Structure):
    _fields_ = [("box_lo", ctypes.c_double * 3), ("box_len", ctypes.c_double), ("n_mesh", ctypes.c_int),
                ("assign", ctypes.c_int), ("ell_max", ctypes.c_int), ("los", ctypes.c_int),
                ("order", ctypes.c_int), ("compensate", ctypes.c_int), ("precision", ctypes.c_int),
                ("norm", ctypes.c_int),
                ("interlace", ctypes.c_int)]


class Bins(ctypes.Structure):
    _fields_ = [("edges", ctypes.c_void_p), ("nbins", ctypes.c_int)]


class Request(ctypes.Structure):
    _fields_ = [("gal", Catalog), ("ran", Catalog), ("params", Params), ("kbins", Bins), ("rbins", Bins)]


class Result(ctypes.Structure):
    _fields_ = [("pk", ctypes.c_void_p), ("k_mean", ctypes.c_void_p), ("n_modes", ctypes.c_void_p),
                ("xi", ctypes.c_void_p), ("r_mean", ctypes.c_void_p), ("n_cells", ctypes.c_void_p)]


_lib_handle = None


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib_handle
    if _lib_handle is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64p, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)
        L.bym_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_size_t]
        L.bym_destroy.argtypes = [vp]
        L.bym_destroy.restype = None
        L.bym_last_error.argtypes = [vp]
        L.bym_last_error.restype = ctypes.c_char_p
        L.bym_version.restype = ctypes.c_char_p
        L.bym_footprint.argtypes = [ctypes.POINTER(Params), ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                    ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]
        cat_p, par_p, bins_p = ctypes.POINTER(Catalog), ctypes.POINTER(Params), ctypes.POINTER(Bins)
        L.bym_pk_multipoles.argtypes = [vp, cat_p, cat_p, par_p, bins_p, dp, dp, i64p, vp]
        L.bym_xi_multipoles.argtypes = [vp, cat_p, cat_p, par_p, bins_p, dp, dp, i64p, vp]
        L.bym_pk_xi_multipoles.argtypes = [vp, cat_p, cat_p, par_p, bins_p, bins_p, dp, dp, i64p, dp, dp, i64p,
                                           vp]
        L.bym_pk_xi_cross.argtypes = [vp, cat_p, cat_p, cat_p, cat_p, par_p, bins_p, bins_p, dp, dp, i64p, dp, dp,
                                      i64p, vp]
        L.bym_pk_xi_cross_odd.argtypes = L.bym_pk_xi_cross.argtypes
        L.bym_jit_check.argtypes = [par_p, ctypes.c_char_p, ctypes.c_size_t]
        L.bym_shot_noise.argtypes = [vp, cat_p, cat_p, par_p, dp]
        L.bym_serve_start.argtypes = [vp, ctypes.c_int, ctypes.c_size_t]
        L.bym_serve_stop.argtypes = [vp]
        L.bym_submit.argtypes = [vp, ctypes.POINTER(Request), ctypes.POINTER(Result), ctypes.POINTER(ctypes.c_uint64)]
        L.bym_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)]
        L.bym_wait.argtypes = [vp, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(ctypes.c_int)]
        L.bym_serve_stats.argtypes = [vp, dp]
        L.bym_serve_reset_stats.argtypes = [vp]
        L.bym_batch_run.argtypes = [vp, ctypes.c_int, ctypes.POINTER(Request), ctypes.POINTER(Result),
                                    ctypes.POINTER(ctypes.c_int)]
        L.bym_batch_graph.argtypes = L.bym_batch_run.argtypes
        L.bym_batch_plan_create.argtypes = [vp, ctypes.c_int, ctypes.POINTER(Request), ctypes.POINTER(Result),
                                            ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int)]
        L.bym_batch_plan_launch.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
        L.bym_batch_plan_destroy.argtypes = [vp]
        L.bym_batch_plan_destroy.restype = None
        L.bym_profile_enable.argtypes = [vp, ctypes.c_int]
        L.bym_autotune.argtypes = [vp, cat_p, cat_p, par_p, bins_p, bins_p, ctypes.c_char_p, ctypes.c_char_p,
                                   ctypes.c_size_t]
        L.bym_set_fft_backend.argtypes = [vp, ctypes.c_int]
        L.bym_set_field_chunk.argtypes = [vp, ctypes.c_int]
        L.bym_fft3d.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp]
        L.bym_profile_read.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t, ctypes.c_int]
        _lib_handle = L
    return _lib_handle


def make_params(*, box_lo, box_len, n_mesh, assign=2, ell_max=4, los="yamamoto", order=0,
                compensate=False, precision=32, norm=1, interlace=False) -> Params:
    p = Params()
    p.box_lo[:] = [float(v) for v in box_lo]
    p.box_len = float(box_len)
    p.n_mesh = int(n_mesh)
    p.assign = int(assign)
    p.ell_max = int(ell_max)
    p.los = LOS[los] if isinstance(los, str) else int(los)
    p.order = int(order)
    p.compensate = int(bool(compensate))
    p.precision = int(precision)
    p.norm = int(norm)
    p.interlace = int(bool(interlace))
    return p


def _catalog(xyzw, nbar, keep):
    """Catalog struct for a numpy (host) or CUDA torch (device) array."""
    c = Catalog()
    if xyzw is None:
        return None
    if hasattr(xyzw, "is_cuda") and xyzw.is_cuda:
        import torch
        assert xyzw.dtype == torch.float32 and xyzw.dim() == 2 and xyzw.shape[1] == 4
        xyzw = xyzw.contiguous()
        keep.append(xyzw)
        c.xyzw, c.n, c.on_device = xyzw.data_ptr(), xyzw.shape[0], 1
        if nbar is not None:
            nbar = nbar.contiguous().to(torch.float32)
            keep.append(nbar)
            c.nbar = nbar.data_ptr()
        return c
    a = np.ascontiguousarray(xyzw, dtype=np.float32)
    if a.ndim != 2 or a.shape[1] != 4:
        raise ValueError("catalog must be (n, 4) float32")
    keep.append(a)
    c.xyzw, c.n, c.on_device = a.ctypes.data, a.shape[0], 0
    if nbar is not None:
        nb = np.ascontiguousarray(nbar, dtype=np.float32)
        keep.append(nb)
        c.nbar = nb.ctypes.data
    return c


def _bins(edges, keep):
    e = np.ascontiguousarray(edges, dtype=np.float64)
    keep.append(e)
    b = Bins()
    b.edges, b.nbins = e.ctypes.data, len(e) - 1
    return b


def _ptr(obj):
    return ctypes.byref(obj) if obj is not None else None


class Context:
    """One library context on a CUDA device (plans, tables and kernels cached)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self._L = lib()
        h = ctypes.c_void_p()
        rc = self._L.bym_create(ctypes.byref(h), int(device), int(hbm_budget_bytes))
        if rc != BYM_OK:
            raise BymError(rc, "bym_create failed")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._L.bym_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return self._L.bym_last_error(self._h).decode()

    def _check(self, rc):
        if rc != BYM_OK:
            raise BymError(rc, self._L.bym_last_error(self._h).decode())

    def _run(self, which, gal, ran, params, kedges, redges, gal_nbar, ran_nbar, stream):
        keep = []
        g = _catalog(gal, gal_nbar, keep)
        r = _catalog(ran, ran_nbar, keep)
        nl = params.ell_max // 2 + 1
        out = {}
        st = ctypes.c_void_p(stream) if stream else None
        dp = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        if kedges is not None:
            kb = _bins(kedges, keep)
            nbk = kb.nbins
            out["pk"] = np.zeros((nl, nbk))
            out["k_mean"] = np.zeros(nbk)
            out["n_modes"] = np.zeros(nbk, dtype=np.int64)
        if redges is not None:
            rb = _bins(redges, keep)
            nbr = rb.nbins
            out["xi"] = np.zeros((nl, nbr))
            out["r_mean"] = np.zeros(nbr)
            out["n_cells"] = np.zeros(nbr, dtype=np.int64)
        if which == "pk":
            rc = self._L.bym_pk_multipoles(self._h, _ptr(g), _ptr(r), ctypes.byref(params), ctypes.byref(kb),
                                           out["pk"].ctypes.data_as(dp), out["k_mean"].ctypes.data_as(dp),
                                           out["n_modes"].ctypes.data_as(i64p), st)
        elif which == "xi":
            rc = self._L.bym_xi_multipoles(self._h, _ptr(g), _ptr(r), ctypes.byref(params), ctypes.byref(rb),
                                           out["xi"].ctypes.data_as(dp), out["r_mean"].ctypes.data_as(dp),
                                           out["n_cells"].ctypes.data_as(i64p), st)
        else:
            rc = self._L.bym_pk_xi_multipoles(self._h, _ptr(g), _ptr(r), ctypes.byref(params), ctypes.byref(kb),
                                              ctypes.byref(rb), out["pk"].ctypes.data_as(dp),
                                              out["k_mean"].ctypes.data_as(dp),
                                              out["n_modes"].ctypes.data_as(i64p), out["xi"].ctypes.data_as(dp),
                                              out["r_mean"].ctypes.data_as(dp),
                                              out["n_cells"].ctypes.data_as(i64p), st)
        self._check(rc)
        out["ells"] = list(range(0, params.ell_max + 1, 2))
        return out

    def autotune(self, gal, ran, params, kedges=None, redges=None, gal_nbar=None, ran_nbar=None,
                 cache_path=None):
        """Pick launch shapes for requests like this one (see bym_autotune); returns the choice."""
        import json
        keep = []
        g = _catalog(gal, gal_nbar, keep)
        r = _catalog(ran, ran_nbar, keep)
        kb = _bins(kedges, keep) if kedges is not None else None
        rb = _bins(redges, keep) if redges is not None else None
        rep = ctypes.create_string_buffer(1024)
        self._check(self._L.bym_autotune(self._h, _ptr(g), _ptr(r), ctypes.byref(params), _ptr(kb), _ptr(rb),
                                         cache_path.encode() if cache_path else None, rep, len(rep)))
        return json.loads(rep.value.decode())

    def set_field_chunk(self, max_fields: int):
        """Midpoint g fields generated and consumed in ranges of at most max_fields (0: only when needed)."""
        self._check(self._L.bym_set_field_chunk(self._h, int(max_fields)))

    def set_fft_backend(self, mode: int):
        """0: cuFFT, 1: the library's cluster plane pass + x pass where they apply (8-CTA clusters), 2: as
        tuned (default), 3: the same with 16-CTA clusters, 4: cuFFT plane transforms + the library's x pass,
        5: cuFFT plane transforms + cuFFT along x, 6: the library's z, y and x passes (bym_set_fft_backend)."""
        self._check(self._L.bym_set_fft_backend(self._h, int(mode)))

    # ------------------------------------------------------------ serving
    def _request(self, gal, ran, params, kedges, redges, gal_nbar, ran_nbar):
        """Request + Result structs and the output arrays (kept alive by the caller)."""
        keep = []
        req = Request()
        g = _catalog(gal, gal_nbar, keep)
        req.gal = g
        r = _catalog(ran, ran_nbar, keep) if ran is not None else None
        if r is not None:
            req.ran = r
        req.params = params
        nl = params.ell_max // 2 + 1
        out = {"ells": list(range(0, params.ell_max + 1, 2))}
        res = Result()
        if kedges is not None:
            req.kbins = _bins(kedges, keep)
            nb = req.kbins.nbins
            out.update(pk=np.zeros((nl, nb)), k_mean=np.zeros(nb), n_modes=np.zeros(nb, dtype=np.int64))
            res.pk, res.k_mean, res.n_modes = (out["pk"].ctypes.data, out["k_mean"].ctypes.data,
                                               out["n_modes"].ctypes.data)
        if redges is not None:
            req.rbins = _bins(redges, keep)
            nb = req.rbins.nbins
            out.update(xi=np.zeros((nl, nb)), r_mean=np.zeros(nb), n_cells=np.zeros(nb, dtype=np.int64))
            res.xi, res.r_mean, res.n_cells = (out["xi"].ctypes.data, out["r_mean"].ctypes.data,
                                               out["n_cells"].ctypes.data)
        return req, res, out, keep

    def serve_start(self, n_slots=4, hbm_budget_bytes=0):
        self._check(self._L.bym_serve_start(self._h, int(n_slots), int(hbm_budget_bytes)))
        self._pending = {}

    def serve_stop(self):
        self._check(self._L.bym_serve_stop(self._h))

    def submit(self, gal, ran, params, kedges=None, redges=None, gal_nbar=None, ran_nbar=None):
        """Queue a request; returns a ticket.  Outputs are returned by wait()."""
        req, res, out, keep = self._request(gal, ran, params, kedges, redges, gal_nbar, ran_nbar)
        t = ctypes.c_uint64()
        self._check(self._L.bym_submit(self._h, ctypes.byref(req), ctypes.byref(res), ctypes.byref(t)))
        self._pending[t.value] = (req, res, out, keep)
        return t.value

    def poll(self, ticket):
        d = ctypes.c_int()
        self._check(self._L.bym_poll(self._h, ctypes.c_uint64(ticket), ctypes.byref(d)))
        return bool(d.value)

    def wait(self, ticket, timeout_s=-1.0):
        """Outputs of a finished request; raises BymError (code -5) on timeout."""
        st = ctypes.c_int()
        self._check(self._L.bym_wait(self._h, ctypes.c_uint64(ticket), float(timeout_s), ctypes.byref(st)))
        req, res, out, keep = self._pending.pop(ticket)
        if st.value != BYM_OK:
            raise BymError(st.value, f"request {ticket} failed")
        return out

    def serve_reset_stats(self):
        self._check(self._L.bym_serve_reset_stats(self._h))

    def serve_stats(self):
        a = (ctypes.c_double * 7)()
        self._check(self._L.bym_serve_stats(self._h, a))
        return {"count": int(a[0]), "p50_s": a[1], "p99_s": a[2], "run_p50_s": a[3], "run_p99_s": a[4],
                "mean_queue_s": a[5], "peak_hbm_bytes": a[6]}

    def batch_graph(self, items):
        """As batch_run, but all requests captured into one CUDA graph and launched once."""
        return self.batch_run(items, graph=True)

    def batch_plan(self, items, n_streams=0):
        """A captured batch kept for repeated launches: BatchPlan.launch() returns the outputs."""
        return BatchPlan(self, items, n_streams)

    def batch_run(self, items, graph=False):
        """items: list of dicts with gal, ran, params, kedges, redges, ran_nbar.  Returns outputs."""
        n = len(items)
        reqs = (Request * n)()
        ress = (Result * n)()
        outs, keeps = [], []
        for i, it in enumerate(items):
            rq, rs, out, keep = self._request(it["gal"], it.get("ran"), it["params"], it.get("kedges"),
                                              it.get("redges"), it.get("gal_nbar"), it.get("ran_nbar"))
            reqs[i], ress[i] = rq, rs
            outs.append(out)
            keeps.append(keep)
        status = (ctypes.c_int * n)()
        fn = self._L.bym_batch_graph if graph else self._L.bym_batch_run
        rc = fn(self._h, n, reqs, ress, status)
        for i in range(n):
            if status[i] != BYM_OK:
                raise BymError(status[i], f"batch item {i} failed: {self.last_error()}")
        self._check(rc)
        return outs

    def pk_multipoles(self, gal, ran, params, kedges, gal_nbar=None, ran_nbar=None, stream=None):
        return self._run("pk", gal, ran, params, kedges, None, gal_nbar, ran_nbar, stream)

    def xi_multipoles(self, gal, ran, params, redges, gal_nbar=None, ran_nbar=None, stream=None):
        return self._run("xi", gal, ran, params, None, redges, gal_nbar, ran_nbar, stream)

    def pk_xi_multipoles(self, gal, ran, params, kedges, redges, gal_nbar=None, ran_nbar=None, stream=None):
        return self._run("both", gal, ran, params, kedges, redges, gal_nbar, ran_nbar, stream)

    def pk_xi_cross(self, gal_a, ran_a, gal_b, ran_b, params, kedges=None, redges=None, ran_nbar_a=None,
                    ran_nbar_b=None, stream=None, odd=False):
        """Cross multipoles of tracer A (gal_a, ran_a) with tracer B (gal_b, ran_b): even ell up to
        params.ell_max, or with odd the odd ell = 1, 3, .., params.ell_max (odd; not the parity-even
        midpoint form); P_ell when kedges is given, xi_ell when redges is given."""
        if kedges is None and redges is None:
            raise ValueError("kedges or redges is required")
        keep = []
        cats = [_catalog(gal_a, None, keep), _catalog(ran_a, ran_nbar_a, keep), _catalog(gal_b, None, keep),
                _catalog(ran_b, ran_nbar_b, keep)]
        nl = (params.ell_max + 1) // 2 if odd else params.ell_max // 2 + 1
        dp = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        out, ptrs = {}, []
        for edges, keys in ((kedges, ("pk", "k_mean", "n_modes")), (redges, ("xi", "r_mean", "n_cells"))):
            if edges is None:
                ptrs += [None, None, None, None]
                continue
            b = _bins(edges, keep)
            keep.append(b)
            out[keys[0]] = np.zeros((nl, b.nbins))
            out[keys[1]] = np.zeros(b.nbins)
            out[keys[2]] = np.zeros(b.nbins, dtype=np.int64)
            ptrs += [ctypes.byref(b), out[keys[0]].ctypes.data_as(dp), out[keys[1]].ctypes.data_as(dp),
                     out[keys[2]].ctypes.data_as(i64p)]
        st = ctypes.c_void_p(stream) if stream else None
        fn = self._L.bym_pk_xi_cross_odd if odd else self._L.bym_pk_xi_cross
        rc = fn(self._h, *[_ptr(c) for c in cats], ctypes.byref(params), ptrs[0], ptrs[4],
                ptrs[1], ptrs[2], ptrs[3], ptrs[5], ptrs[6], ptrs[7], st)
        self._check(rc)
        out["ells"] = list(range(1 if odd else 0, params.ell_max + 1, 2))
        return out

    def shot_noise(self, gal, ran, params, gal_nbar=None, ran_nbar=None) -> float:
        """(sum_g w^2 + alpha_r^2 sum_r w^2) / A, the shot-noise level of P_0 (not subtracted by the estimators)."""
        keep = []
        g = _catalog(gal, gal_nbar, keep)
        r = _catalog(ran, ran_nbar, keep)
        out = ctypes.c_double(0.0)
        self._check(self._L.bym_shot_noise(self._h, ctypes.byref(g), ctypes.byref(r) if r is not None else None,
                                           ctypes.byref(params), ctypes.byref(out)))
        return out.value


class BatchPlan:
    """A batch of requests captured once as a CUDA graph (bym_batch_plan_*).  Each launch()
    recomputes every request from the current contents of its catalogs (device catalogs can
    be rewritten in place between launches; host catalogs were copied at creation)."""

    def __init__(self, ctx, items, n_streams=0):
        self._ctx, self._L = ctx, ctx._L
        n = len(items)
        self._reqs = (Request * n)()
        self._ress = (Result * n)()
        self.outputs, self._keeps = [], []
        for i, it in enumerate(items):
            rq, rs, out, keep = ctx._request(it["gal"], it.get("ran"), it["params"], it.get("kedges"),
                                             it.get("redges"), it.get("gal_nbar"), it.get("ran_nbar"))
            self._reqs[i], self._ress[i] = rq, rs
            self.outputs.append(out)
            self._keeps.append(keep)
        self._n = n
        self._h = ctypes.c_void_p()
        status = (ctypes.c_int * n)()
        rc = self._L.bym_batch_plan_create(ctx._h, n, self._reqs, self._ress, int(n_streams), ctypes.byref(self._h),
                                           status)
        for i in range(n):
            if status[i] != BYM_OK:
                msg = ctx.last_error()
                self.close()
                raise BymError(status[i], f"batch item {i} failed: {msg}")
        ctx._check(rc)

    def launch(self):
        status = (ctypes.c_int * self._n)()
        rc = self._L.bym_batch_plan_launch(self._h, status)
        for i in range(self._n):
            if status[i] != BYM_OK:
                raise BymError(status[i], f"batch item {i} failed: {self._ctx.last_error()}")
        self._ctx._check(rc)
        return self.outputs

    def close(self):
        if self._h:
            self._L.bym_batch_plan_destroy(self._h)
            self._h = ctypes.c_void_p()


def footprint(params: Params, n_gal: int, n_ran: int, want_pk=True, want_xi=True) -> int:
    n = ctypes.c_size_t()
    rc = lib().bym_footprint(ctypes.byref(params), int(n_gal), int(n_ran), int(want_pk), int(want_xi),
                             ctypes.byref(n))
    if rc != BYM_OK:
        raise BymError(rc, "bym_footprint failed")
    return n.value


def jit_check(params: Params) -> str:
    buf = ctypes.create_string_buffer(1 << 16)
    rc = lib().bym_jit_check(ctypes.byref(params), buf, len(buf))
    if rc != BYM_OK:
        raise BymError(rc, buf.value.decode(errors="replace"))
    return buf.value.decode(errors="replace")


def version() -> str:
    return lib().bym_version().decode()
