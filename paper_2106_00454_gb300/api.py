"""Python binding of the C ABI (argument marshalling only).

Device buffers are torch tensors (float64, on the context's device); the
context stream is a torch CUDA stream.  Every computation runs in libwpcd's
kernels; this module only converts arguments and raises on error codes.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from . import inputs as W

WPCD_OK = 0
WPCD_ERR_NOTREADY = -7
PREC_FP64, PREC_MIXED = 0, 1
AVG_FREE_BIN, AVG_SWP_INDEX, POINT = 0, 1, 2  # resolvent (wpcd_resolvent)
EXEC_BATCHED, EXEC_PLAIN = 0, 1
REFINE_TENSOR, REFINE_FP64 = 0, 1
OPT_EXEC, OPT_REFINE, OPT_AUTOTUNE, OPT_GRAPH, OPT_BIG_SLOTS, OPT_ROTATE, OPT_REFINE_ITERS, OPT_REFINE_DIGITS = \
    1, 2, 3, 4, 5, 6, 7, 8


class WpcdError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = _lib.load().wpcd_strerror(code).decode()
        super().__init__(f"{where}: {msg} ({code})")
        self.code = code


def _ck(code: int, where: str):
    if code != WPCD_OK:
        raise WpcdError(code, where)


def _ptr(t):
    """Device (or host numpy) pointer of a contiguous float64/int32 buffer, or None."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        assert t.flags.c_contiguous
        return ctypes.c_void_p(t.ctypes.data)
    assert t.is_contiguous(), "buffers must be contiguous"
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """One libwpcd context bound to a CUDA device and a torch stream."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, stream=None):
        import torch
        self._torch = torch
        self.lib = _lib.load()
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        h = ctypes.c_void_p()
        _ck(self.lib.wpcd_create(ctypes.byref(h), device, hbm_budget_bytes, ctypes.c_void_p(self.stream.cuda_stream)),
            "wpcd_create")
        self.h = h
        self.refine_engine = REFINE_TENSOR  # the library's default

    def close(self):
        if self.h:
            self.lib.wpcd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ options / sync
    def set_exec(self, mode: int):
        _ck(self.lib.wpcd_set_option(self.h, OPT_EXEC, mode), "wpcd_set_option")

    def set_refine_engine(self, engine: int):
        _ck(self.lib.wpcd_set_option(self.h, OPT_REFINE, engine), "wpcd_set_option")
        self.refine_engine = engine

    def batched_dgemm(self, A, B, C, trans_a=False, engine=REFINE_TENSOR):
        """C[b] = op(A[b]) @ B[b] for (items, n, n) float64 device tensors."""
        items, n, _ = A.shape
        _ck(self.lib.wpcd_batched_dgemm(self.h, n, items, 1 if trans_a else 0, _ptr(A), _ptr(B), _ptr(C), engine),
            "wpcd_batched_dgemm")

    def set_interp_point(self, frac: float):
        """Interpolation point of every bin as a fraction of it (Sec. 5.1.1; 0.5 = midpoint)."""
        _ck(self.lib.wpcd_set_interp_point(self.h, float(frac)), "wpcd_set_interp_point")

    def set_refine_iters(self, iters: int):
        """FP64 refinement iterations of the mixed path (1..4, default 2)."""
        _ck(self.lib.wpcd_set_option(self.h, OPT_REFINE_ITERS, int(iters)), "wpcd_set_option")

    def set_refine_digits(self, digits: int):
        """Digits per operand of the mixed path's refinement products (4..6, default 6)."""
        _ck(self.lib.wpcd_set_option(self.h, OPT_REFINE_DIGITS, int(digits)), "wpcd_set_option")

    def set_rotate(self, on: bool):
        """Mixed path: FP32 eigensolve in the mean-potential eigenbasis (default on)."""
        _ck(self.lib.wpcd_set_option(self.h, OPT_ROTATE, 1 if on else 0), "wpcd_set_option")

    def set_big_slots(self, slots: int):
        """CTAs of the global-memory eigensolver (0 = automatic)."""
        _ck(self.lib.wpcd_set_option(self.h, OPT_BIG_SLOTS, int(slots)), "wpcd_set_option")

    def set_autotune(self, on: bool):
        _ck(self.lib.wpcd_set_option(self.h, OPT_AUTOTUNE, 1 if on else 0), "wpcd_set_option")

    def set_graphs(self, on: bool):
        _ck(self.lib.wpcd_set_option(self.h, OPT_GRAPH, 1 if on else 0), "wpcd_set_option")

    def device_log(self, x, y):
        """y = the resolvent kernel's log(x), elementwise (float64 device tensors)."""
        _ck(self.lib.wpcd_device_log(self.h, _ptr(x), _ptr(y), x.numel()), "wpcd_device_log")

    def graph_stats(self) -> dict:
        cap, rep, cached = ctypes.c_ulonglong(0), ctypes.c_ulonglong(0), ctypes.c_int(0)
        _ck(self.lib.wpcd_graph_stats(self.h, ctypes.byref(cap), ctypes.byref(rep), ctypes.byref(cached)),
            "wpcd_graph_stats")
        return {"captures": cap.value, "replays": rep.value, "cached": cached.value}

    def tuning(self) -> list:
        m = 64
        n = np.zeros(m, dtype=np.int32)
        p = np.zeros(m, dtype=np.int32)
        t = np.zeros(m, dtype=np.int32)
        ms = np.zeros(5 * m, dtype=np.float32)
        k = self.lib.wpcd_tuning(self.h, m, _ptr(n), _ptr(p), _ptr(t), _ptr(ms))
        return [{"n": int(n[i]), "precision": ("fp64", "mixed")[int(p[i])], "threads": int(t[i]),
                 "ms_per_solve": {c: float(ms[5 * i + j]) for j, c in enumerate((64, 128, 256, 512, 1024))}}
                for i in range(k)]

    def sync(self):
        _ck(self.lib.wpcd_sync(self.h), "wpcd_sync")

    def sync_status(self) -> int:
        return self.lib.wpcd_sync(self.h)

    def bytes_in_use(self) -> int:
        return self.lib.wpcd_bytes_in_use(self.h)

    PHASES = ["mesh", "project", "eigen", "plan", "tmatrix", "gather", "observables", "refine", "mi"]

    def kernel_launches(self) -> int:
        return int(self.lib.wpcd_kernel_launches(self.h))

    def profile(self, enable: bool):
        _ck(self.lib.wpcd_profile(self.h, 1 if enable else 0), "wpcd_profile")

    def profile_read(self) -> dict:
        out = {}
        for k, name in enumerate(self.PHASES):
            ms, n = ctypes.c_double(), ctypes.c_long()
            _ck(self.lib.wpcd_profile_read(self.h, k, ctypes.byref(ms), ctypes.byref(n)), "wpcd_profile_read")
            out[name] = (ms.value, n.value)
        return out

    def release(self, hid: int):
        _ck(self.lib.wpcd_release(self.h, hid), "wpcd_release")

    # ------------------------------------------------------------------ mesh / projection
    def mesh(self, n_wp, kind=W.MESH_KIND_CAPPED, alpha=W.MESH_ALPHA_FM, t=W.MESH_T, kmax=W.MESH_KMAX_FM,
             n_quad=W.MESH_Q, wp_kind=W.WP_MOMENTUM) -> int:
        mid = ctypes.c_int()
        _ck(self.lib.wpcd_mesh(self.h, n_wp, kind, alpha, t, kmax, n_quad, wp_kind, ctypes.byref(mid)), "wpcd_mesh")
        return mid.value

    def mesh_get(self, mesh_id, n_wp, n_quad):
        kb = np.zeros(n_wp + 1)
        kq = np.zeros(n_wp * n_quad)
        wq = np.zeros(n_wp * n_quad)
        _ck(self.lib.wpcd_mesh_get(self.h, mesh_id, _ptr(kb), _ptr(kq), _ptr(wq)), "wpcd_mesh_get")
        return kb, kq, wq

    def project(self, mesh_ids, channels, gen, gen_params, n_terms, v_fine=None, prec=PREC_FP64) -> int:
        """Projected potential set; prec = PREC_MIXED: angle integrals on the tensor cores (Yukawa)."""
        n = len(channels)
        arr = (_lib.wpcd_channel * n)(*[_lib.wpcd_channel(*c.astuple()) if hasattr(c, "astuple")
                                        else _lib.wpcd_channel(*c) for c in channels])
        mids = (ctypes.c_int * n)(*mesh_ids)
        gp = None if gen_params is None else np.ascontiguousarray(gen_params, dtype=np.float64)
        vid = ctypes.c_int()
        _ck(self.lib.wpcd_project_prec(self.h, mids, arr, n, gen, _ptr(gp), 0 if gp is None else gp.size,
                                       _ptr(v_fine), n_terms, prec, ctypes.byref(vid)), "wpcd_project_prec")
        return vid.value

    def vset_info(self, vset_id, channel=0):
        nch, nterm, n = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _ck(self.lib.wpcd_vset_info(self.h, vset_id, ctypes.byref(nch), ctypes.byref(nterm), channel,
                                    ctypes.byref(n)), "wpcd_vset_info")
        return nch.value, nterm.value, n.value

    def vset_get(self, vset_id, channel):
        _, nterm, n = self.vset_info(vset_id, channel)
        out = np.zeros((nterm, n, n))
        _ck(self.lib.wpcd_vset_get(self.h, vset_id, channel, _ptr(out)), "wpcd_vset_get")
        return out

    # ------------------------------------------------------------------ hot path
    def diag(self, vset_id, coeffs, n_samples, prec=PREC_FP64) -> int:  # noqa: D401
        eid = ctypes.c_int()
        _ck(self.lib.wpcd_diag(self.h, vset_id, _ptr(coeffs), n_samples, prec, ctypes.byref(eid)), "wpcd_diag")
        return eid.value

    def diag_status(self, eig_id, out):
        _ck(self.lib.wpcd_diag_status(self.h, eig_id, _ptr(out)), "wpcd_diag_status")

    def eig_get(self, eig_id, sample, channel, n):
        eps = np.zeros(n)
        C = np.zeros((n, n))
        _ck(self.lib.wpcd_eig_get(self.h, eig_id, sample, channel, _ptr(eps), _ptr(C)), "wpcd_eig_get")
        return eps, C

    def tmatrix(self, eig_id, e_lab, t_out, res=AVG_FREE_BIN):
        _ck(self.lib.wpcd_tmatrix(self.h, eig_id, _ptr(e_lab), e_lab.numel(), res, _ptr(t_out)), "wpcd_tmatrix")

    def observables(self, eig_id, e_lab, delta=None, sigma=None, res=AVG_FREE_BIN):
        if res == AVG_FREE_BIN:
            _ck(self.lib.wpcd_observables(self.h, eig_id, _ptr(e_lab), e_lab.numel(), _ptr(delta), _ptr(sigma)),
                "wpcd_observables")
        else:
            _ck(self.lib.wpcd_observables_res(self.h, eig_id, _ptr(e_lab), e_lab.numel(), res, _ptr(delta),
                                              _ptr(sigma)), "wpcd_observables_res")

    def solve(self, vset_id, coeffs, n_samples, e_lab, t_out=None, delta=None, sigma=None, prec=PREC_FP64,
              res=AVG_FREE_BIN):
        _ck(self.lib.wpcd_solve(self.h, vset_id, _ptr(coeffs), n_samples, _ptr(e_lab), e_lab.numel(), prec,
                                res, _ptr(t_out), _ptr(delta), _ptr(sigma)), "wpcd_solve")

    # ------------------------------------------------------------------ spin observables
    def saclay(self, channels, delta, n_samples, e_lab, theta, abcde=None, dsig=None):
        """Saclay amplitudes (abcde: float64 device tensor [S, n_E, n_theta, 5, 2])
        and dsigma/dOmega (dsig: [S, n_E, n_theta] mb/sr) from the phases delta
        [S, n_ch, n_E, 3] of the channels, at angles theta (radians)."""
        n = len(channels)
        arr = (_lib.wpcd_channel * n)(*[_lib.wpcd_channel(*c.astuple()) if hasattr(c, "astuple")
                                        else _lib.wpcd_channel(*c) for c in channels])
        _ck(self.lib.wpcd_saclay(self.h, arr, n, _ptr(delta), n_samples, _ptr(e_lab), e_lab.numel(), _ptr(theta),
                                 theta.numel(), _ptr(abcde), _ptr(dsig)), "wpcd_saclay")

    # ------------------------------------------------------------------ MI comparison method
    def mi_prepare(self, channels, gen, gen_params, n_terms, n_quad=96, c_map=1.0) -> int:
        n = len(channels)
        arr = (_lib.wpcd_channel * n)(*[_lib.wpcd_channel(*c.astuple()) if hasattr(c, "astuple")
                                        else _lib.wpcd_channel(*c) for c in channels])
        gp = np.ascontiguousarray(gen_params, dtype=np.float64)
        mid = ctypes.c_int()
        _ck(self.lib.wpcd_mi_prepare(self.h, arr, n, gen, _ptr(gp), gp.size, n_terms, n_quad, float(c_map),
                                     ctypes.byref(mid)), "wpcd_mi_prepare")
        return mid.value

    def mi_solve(self, mi_id, coeffs, n_samples, e_int, e_lab, k_out=None, delta=None, sigma=None, status=None):
        """MI at the interpolation energies e_int (device tensor, MeV) and the
        phases / cross sections interpolated to e_lab (device tensor); status
        (int32 device tensor [S, n_ch]) receives the refinement step counts."""
        _ck(self.lib.wpcd_mi_solve(self.h, mi_id, _ptr(coeffs), n_samples, _ptr(e_int), e_int.numel(), _ptr(e_lab),
                                   e_lab.numel(), _ptr(k_out), _ptr(delta), _ptr(sigma), _ptr(status)),
            "wpcd_mi_solve")

    def solve_host(self, vset_id, coeffs, n_samples, e_lab, t_out=None, delta=None, sigma=None, prec=PREC_FP64,
                   res=AVG_FREE_BIN):
        e_lab = np.ascontiguousarray(e_lab, dtype=np.float64)
        coeffs = None if coeffs is None else np.ascontiguousarray(coeffs, dtype=np.float64)
        _ck(self.lib.wpcd_solve_host(self.h, vset_id, _ptr(coeffs), n_samples, _ptr(e_lab), e_lab.size, prec,
                                     res, _ptr(t_out), _ptr(delta), _ptr(sigma)), "wpcd_solve_host")


class ServedResult:
    """One finished request: delta [n_ch, n_E, 3] deg, sigma [n_E] mb, T [n_ch, n_E, 2, 2] complex."""

    def __init__(self, r):
        nch, nE = r.n_ch, r.n_E
        self.status = r.status
        self.latency_us = r.latency_us
        self.delta = np.ctypeslib.as_array(r.delta, shape=(nch * nE * 3,)).reshape(nch, nE, 3).copy()
        self.sigma = np.ctypeslib.as_array(r.sigma, shape=(nE,)).copy()
        t = np.ctypeslib.as_array(r.T, shape=(nch * nE * 8,)).copy()
        self.T = t.view(np.complex128).reshape(nch, nE, 2, 2)


def _serve_methods():
    def serve_start(self, channels, gen, gen_params, n_terms, n_wp_list, max_batch=64, n_slots=4,
                    max_queue=1 << 16):
        n = len(channels)
        arr = (_lib.wpcd_channel * n)(*[_lib.wpcd_channel(*c.astuple()) for c in channels])
        gp = np.ascontiguousarray(gen_params, dtype=np.float64)
        nw = (ctypes.c_int * len(n_wp_list))(*n_wp_list)
        _ck(self.lib.wpcd_serve_start(self.h, arr, n, gen, _ptr(gp), gp.size, n_terms, nw, len(n_wp_list),
                                      max_batch, n_slots, max_queue), "wpcd_serve_start")
        self._n_terms = n_terms

    def submit(self, coeffs, e_lab, n_wp, prec=PREC_FP64, raise_on_error=True):
        e = np.ascontiguousarray(e_lab, dtype=np.float64)
        c = None if coeffs is None else np.ascontiguousarray(coeffs, dtype=np.float64)
        rq = _lib.wpcd_request(
            None if c is None else c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0 if c is None else c.size,
            e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), e.size, n_wp, prec)
        t = ctypes.c_uint64()
        code = self.lib.wpcd_submit(self.h, ctypes.byref(rq), ctypes.byref(t))
        if code != WPCD_OK:
            if raise_on_error:
                raise WpcdError(code, "wpcd_submit")
            return code
        return t.value

    def poll(self, ticket):
        r = _lib.wpcd_result()
        code = self.lib.wpcd_poll(self.h, ticket, ctypes.byref(r))
        if code == WPCD_ERR_NOTREADY:
            return None
        _ck(code, "wpcd_poll")
        return ServedResult(r)

    def wait(self, ticket, timeout_ms=60000):
        r = _lib.wpcd_result()
        _ck(self.lib.wpcd_wait(self.h, ticket, timeout_ms, ctypes.byref(r)), "wpcd_wait")
        return ServedResult(r)

    def release_result(self, ticket):
        self.lib.wpcd_release_result(self.h, ticket)

    def serve_stop(self):
        _ck(self.lib.wpcd_serve_stop(self.h), "wpcd_serve_stop")

    def serve_stats(self):
        a, b, q = ctypes.c_ulonglong(), ctypes.c_ulonglong(), ctypes.c_ulonglong()
        _ck(self.lib.wpcd_serve_stats(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(q)), "wpcd_serve_stats")
        return {"completed": a.value, "batches": b.value, "queued": q.value}

    for f in (serve_start, submit, poll, wait, release_result, serve_stop, serve_stats):
        setattr(Context, f.__name__, f)


_serve_methods()


class Model:
    """Meshes + projected potential for one workload's channel set."""

    def __init__(self, ctx: Context, wl: W.Workload, v_fine=None, proj_prec=PREC_FP64):
        self.ctx = ctx
        self.wl = wl
        self.mesh_of_n = {}
        for n in sorted(set(wl.nwp)):
            self.mesh_of_n[n] = ctx.mesh(n, wl.mesh_kind, wl.alpha, wl.t, wl.kmax, wl.Q, wl.wp_kind)
        mids = [self.mesh_of_n[n] for n in wl.nwp]
        self.vset = ctx.project(mids, wl.channels, wl.gen if v_fine is None else -1, wl.gen_params, wl.n_terms,
                                v_fine, prec=proj_prec)

    @property
    def n_ch(self):
        return len(self.wl.channels)

    def release(self):
        """Free the projected set and the meshes."""
        self.ctx.release(self.vset)
        for mid in self.mesh_of_n.values():
            self.ctx.release(mid)
        self.mesh_of_n = {}
