"""GB300 (sm_103a) marching-on-in-time solver for the quasi-Helmholtz projected TD-CFIE.

Thin Python layer over the C ABI in include/tdcfie.h (libtdcfie.so, built in-tree).  PyTorch is
used only for device memory and streams; every step of the march runs in the library's CUDA
kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import BF16X3, FP16X3, FP32, FP64, TdcfieError  # noqa: F401

__all__ = ["Solver", "Batch", "block_gemv", "block_gemv_noalloc", "tc_gemm", "mlp_grad", "mlp_train", "mlp_predict", "mlp_samples",
           "FP64", "FP32", "BF16X3", "FP16X3", "TdcfieError"]


def block_gemv(blocks, x, out=None, stream=None):
    """out[r][i] = sum_q sum_j blocks[q][i][j] x[q][r][j] through tdcfie_block_gemv.

    blocks (nblk, n, n) and x (nblk, R, n): contiguous CUDA tensors, both float64 or both float32."""
    import torch
    nblk, n, _ = blocks.shape
    R = x.shape[1]
    if out is None:
        out = torch.empty((R, n), dtype=blocks.dtype, device=blocks.device)
    prec = FP64 if blocks.dtype == torch.float64 else FP32
    s = stream if stream is not None else torch.cuda.current_stream(blocks.device).cuda_stream
    _lib.check(_lib.load().tdcfie_block_gemv(prec, ctypes.c_void_p(blocks.data_ptr()), nblk, n,
                                             ctypes.c_void_p(x.data_ptr()), R, ctypes.c_void_p(out.data_ptr()),
                                             ctypes.c_void_p(s)))
    return out


def block_gemv_noalloc(blocks, x, out, stream=None):
    """block_gemv through tdcfie_block_gemv_noalloc: no device allocation by the library (the caller
    provides `out`; partial sums use the library's 32 MiB static device scratch)."""
    import torch
    nblk, n, _ = blocks.shape
    R = x.shape[1]
    prec = FP64 if blocks.dtype == torch.float64 else FP32
    s = stream if stream is not None else torch.cuda.current_stream(blocks.device).cuda_stream
    _lib.check(_lib.load().tdcfie_block_gemv_noalloc(prec, ctypes.c_void_p(blocks.data_ptr()), nblk, n,
                                                     ctypes.c_void_p(x.data_ptr()), R,
                                                     ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(s)))
    return out


def tc_gemm(blocks, x, precision=FP16X3, out=None, stream=None):
    """out[r][i] = sum_q sum_j blocks[q][i][j] x[q][r][j] in the split tensor-core arithmetic of the
    FP16X3 / BF16X3 paths, through tdcfie_tc_gemm.

    blocks (nblk, rows, cols) and x (nblk, 64, cols): contiguous float64 CUDA tensors; returns
    (64, rows) float64."""
    import torch
    nblk, rows, cols = blocks.shape
    R = x.shape[1]
    if out is None:
        out = torch.empty((R, rows), dtype=torch.float64, device=blocks.device)
    s = stream if stream is not None else torch.cuda.current_stream(blocks.device).cuda_stream
    _lib.check(_lib.load().tdcfie_tc_gemm(int(precision), ctypes.c_void_p(blocks.data_ptr()), nblk, rows, cols,
                                          ctypes.c_void_p(x.data_ptr()), R, ctypes.c_void_p(out.data_ptr()),
                                          ctypes.c_void_p(s)))
    return out


def _stream(t, stream):
    import torch
    return stream if stream is not None else torch.cuda.current_stream(t.device).cuda_stream


def _vp(t):
    return ctypes.c_void_p(t.data_ptr())


def mlp_grad(params, X, Y, stream=None):
    """(grad, loss) of the learned-guess network's loss (1/2n) sum (f(X) - Y)^2 through tdcfie_mlp_grad.

    params (4801,), X (n, 8), Y (n,): contiguous float32 CUDA tensors."""
    import torch
    grad = torch.empty_like(params)
    loss = torch.empty(1, dtype=torch.float32, device=params.device)
    _lib.check(_lib.load().tdcfie_mlp_grad(_vp(params), _vp(X), _vp(Y), X.shape[0], _vp(grad), _vp(loss),
                                           ctypes.c_void_p(_stream(params, stream))))
    return grad, loss


def mlp_train(params, X, Y, epochs: int, batch: int = 4096, lr: float = 1e-3, seed: int = 0, stream=None):
    """Adam training in place through tdcfie_mlp_train; returns the per-pass mean loss (numpy)."""
    hist = np.zeros(int(epochs), dtype=np.float32)
    _lib.check(_lib.load().tdcfie_mlp_train(_vp(params), _vp(X), _vp(Y), X.shape[0], int(epochs), int(batch),
                                            float(lr), int(seed), _lib._ptr(hist),
                                            ctypes.c_void_p(_stream(params, stream))))
    return hist


def mlp_predict(params, X, stream=None):
    """f(X) with FP16-rounded weights through tdcfie_mlp_predict."""
    import torch
    out = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
    _lib.check(_lib.load().tdcfie_mlp_predict(_vp(params), _vp(X), X.shape[0], _vp(out),
                                              ctypes.c_void_p(_stream(params, stream))))
    return out


def mlp_samples(y, base: str = "prev", stream=None):
    """(X, Y) training samples of a stored march y (nt, R, ne) through tdcfie_mlp_samples; the target
    is the correction to base "prev" (y_{n-1}) or "extrap" (cubic extrapolation)."""
    import torch
    nt, R, ne = y.shape
    ns = (nt - 8) * R * ne
    X = torch.empty((ns, 8), dtype=torch.float32, device=y.device)
    Y = torch.empty(ns, dtype=torch.float32, device=y.device)
    prec = FP64 if y.dtype == torch.float64 else FP32
    _lib.check(_lib.load().tdcfie_mlp_samples(prec, {"prev": 0, "extrap": 1}[base], _vp(y), nt, R, ne, _vp(X), _vp(Y),
                                              ctypes.c_void_p(_stream(y, stream))))
    return X, Y


_FORM = {"dense": 0, "factored": 1}
_SOLVE = {"direct": _lib.SOLVE_DIRECT, "gmres": _lib.SOLVE_GMRES}
_GUESS = {"zero": _lib.GUESS_ZERO, "prev": _lib.GUESS_PREV, "mlp": _lib.GUESS_MLP, "extrap": _lib.GUESS_EXTRAP,
          "mlp_extrap": _lib.GUESS_MLP_EXTRAP}
_PREC = {"fp64": FP64, "fp32": FP32, "bf16x3": BF16X3, "fp16x3": FP16X3}


class Solver:
    """One scatterer: create (host tables) -> assemble (device, FP64) -> march/step (hot path)."""

    def __init__(self, V, F, dt: float, nt: int, alpha: float = 1.0, precision="fp64", R: int = 1,
                 stream=None, device: int = 0, solver: str = "direct", gmres_tol: float | None = None,
                 gmres_restart: int | None = None, gmres_maxit: int | None = None, guess: str | None = None,
                 time_order: int = 1):
        L = _lib.load()
        self._V = np.ascontiguousarray(V, dtype=np.float64)
        self._F = np.ascontiguousarray(F, dtype=np.int32)
        o = _lib.default_opts()
        o.precision = _PREC[precision] if isinstance(precision, str) else int(precision)
        o.max_rhs = int(R)
        o.device = int(device)
        o.stream = ctypes.c_void_p(stream) if stream else None
        o.solver = _SOLVE[solver]
        o.time_order = int(time_order)
        if gmres_tol is not None:
            o.gmres_tol = float(gmres_tol)
        if gmres_restart is not None:
            o.gmres_restart = int(gmres_restart)
        if gmres_maxit is not None:
            o.gmres_maxit = int(gmres_maxit)
        if guess is not None:
            o.guess = _GUESS[guess]
        self.precision = o.precision
        self.R = int(R)
        self.nt = int(nt)
        h = ctypes.c_void_p()
        _lib.check(L.tdcfie_create(_lib._ptr(self._V), self._V.shape[0], _lib._ptr(self._F), self._F.shape[0],
                                   float(dt), int(nt), float(alpha), ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        ne, nc, nv, K = (ctypes.c_int64() for _ in range(4))
        g = ctypes.c_int32()
        D = ctypes.c_double()
        _lib.check(L.tdcfie_info(h, ctypes.byref(ne), ctypes.byref(nc), ctypes.byref(nv), ctypes.byref(K),
                                 ctypes.byref(g), ctypes.byref(D)), h)
        self.ne, self.nc, self.nv, self.K, self.genus, self.D = ne.value, nc.value, nv.value, K.value, g.value, D.value

    # ------------------------------------------------------------------ host queries
    def topology(self):
        E = np.zeros((self.ne, 2), dtype=np.int32)
        cp = np.zeros(self.ne, dtype=np.int32)
        cm = np.zeros(self.ne, dtype=np.int32)
        _lib.check(_lib.load().tdcfie_topology(self._h, _lib._ptr(E), _lib._ptr(cp), _lib._ptr(cm)), self._h)
        return E, cp, cm

    def bc_table(self):
        L = _lib.load()
        n = ctypes.c_int64()
        _lib.check(L.tdcfie_bc_table(self._h, ctypes.byref(n), None, None, None, None, None), self._h)
        ft = np.zeros(n.value, dtype=np.int32)
        fn = np.zeros(n.value, dtype=np.int32)
        ph = np.zeros((n.value, 3), dtype=np.float64)
        fV = np.zeros((self.nv + self.ne + self.nc, 3), dtype=np.float64)
        fF = np.zeros((6 * self.nc, 3), dtype=np.int32)
        _lib.check(L.tdcfie_bc_table(self._h, ctypes.byref(n), _lib._ptr(ft), _lib._ptr(fn), _lib._ptr(ph),
                                     _lib._ptr(fV), _lib._ptr(fF)), self._h)
        return ft, fn, ph, fV, fF

    # ------------------------------------------------------------------ device work
    def assemble(self):
        _lib.check(_lib.load().tdcfie_assemble(self._h), self._h)
        return self

    def matrix(self, which: str, k: int = 0) -> np.ndarray:
        ids = {"T": 0, "S": 1, "H": 2, "MM": 3, "G": 4, "Zs": 5, "Zh": 6, "M": 7, "PS": 8, "L1": 9, "L2": 10,
               "Phi": 11}
        n = self.nc if which == "Phi" else self.ne
        out = np.zeros((n, n), dtype=np.float64)
        _lib.check(_lib.load().tdcfie_get_matrix(self._h, ids[which], int(k), _lib._ptr(out)), self._h)
        return out

    def _pw(self, pw: dict):
        arrs = [np.ascontiguousarray(pw[k], dtype=np.float64) for k in ("k", "p", "amp", "t0", "sigma")]
        self._pw_keep = arrs
        return _lib.PlaneWaves(arrs[0].shape[0], *(a.ctypes.data for a in arrs))

    def set_excitation(self, pw: dict):
        p = self._pw(pw)
        _lib.check(_lib.load().tdcfie_set_excitation(self._h, ctypes.byref(p)), self._h)

    def step(self, nsteps: int, out=None):
        """out: torch CUDA tensor (nsteps, R, ne) of the path dtype, or None to discard."""
        ptr = None if out is None else ctypes.c_void_p(out.data_ptr())
        _lib.check(_lib.load().tdcfie_step(self._h, int(nsteps), ptr), self._h)

    def step_y(self, nsteps: int, out=None, y_out=None):
        """step() that also writes y_n (nsteps, R, ne) of the path dtype to y_out."""
        ptr = None if out is None else ctypes.c_void_p(out.data_ptr())
        yp = None if y_out is None else ctypes.c_void_p(y_out.data_ptr())
        _lib.check(_lib.load().tdcfie_step_y(self._h, int(nsteps), ptr, yp), self._h)

    def gmres_stats(self):
        v = [ctypes.c_int64() for _ in range(4)]
        _lib.check(_lib.load().tdcfie_gmres_stats(self._h, *(ctypes.byref(x) for x in v)), self._h)
        return dict(zip(("iterations", "steps", "max_per_step", "not_converged"), (x.value for x in v)))

    def replan(self, precision: str, R: int):
        """Rebuild the step plan for another path precision / number of waves (tdcfie_replan)."""
        o = _PREC[precision] if isinstance(precision, str) else int(precision)
        _lib.check(_lib.load().tdcfie_replan(self._h, o, int(R)), self._h)
        self.precision, self.R = o, int(R)

    def set_solver(self, solver: str = "gmres", guess: str = "prev", gmres_tol: float = 1e-8):
        """Switch the per-step solve of the assembled handle (tdcfie_set_solver)."""
        _lib.check(_lib.load().tdcfie_set_solver(self._h, _SOLVE[solver], _GUESS[guess], float(gmres_tol)), self._h)

    def set_history_form(self, form: str = "factored"):
        """Stream the dense T_k ("dense") or the shell-sparse retarded matrices ("factored") in the
        history sum (tdcfie_set_history_form); the excitation must be set again."""
        _lib.check(_lib.load().tdcfie_set_history_form(self._h, _FORM[form]), self._h)

    def history_stats(self):
        """Form of the current plan, shell nonzeros and algorithmic bytes per step (tdcfie_history_stats)."""
        f, n = ctypes.c_int32(), ctypes.c_int64()
        a, b = ctypes.c_double(), ctypes.c_double()
        _lib.check(_lib.load().tdcfie_history_stats(self._h, ctypes.byref(f), ctypes.byref(n), ctypes.byref(a),
                                                    ctypes.byref(b)), self._h)
        return {"form": ("dense", "factored")[f.value], "nnz": n.value, "history_bytes": a.value,
                "step_bytes": b.value}

    def set_formulation(self, formulation: str = "mfie"):
        """March the qHP TD-CFIE ("qhp") or the mixed TD-MFIE comparison formulation ("mfie") on the
        same matrices (tdcfie_set_formulation); the excitation must be set again."""
        _lib.check(_lib.load().tdcfie_set_formulation(self._h, {"qhp": 0, "mfie": 1}[formulation]), self._h)

    def far_field(self, currents, w: float, rhat):
        """Far-field amplitude (ndir, R, 3) complex at angular frequency w of the currents (torch CUDA
        tensor (nt, R, ne) from step()/march() starting at the first step) (tdcfie_far_field)."""
        d = np.ascontiguousarray(np.atleast_2d(np.asarray(rhat, dtype=np.float64)))
        out = np.zeros((d.shape[0], self.R, 3, 2), dtype=np.float64)
        _lib.check(_lib.load().tdcfie_far_field(self._h, ctypes.c_void_p(currents.data_ptr()), int(currents.shape[0]),
                                                float(w), _lib._ptr(d), d.shape[0], _lib._ptr(out)), self._h)
        return out[..., 0] + 1j * out[..., 1]

    def mlp_load(self, params):
        """Load 4801 learned-guess parameters (array-like, float32) into the march."""
        a = np.ascontiguousarray(np.asarray(params, dtype=np.float32).ravel())
        assert a.size == _lib.MLP_NPARAM
        _lib.check(_lib.load().tdcfie_mlp_load(self._h, _lib._ptr(a)), self._h)

    def march(self, pw: dict, out=None, out_on_host: bool = False):
        p = self._pw(pw)
        if out is None:
            ptr = None
        elif isinstance(out, np.ndarray):
            ptr = _lib._ptr(out)
        else:
            ptr = ctypes.c_void_p(out.data_ptr())
        _lib.check(_lib.load().tdcfie_march(self._h, ctypes.byref(p), ptr, int(out_on_host)), self._h)

    def timing(self):
        a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        n = ctypes.c_int64()
        _lib.check(_lib.load().tdcfie_last_timing(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                                  ctypes.byref(n)), self._h)
        return {"step_ms": a.value, "history_ms": b.value, "history_bytes": c.value, "launches": n.value}

    def assembly_timing(self):
        """Seconds per assembly phase: upload, retarded EFIE, retarded MFIE, static, formation, plan."""
        out = np.zeros(6)
        _lib.check(_lib.load().tdcfie_assembly_timing(self._h, _lib._ptr(out)), self._h)
        return dict(zip(("upload", "retarded_efie", "retarded_mfie", "static", "formation", "plan"), out.tolist()))

    def release_assembly(self):
        """Free the FP64 assembly matrices; the march keeps working (tdcfie_release_assembly)."""
        _lib.check(_lib.load().tdcfie_release_assembly(self._h), self._h)

    def close(self):
        if getattr(self, "_h", None):
            _lib.load().tdcfie_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.precision == FP64 else torch.float32


class Batch:
    """Several assembled Solvers stepped by one graph launch per step (tdcfie_batch_*).

    The solvers are borrowed: keep them alive and close the batch first."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        arr = (ctypes.c_void_p * len(self.solvers))(*[s._h.value for s in self.solvers])
        b = ctypes.c_void_p()
        _lib.check(_lib.load().tdcfie_batch_create(arr, len(self.solvers), ctypes.byref(b)))
        self._b = b

    def step(self, nsteps: int, outs=None):
        """outs: None, or one torch CUDA tensor (nsteps, R, ne) of the path dtype (or None) per solver."""
        ptrs = None
        if outs is not None:
            ptrs = (ctypes.c_void_p * len(outs))(*[None if o is None else o.data_ptr() for o in outs])
        _lib.check(_lib.load().tdcfie_batch_step(self._b, int(nsteps), ptrs))

    def tune(self, steps_per_candidate: int = 3):
        """Measure the persistent kernel's launch shapes and keep the fastest (tdcfie_batch_tune);
        the members are reset to the start of their march.  Returns the chosen configuration."""
        cfg = np.zeros(4, dtype=np.int32)
        _lib.check(_lib.load().tdcfie_batch_tune(self._b, int(steps_per_candidate), _lib._ptr(cfg)))
        return dict(zip(("persistent", "rows_per_warp", "threads", "blocks_per_sm"), cfg.tolist()))

    def timing(self):
        ms, n = ctypes.c_double(), ctypes.c_int64()
        _lib.check(_lib.load().tdcfie_batch_timing(self._b, ctypes.byref(ms), ctypes.byref(n)))
        return {"step_ms": ms.value, "launches": n.value}

    def close(self):
        if getattr(self, "_b", None):
            _lib.load().tdcfie_batch_destroy(self._b)
            self._b = None
