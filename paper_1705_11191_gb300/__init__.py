"""Single-GPU (GB300, sm_103a) dense Kohn-Sham solver: thin ctypes binding of the C ABI
declared in ``include/elsi_gb.h`` (arXiv:1705.11191, the ELPA route driven by ELSI).

Every step of a solve runs in the CUDA kernels of ``libelsi_gb.so``; this module only
marshals arguments (torch CUDA tensors -> device pointers). There is no CPU fallback:
if the library cannot be loaded, every call raises.

Matrices are n x n float64 CUDA tensors. The library reads them column-major; for the
symmetric H and S that is the same memory as torch's row-major layout. Eigenvectors
come back as an (n, n_state) tensor whose column l is eigenvector l.
"""
from __future__ import annotations

import ctypes
import os
import threading

__all__ = ["load", "Handle", "ElsiError", "solve_dm", "solve_ev", "STAGES",
           "SOLVER_ELPA", "FORMAT_DENSE", "MODE_SINGLE_PROC", "OCC_INTEGER",
           "OCC_GAUSSIAN", "OCC_FERMI", "OCC_MP0", "OCC_MP1", "PREC_FP64", "PREC_FP32_REFINE", "LIB_PATH"]

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libelsi_gb.so")

SOLVER_ELPA, FORMAT_DENSE, MODE_MULTI_PROC, MODE_SINGLE_PROC = 1, 1, 1, 2
OCC_INTEGER, OCC_GAUSSIAN, OCC_FERMI = 0, 1, 2
OCC_MP0, OCC_MP1 = 3, 4  # Methfessel-Paxton of order 0 (= Gaussian) and 1
PREC_FP64, PREC_FP32_REFINE = 0, 1

ERR_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_UNSUPPORTED", 3: "ERR_NOT_PD",
             4: "ERR_NONFINITE", 5: "ERR_NO_CONVERGENCE", 6: "ERR_TIMEOUT",
             7: "ERR_CUDA", 8: "ERR_STATE", 9: "ERR_NOMEM", 10: "ERR_TOO_LARGE"}

_lib = None
_lock = threading.Lock()
_vp, _dp, _ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
_pp = ctypes.POINTER(ctypes.c_void_p)


class ElsiError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


def _declare(lib):
    i, d = ctypes.c_int, ctypes.c_double
    H = _vp
    sig = {
        "elsi_init": ([ctypes.POINTER(_vp), i, i, i, i, i, d], i),
        "elsi_finalize": ([ctypes.POINTER(_vp)], i),
        "elsi_set_overlap_is_unit": ([H, i], i),
        "elsi_set_broadening_scheme": ([H, i], i),
        "elsi_set_broadening_width": ([H, d], i),
        "elsi_set_occ_accuracy": ([H, d], i),
        "elsi_set_mu_max_steps": ([H, i], i),
        "elsi_set_precision": ([H, i], i),
        "elsi_set_band_width": ([H, i], i),
        "elsi_set_refine_max_iter": ([H, i], i),
        "elsi_set_stream": ([H, _vp], i),
        "elsi_set_reuse_ovlp_factor": ([H, i], i),
        "elsi_ev_real": ([H, _vp, _vp, _vp, _vp], i),
        "elsi_dm_real": ([H, _vp, _vp, _vp, _dp], i),
        "elsi_get_edm_real": ([H, _vp], i),
        "elsi_ev_complex": ([H, _vp, _vp, _vp, _vp], i),
        "elsi_dm_complex": ([H, _vp, _vp, _vp, _dp], i),
        "elsi_get_edm_complex": ([H, _vp], i),
        "elsi_get_mu": ([H, _dp], i),
        "elsi_get_occ": ([H, _vp], i),
        "elsi_get_eval": ([H, _vp], i),
        "elsi_dm_real_host": ([H, _vp, _vp, _vp, _vp, _dp], i),
        "elsi_get_stage_times": ([H, ctypes.POINTER(ctypes.c_float), i], i),
        "elsi_stage_name": ([i], ctypes.c_char_p),
        "elsi_get_refine_info": ([H, _ip, _dp], i),
        "elsi_get_last_error": ([H], ctypes.c_char_p),
        "elsi_gb_version": ([], ctypes.c_char_p),
        "elsi_gb_launch_count": ([], ctypes.c_longlong),
        "elsi_gb_set_spin_limit": ([ctypes.c_longlong], i),
        "elsi_gb_get_spin_limit": ([], ctypes.c_longlong),
        "elsi_density_noalloc": ([i, i, _vp, _vp, _vp, _vp, _vp, _vp], i),
        "elsi_dm_batched_real": ([H, i, _ip, _ip, _pp, _pp, _dp, _dp, i, _pp, _pp, _dp, _dp], i),
        "elsi_dm_batched_complex": ([H, i, _ip, _ip, _pp, _pp, _dp, _dp, i, _pp, _pp, _dp, _dp], i),
        "elsi_batch_ev_real": ([H, i, _ip, _ip, _pp, _pp, _vp], i),
        "elsi_batch_ev_complex": ([H, i, _ip, _ip, _pp, _pp, _vp], i),
        "elsi_occupation_weighted": ([H, i, _vp, _vp, d, _vp, _dp], i),
        "elsi_batch_dm": ([H, _vp, _pp, _pp, _dp], i),
        "elsi_get_entropy": ([H, _dp], i),
        "elsi_set_sing_check": ([H, i], i),
        "elsi_set_elpa_solver": ([H, i], i),
        "elsi_set_batch_streams": ([H, i], i),
        "elsi_set_batch_autotune": ([H, i], i),
        "elsi_get_batch_tuning": ([H, i, i, _ip, _ip, _ip], i),
        "elsi_set_csc": ([H, i, _vp, _vp, i], i),
        "elsi_ev_real_sparse": ([H, _vp, _vp, _vp, _vp], i),
        "elsi_dm_real_sparse": ([H, _vp, _vp, _vp, _dp], i),
        "elsi_get_edm_real_sparse": ([H, _vp], i),
        "elsi_set_sing_tol": ([H, d], i),
        "elsi_get_n_nonsing": ([H, _ip], i),
        "elsi_dm_adjoint_real": ([H, i, d, _vp, _vp, _vp, _vp], i),
        "elsi_ev_adjoint_real": ([H, i, i, _vp, _vp, _vp, _vp, _vp, _vp], i),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res


def load(path: str | None = None):
    """Load libelsi_gb.so (building it first if it is missing). Raises if impossible."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                from . import build as _build
                _build.build()
            lib = ctypes.CDLL(p)
            _declare(lib)
            _lib = lib
    return _lib


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load().elsi_gb_launch_count())


def _n_stages(lib) -> int:
    k = 0
    while lib.elsi_stage_name(k):
        k += 1
    return k


def stage_names() -> list[str]:
    lib = load()
    return [lib.elsi_stage_name(i).decode() for i in range(_n_stages(lib))]


STAGES = None


def _ptr(t, dtype=None) -> int:
    import torch
    dtype = dtype or torch.float64
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"expected a contiguous {dtype} CUDA tensor")
    return t.data_ptr()


def _colmajor(t):
    """Column-major copy of a (n, n) tensor (the library's layout); a no-op copy is
    avoided for real symmetric inputs by the callers."""
    return t.transpose(0, 1).contiguous()


class Handle:
    """An ELSI handle (sec. 4.1/4.3) bound to the current CUDA device and torch stream."""

    def __init__(self, n_basis: int, n_state: int, n_electron: float, *,
                 solver: int = SOLVER_ELPA, fmt: int = FORMAT_DENSE,
                 mode: int = MODE_SINGLE_PROC, stream=None):
        self._lib = load()
        self._h = _vp()
        rc = self._lib.elsi_init(ctypes.byref(self._h), solver, fmt, mode, int(n_basis),
                                 int(n_state), float(n_electron))
        if rc:
            raise ElsiError(rc, "elsi_init")
        self.n, self.n_state, self.n_electron = int(n_basis), int(n_state), float(n_electron)
        if stream is not None:
            self.set_stream(stream)

    # -- lifetime
    def close(self):
        if self._h:
            self._lib.elsi_finalize(ctypes.byref(self._h))
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, rc: int, what: str):
        if rc:
            msg = self._lib.elsi_get_last_error(self._h)
            raise ElsiError(rc, f"{what}: {msg.decode() if msg else ''}")

    # -- customisation
    def set_overlap_is_unit(self, v: bool):
        self._check(self._lib.elsi_set_overlap_is_unit(self._h, int(bool(v))), "set_overlap_is_unit")

    def set_broadening(self, scheme: int, width: float | None = None):
        self._check(self._lib.elsi_set_broadening_scheme(self._h, int(scheme)), "set_broadening_scheme")
        if width is not None:
            self._check(self._lib.elsi_set_broadening_width(self._h, float(width)), "set_broadening_width")

    def set_occ_accuracy(self, a: float):
        self._check(self._lib.elsi_set_occ_accuracy(self._h, float(a)), "set_occ_accuracy")

    def set_mu_max_steps(self, s: int):
        self._check(self._lib.elsi_set_mu_max_steps(self._h, int(s)), "set_mu_max_steps")

    def set_precision(self, p: int):
        self._check(self._lib.elsi_set_precision(self._h, int(p)), "set_precision")

    def set_band_width(self, b: int):
        self._check(self._lib.elsi_set_band_width(self._h, int(b)), "set_band_width")

    def set_refine_max_iter(self, it: int):
        self._check(self._lib.elsi_set_refine_max_iter(self._h, int(it)), "set_refine_max_iter")

    def set_reuse_ovlp_factor(self, r: bool):
        self._check(self._lib.elsi_set_reuse_ovlp_factor(self._h, int(bool(r))), "set_reuse_ovlp_factor")

    def set_stream(self, stream):
        ptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        self._check(self._lib.elsi_set_stream(self._h, _vp(ptr)), "set_stream")

    def use_current_stream(self):
        import torch
        self.set_stream(torch.cuda.current_stream())

    # -- solves
    def ev_real(self, ham, ovlp=None):
        """Returns (eval (n,), evec (n, n_state)) as CUDA tensors."""
        import torch
        ev = torch.empty(self.n, dtype=torch.float64, device=ham.device)
        vec = torch.empty((self.n_state, self.n), dtype=torch.float64, device=ham.device)
        rc = self._lib.elsi_ev_real(self._h, _vp(_ptr(ham)), _vp(_ptr(ovlp) if ovlp is not None else None),
                                    _vp(_ptr(ev)), _vp(_ptr(vec)))
        self._check(rc, "elsi_ev_real")
        return ev, vec.t()

    def dm_real(self, ham, ovlp=None, out=None):
        """Returns (P (n, n), band energy) ; W is kept for get_edm()."""
        import torch
        p = out if out is not None else torch.empty((self.n, self.n), dtype=torch.float64, device=ham.device)
        e = ctypes.c_double(0.0)
        rc = self._lib.elsi_dm_real(self._h, _vp(_ptr(ham)), _vp(_ptr(ovlp) if ovlp is not None else None),
                                    _vp(_ptr(p)), ctypes.byref(e))
        self._check(rc, "elsi_dm_real")
        return p, e.value

    def ev_complex(self, ham, ovlp=None):
        """Complex Hermitian eigenpairs: (eval (n,) float64, evec (n, n_state) complex128)."""
        import torch
        c128 = torch.complex128
        hc = _colmajor(ham)
        sc = _colmajor(ovlp) if ovlp is not None else None
        ev = torch.empty(self.n, dtype=torch.float64, device=ham.device)
        vec = torch.empty((self.n_state, self.n), dtype=c128, device=ham.device)
        rc = self._lib.elsi_ev_complex(self._h, _vp(_ptr(hc, c128)),
                                       _vp(_ptr(sc, c128) if sc is not None else None),
                                       _vp(_ptr(ev)), _vp(_ptr(vec, c128)))
        self._check(rc, "elsi_ev_complex")
        return ev, vec.t()

    def dm_complex(self, ham, ovlp=None):
        """Complex density matrix P (n, n) complex128 and the band energy."""
        import torch
        c128 = torch.complex128
        hc = _colmajor(ham)
        sc = _colmajor(ovlp) if ovlp is not None else None
        p = torch.empty((self.n, self.n), dtype=c128, device=ham.device)
        e = ctypes.c_double(0.0)
        rc = self._lib.elsi_dm_complex(self._h, _vp(_ptr(hc, c128)),
                                       _vp(_ptr(sc, c128) if sc is not None else None),
                                       _vp(_ptr(p, c128)), ctypes.byref(e))
        self._check(rc, "elsi_dm_complex")
        return p.t(), e.value

    def get_edm_complex(self):
        import torch
        w = torch.empty((self.n, self.n), dtype=torch.complex128, device="cuda")
        self._check(self._lib.elsi_get_edm_complex(self._h, _vp(_ptr(w, torch.complex128))),
                    "elsi_get_edm_complex")
        return w.t()

    def get_edm(self, out=None):
        import torch
        w = out if out is not None else torch.empty((self.n, self.n), dtype=torch.float64, device="cuda")
        self._check(self._lib.elsi_get_edm_real(self._h, _vp(_ptr(w))), "elsi_get_edm_real")
        return w

    def get_mu(self) -> float:
        mu = ctypes.c_double(0.0)
        self._check(self._lib.elsi_get_mu(self._h, ctypes.byref(mu)), "elsi_get_mu")
        return mu.value

    def get_occ(self):
        import torch
        f = torch.empty(self.n_state, dtype=torch.float64, device="cuda")
        self._check(self._lib.elsi_get_occ(self._h, _vp(_ptr(f))), "elsi_get_occ")
        return f

    def get_eval(self):
        """The n_state eigenvalues occupied by the last dm_real call (device tensor)."""
        import torch
        w = torch.empty(self.n_state, dtype=torch.float64, device="cuda")
        self._check(self._lib.elsi_get_eval(self._h, _vp(_ptr(w))), "elsi_get_eval")
        return w

    def dm_real_host(self, ham, ovlp, den, edm=None) -> float:
        """Host-buffer entry point: numpy or pinned torch CPU float64 arrays (n, n)."""
        def hp(a):
            if a is None:
                return None
            if hasattr(a, "data_ptr"):
                return a.data_ptr()
            return a.ctypes.data
        e = ctypes.c_double(0.0)
        rc = self._lib.elsi_dm_real_host(self._h, _vp(hp(ham)), _vp(hp(ovlp)), _vp(hp(den)),
                                         _vp(hp(edm)), ctypes.byref(e))
        self._check(rc, "elsi_dm_real_host")
        return e.value

    # ---- sparse (CSC) input
    def set_csc(self, row_idx, col_ptr, index_base: int = 0):
        """CSC pattern of H and S: int32 tensors (CUDA or CPU) of nnz row indices and n + 1
        column starts."""
        import torch
        def ip(t):
            if t.dtype != torch.int32 or not t.is_contiguous():
                raise ValueError("expected a contiguous int32 tensor")
            return t.data_ptr()
        self._csc_nnz = int(row_idx.numel())
        rc = self._lib.elsi_set_csc(self._h, self._csc_nnz, _vp(ip(row_idx)), _vp(ip(col_ptr)),
                                    int(index_base))
        self._check(rc, "elsi_set_csc")

    def ev_real_sparse(self, hval, sval=None):
        import torch
        ev = torch.empty(self.n, dtype=torch.float64, device=hval.device)
        vec = torch.empty((self.n_state, self.n), dtype=torch.float64, device=hval.device)
        rc = self._lib.elsi_ev_real_sparse(self._h, _vp(_ptr(hval)),
                                           _vp(_ptr(sval) if sval is not None else None),
                                           _vp(_ptr(ev)), _vp(_ptr(vec)))
        self._check(rc, "elsi_ev_real_sparse")
        return ev, vec.t()

    def dm_real_sparse(self, hval, sval=None):
        """Returns (P at the pattern (nnz values), band energy)."""
        import torch
        p = torch.empty_like(hval)
        e = ctypes.c_double(0.0)
        rc = self._lib.elsi_dm_real_sparse(self._h, _vp(_ptr(hval)),
                                           _vp(_ptr(sval) if sval is not None else None),
                                           _vp(_ptr(p)), ctypes.byref(e))
        self._check(rc, "elsi_dm_real_sparse")
        return p, e.value

    def get_edm_sparse(self):
        import torch
        w = torch.empty(self._csc_nnz, dtype=torch.float64, device="cuda")
        self._check(self._lib.elsi_get_edm_real_sparse(self._h, _vp(_ptr(w))), "elsi_get_edm_real_sparse")
        return w

    def set_batch_streams(self, streams: int):
        """Concurrent solves in batched calls (0: chosen by the autotuner)."""
        self._check(self._lib.elsi_set_batch_streams(self._h, int(streams)), "elsi_set_batch_streams")

    def set_batch_autotune(self, on: bool):
        """Per-size tuning of band width, tridiagonalisation and concurrency (default on)."""
        self._check(self._lib.elsi_set_batch_autotune(self._h, 1 if on else 0), "elsi_set_batch_autotune")

    def batch_tuning(self, n: int, cplx: bool = False):
        """(band_width, elpa_solver, streams) chosen for problems of size n, or None."""
        b, s, w = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        rc = self._lib.elsi_get_batch_tuning(self._h, int(n), 1 if cplx else 0, ctypes.byref(b),
                                             ctypes.byref(s), ctypes.byref(w))
        if rc != 0:
            return None
        return b.value, s.value, w.value

    def set_elpa_solver(self, solver: int):
        """1: one-stage tridiagonalisation, 2: two-stage (default)."""
        self._check(self._lib.elsi_set_elpa_solver(self._h, int(solver)), "elsi_set_elpa_solver")

    def set_sing_check(self, mode: int, tol: float | None = None):
        """Singularity check of S (0 off, 1 check, 2 always transform) and its tolerance."""
        self._check(self._lib.elsi_set_sing_check(self._h, int(mode)), "elsi_set_sing_check")
        if tol is not None:
            self._check(self._lib.elsi_set_sing_tol(self._h, float(tol)), "elsi_set_sing_tol")

    def get_n_nonsing(self) -> int:
        v = ctypes.c_int(0)
        self._check(self._lib.elsi_get_n_nonsing(self._h, ctypes.byref(v)), "elsi_get_n_nonsing")
        return v.value

    def get_entropy(self) -> float:
        """-kT S_ent of the last density-matrix solve (F = E_band + this)."""
        ts = ctypes.c_double(0.0)
        self._check(self._lib.elsi_get_entropy(self._h, ctypes.byref(ts)), "elsi_get_entropy")
        return ts.value

    def dm_adjoint(self, f_bar: float, P, W):
        """(dL/dH, dL/dS) = (f_bar P, -f_bar W) for dL/dF = f_bar."""
        import torch
        n = P.shape[0]
        hb = torch.empty_like(P)
        sb = torch.empty_like(P)
        rc = self._lib.elsi_dm_adjoint_real(self._h, n, float(f_bar), _vp(_ptr(P)), _vp(_ptr(W)),
                                            _vp(_ptr(hb)), _vp(_ptr(sb)))
        self._check(rc, "elsi_dm_adjoint_real")
        return hb, sb

    def ev_adjoint(self, ev, C, ev_bar=None, C_bar=None):
        """(dL/dH, dL/dS) for dL/d ev = ev_bar (n) and dL/dC[:, :k] = C_bar (n, k); C holds
        all n eigenvectors as columns (n, n)."""
        import torch
        n = ev.shape[0]
        ct = C.t().contiguous()  # column-major storage of C
        gb = C_bar.t().contiguous() if C_bar is not None else None
        k = 0 if C_bar is None else C_bar.shape[1]
        hb = torch.empty((n, n), dtype=torch.float64, device=ev.device)
        sb = torch.empty((n, n), dtype=torch.float64, device=ev.device)
        eb = ev_bar.contiguous() if ev_bar is not None else None
        rc = self._lib.elsi_ev_adjoint_real(self._h, n, k, _vp(_ptr(ev)), _vp(_ptr(ct)),
                                            _vp(_ptr(eb) if eb is not None else None),
                                            _vp(_ptr(gb) if gb is not None else None),
                                            _vp(_ptr(hb)), _vp(_ptr(sb)))
        self._check(rc, "elsi_ev_adjoint_real")
        return hb, sb

    # ---- several problems (k-points / spin channels) ----
    def _batch_inputs(self, hams, ovlps, n_states, inputs_colmajor=False):
        import torch
        cplx = hams[0].is_complex()
        dt = torch.complex128 if cplx else torch.float64
        prep = (lambda t: _colmajor(t)) if (cplx and not inputs_colmajor) else (lambda t: t)
        hs = [prep(t) for t in hams]
        ss = None if ovlps is None else [prep(t) for t in ovlps]
        nprob = len(hs)
        nb = (ctypes.c_int * nprob)(*[int(t.shape[0]) for t in hs])
        ks = (ctypes.c_int * nprob)(*[int(k) for k in n_states])
        hp = (_vp * nprob)(*[_ptr(t, dt) for t in hs])
        sp = None if ss is None else (_vp * nprob)(*[_ptr(t, dt) for t in ss])
        self._batch = dict(n=[int(t.shape[0]) for t in hs], k=[int(k) for k in n_states],
                           cplx=cplx, device=hs[0].device)
        return cplx, dt, hs, ss, nb, ks, hp, sp

    def _batch_outputs(self, want_edm):
        import torch
        b = getattr(self, "_batch", None)
        if b is None:  # no batched eigensolve yet: the library reports ELSI_ERR_STATE
            b = dict(n=[], k=[], cplx=False, device="cuda")
        dt = torch.complex128 if b["cplx"] else torch.float64
        ps = [torch.empty((n, n), dtype=dt, device=b["device"]) for n in b["n"]]
        ws = [torch.empty((n, n), dtype=dt, device=b["device"]) for n in b["n"]] if want_edm else None
        nprob = len(ps)
        pp = (_vp * max(nprob, 1))(*[_ptr(t, dt) for t in ps])
        wp = (_vp * max(nprob, 1))(*[_ptr(t, dt) for t in ws]) if want_edm else None
        fix = (lambda t: t.t()) if b["cplx"] else (lambda t: t)
        return ps, ws, pp, wp, fix

    def dm_batched(self, hams, ovlps, n_states, n_electron, *, weights=None,
                   shared_mu: bool = True, want_edm: bool = True, inputs_colmajor: bool = False):
        """Density matrices of several problems (real float64 or complex128 CUDA tensors).
        shared_mu: one chemical potential, sum_i weights[i] sum_l f_il = n_electron;
        else n_electron is a list, one per problem. inputs_colmajor: complex inputs are
        already column-major (no copy). Returns (P list, W list or None, band energies,
        mu (float, or list))."""
        cplx, dt, hs, ss, nb, ks, hp, sp = self._batch_inputs(hams, ovlps, n_states, inputs_colmajor)
        nprob = len(hs)
        ps, ws, pp, wp, fix = self._batch_outputs(want_edm)
        wts = None if weights is None else (ctypes.c_double * nprob)(*[float(w) for w in weights])
        nel = [float(n_electron)] if shared_mu else [float(x) for x in n_electron]
        nel_a = (ctypes.c_double * len(nel))(*nel)
        en = (ctypes.c_double * nprob)()
        mu = (ctypes.c_double * nprob)()
        fn = self._lib.elsi_dm_batched_complex if cplx else self._lib.elsi_dm_batched_real
        rc = fn(self._h, nprob, nb, ks, hp, sp, wts, nel_a, int(bool(shared_mu)), pp, wp, en, mu)
        self._check(rc, fn.__name__)
        mus = mu[0] if shared_mu else list(mu)
        return ([fix(p) for p in ps], [fix(w) for w in ws] if want_edm else None, list(en), mus)

    def batch_ev(self, hams, ovlps, n_states):
        """Phase 1: eigenpairs of every problem, kept in the handle. Returns the
        n_states[i] lowest eigenvalues of each problem, concatenated (CUDA tensor)."""
        import torch
        cplx, dt, hs, ss, nb, ks, hp, sp = self._batch_inputs(hams, ovlps, n_states)
        ev = torch.empty(sum(self._batch["k"]), dtype=torch.float64, device=hs[0].device)
        fn = self._lib.elsi_batch_ev_complex if cplx else self._lib.elsi_batch_ev_real
        self._check(fn(self._h, len(hs), nb, ks, hp, sp, _vp(_ptr(ev))), fn.__name__)
        return ev

    def occupation_weighted(self, eps, wts, n_electron: float):
        """Phase 2: occupations (CUDA tensor) and one chemical potential over weighted
        eigenvalues (CUDA float64 tensors of equal length)."""
        import torch
        f = torch.empty_like(eps)
        mu = ctypes.c_double(0.0)
        rc = self._lib.elsi_occupation_weighted(self._h, int(eps.numel()), _vp(_ptr(eps)),
                                                _vp(_ptr(wts)), float(n_electron), _vp(_ptr(f)),
                                                ctypes.byref(mu))
        self._check(rc, "elsi_occupation_weighted")
        return f, mu.value

    def batch_dm(self, occ, want_edm: bool = True):
        """Phase 3: (P list, W list or None, band energies) of the last batch_ev."""
        ps, ws, pp, wp, fix = self._batch_outputs(want_edm)
        en = (ctypes.c_double * len(ps))()
        self._check(self._lib.elsi_batch_dm(self._h, _vp(_ptr(occ)), pp, wp, en), "elsi_batch_dm")
        return [fix(p) for p in ps], [fix(w) for w in ws] if want_edm else None, list(en)

    def stage_times(self) -> dict:
        buf = (ctypes.c_float * 32)()
        m = self._lib.elsi_get_stage_times(self._h, buf, 32)
        return {self._lib.elsi_stage_name(i).decode(): float(buf[i]) for i in range(max(m, 0))}

    def refine_info(self):
        it, err = ctypes.c_int(0), ctypes.c_double(0.0)
        self._lib.elsi_get_refine_info(self._h, ctypes.byref(it), ctypes.byref(err))
        return it.value, err.value


def solve_dm(ham, ovlp, n_state: int, n_electron: float, **opts):
    """One-shot density-matrix solve. Returns dict(P, W, energy, mu)."""
    with Handle(ham.shape[0], n_state, n_electron) as h:
        _apply_opts(h, opts)
        p, e = h.dm_real(ham, ovlp)
        return dict(P=p, W=h.get_edm(), energy=e, mu=h.get_mu(), stages=h.stage_times())


def solve_ev(ham, ovlp, n_state: int, **opts):
    with Handle(ham.shape[0], n_state, 0.0) as h:
        _apply_opts(h, opts)
        ev, vec = h.ev_real(ham, ovlp)
        return dict(eval=ev, C=vec, stages=h.stage_times())


def _apply_opts(h: Handle, opts: dict):
    if opts.get("overlap_is_unit"):
        h.set_overlap_is_unit(True)
    if "band_width" in opts:
        h.set_band_width(opts["band_width"])
    if "precision" in opts:
        h.set_precision(opts["precision"])
    if "scheme" in opts:
        h.set_broadening(opts["scheme"], opts.get("kt"))
    if "occ_accuracy" in opts:
        h.set_occ_accuracy(opts["occ_accuracy"])
    if "mu_max_steps" in opts:
        h.set_mu_max_steps(opts["mu_max_steps"])
    if "refine_max_iter" in opts:
        h.set_refine_max_iter(opts["refine_max_iter"])
    if opts.get("use_current_stream", True):
        h.use_current_stream()
