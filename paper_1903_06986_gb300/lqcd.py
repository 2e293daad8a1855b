"""Thin ctypes binding of liblqcd (include/lqcd.h): argument marshalling only.

Every computation happens in the CUDA library; this module converts torch tensors (complex128,
contiguous, on the context's device) to raw pointers and host arrays to ctypes buffers.  There is
no fallback: if the library is missing or a call fails, an exception is raised.

Shapes: gauge links (4, T, Z, Y, X, 3, 3); a block of fields (nrhs, T, Z, Y, X, 4, 3), or one
field (T, Z, Y, X, 4, 3).  Lattice dims are given as (Lx, Ly, Lz, Lt).
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

OK, ERR_INVALID_ARG, ERR_NONFINITE, ERR_NOT_CONVERGED, ERR_TIMEOUT, ERR_CUDA, ERR_OOM = range(7)
PREC_F64, PREC_F32, PREC_F16, PREC_BF16 = 0, 1, 2, 3
APPLY_M, APPLY_G5R, APPLY_DAG, APPLY_HOP = 0, 1, 2, 3
SYS_M, SYS_MG5 = 0, 1
SUB_NONE, SUB_PERT, SUB_POLY, SUB_DEFL, SUB_DEFL_PERT, SUB_DEFL_POLY, SUB_ES = (1 << i for i in range(7))
SUB_ALL = 127
MODES = ["none", "pert", "poly", "defl", "defl_pert", "defl_poly", "es"]
NMODES = len(MODES)
NOPS = 9
KERNEL_CLASSES = ["wilson", "dot", "axpy", "combine", "norm", "contract", "blas1", "noise", "probe", "tensor", "slice"]
DEFL_FP64, DEFL_TENSOR = 0, 1


class LqcdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("lqcd status %d: %s" % (status, msg))
        self.status = status


class KrylovOpts(C.Structure):
    _fields_ = [("m", C.c_int), ("k", C.c_int), ("tol", C.c_double), ("max_cycles", C.c_int),
                ("system", C.c_int), ("prec", C.c_int), ("inner_tol", C.c_double), ("eig_tol", C.c_double),
                ("poly_degree", C.c_int), ("poly_coeffs", C.c_void_p)]


class SolveInfo(C.Structure):
    _fields_ = [("cycles", C.c_int), ("matvecs", C.c_long), ("converged", C.c_int),
                ("true_resid", C.c_double), ("seconds", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class EstOpts(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("nnoise", C.c_int), ("block", C.c_int), ("m", C.c_int), ("k", C.c_int),
                ("m_inner", C.c_int), ("K", C.c_int), ("npoly", C.c_int), ("tol", C.c_double),
                ("tol_special", C.c_double), ("max_cycles", C.c_int), ("modes", C.c_int), ("prec", C.c_int),
                ("inner_tol", C.c_double), ("eig_tol", C.c_double), ("system", C.c_int), ("prec_degree", C.c_int),
                ("evenodd", C.c_int)]


_dp = C.POINTER(C.c_double)


class Estimate(C.Structure):
    _fields_ = [("per_noise", _dp), ("per_t", _dp), ("addback", _dp), ("mean", _dp), ("stderr_", _dp),
                ("lam", _dp), ("poly_a", _dp), ("matvecs_setup", C.c_long), ("matvecs_noise", C.c_long),
                ("seconds_setup", C.c_double), ("seconds_noise", C.c_double), ("max_true_resid", C.c_double),
                ("converged", C.c_int), ("block", C.c_int)]


class LoopInfo(C.Structure):
    _fields_ = [("addback", _dp), ("lam", _dp), ("poly_a", _dp), ("xi_pert", _dp), ("xi_poly", _dp),
                ("Q", C.c_int), ("block", C.c_int), ("matvecs_setup", C.c_long), ("seconds_setup", C.c_double),
                ("eig_resid_max", C.c_double)]


class NoiseInfo(C.Structure):
    _fields_ = [("matvecs", C.c_long), ("seconds", C.c_double), ("max_true_resid", C.c_double),
                ("converged", C.c_int), ("block", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Derivs(C.Structure):
    _fields_ = [("grad_scale", C.c_double), ("dkappa", _dp), ("dkappa_err", _dp), ("per_noise", _dp),
                ("link_grad", C.c_void_p), ("grad_links", C.c_void_p), ("matvecs", C.c_long), ("seconds", C.c_double),
                ("max_true_resid", C.c_double), ("converged", C.c_int)]


_LIB = None


def library_path():
    return _build.LIB


def load(path=None):
    """Load liblqcd.so (built by paper_1903_06986_gb300.build); raises if it is missing."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or library_path()
    if not os.path.exists(path):
        raise RuntimeError("liblqcd.so not found at %s: run `python -m paper_1903_06986_gb300.build`" % path)
    lib = C.CDLL(path)
    vp, i, d, u64, u32 = C.c_void_p, C.c_int, C.c_double, C.c_uint64, C.c_uint32
    sig = {
        "lqcd_ctx_create": [C.POINTER(vp), C.POINTER(C.c_int), i, vp],
        "lqcd_ctx_destroy": [vp],
        "lqcd_set_stream": [vp, vp],
        "lqcd_noise_z4": [vp, u64, u32, i, vp],
        "lqcd_wilson_apply": [vp, vp, d, vp, vp, i, i, i],
        "lqcd_wilson_apply_f32": [vp, vp, d, vp, vp, i, i],
        "lqcd_to_f32": [vp, vp, vp, C.c_longlong],
        "lqcd_pack_f32": [vp, vp, vp, i],
        "lqcd_unpack_f32": [vp, vp, vp, i],
        "lqcd_pack_links_f32": [vp, vp, vp, i],
        "lqcd_wilson_apply_packed": [vp, vp, i, d, vp, vp, i, i, i],
        "lqcd_pack_half": [vp, i, vp, vp, i],
        "lqcd_unpack_half": [vp, i, vp, vp, i],
        "lqcd_wilson_apply_half": [vp, i, vp, i, d, vp, vp, i, i],
        "lqcd_gmresdr_solve": [vp, vp, d, vp, vp, i, C.POINTER(KrylovOpts), C.POINTER(SolveInfo), C.POINTER(vp)],
        "lqcd_minresdr_solve": [vp, vp, d, vp, vp, i, C.POINTER(KrylovOpts), C.POINTER(SolveInfo), C.POINTER(vp)],
        "lqcd_proj_solve": [vp, vp, d, vp, vp, vp, i, C.POINTER(KrylovOpts), C.POINTER(SolveInfo)],
        "lqcd_defl_destroy": [vp],
        "lqcd_defl_info": [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)],
        "lqcd_defl_export": [vp, vp, vp, vp, vp, vp],
        "lqcd_defl_import": [vp, i, vp, vp, C.POINTER(vp)],
        "lqcd_defl_import_space": [vp, i, vp, vp, i, C.POINTER(vp)],
        "lqcd_loop_setup": [vp, vp, d, C.POINTER(EstOpts), C.POINTER(vp)],
        "lqcd_loop_setup_from": [vp, vp, d, C.POINTER(EstOpts), vp, vp, vp, C.POINTER(vp)],
        "lqcd_loop_noises": [vp, vp, u32, i, vp, C.POINTER(NoiseInfo)],
        "lqcd_loop_get": [vp, C.POINTER(LoopInfo)],
        "lqcd_loop_set_noise_opts": [vp, i, d, i],
        "lqcd_loop_set_inner_restart": [vp, i],
        "lqcd_loop_noises_host": [vp, vp, u32, i, vp, C.POINTER(NoiseInfo)],
        "lqcd_loop_destroy": [vp],
        "lqcd_deflate_project": [vp, vp, vp, vp, i, vp],
        "lqcd_set_defl_engine": [vp, i],
        "lqcd_set_wait_limit": [vp, d],
        "lqcd_inject_tc_stall": [vp, i],
        "lqcd_tc_vdag_x": [vp, vp, i, vp, i, vp],
        "lqcd_tc_v_c": [vp, vp, i, vp, i, vp],
        "lqcd_tc_slice_bytes": [C.POINTER(C.c_int), i, C.POINTER(C.c_size_t)],
        "lqcd_hop_series": [vp, vp, d, vp, vp, i, i, vp],
        "lqcd_poly_apply": [vp, vp, d, vp, vp, i, i, vp],
        "lqcd_poly_coeffs": [vp, vp, d, u64, i, vp],
        "lqcd_hop_traces": [vp, vp, d, i, vp],
        "lqcd_xi_inverse": [vp, vp, d, vp, i, i, vp, vp],
        "lqcd_contract": [vp, vp, d, vp, vp, i, vp],
        "lqcd_loop_estimate": [vp, vp, d, C.POINTER(EstOpts), C.POINTER(Estimate)],
        "lqcd_link_grad": [vp, vp, d, vp, vp, i, d, vp, vp],
        "lqcd_loop_derivs": [vp, vp, d, C.POINTER(EstOpts), C.POINTER(Derivs)],
        "lqcd_set_graphs": [vp, i],
        "lqcd_set_rhs_per_thread": [vp, i],
        "lqcd_set_inner_gs_passes": [vp, i],
        "lqcd_set_probe_depth": [vp, i],
        "lqcd_set_inner_window": [vp, i],
        "lqcd_ctx_create_evenodd": [C.POINTER(vp), C.POINTER(C.c_int), i, vp],
        "lqcd_eo_split": [vp, vp, vp, vp, i],
        "lqcd_eo_join": [vp, vp, vp, vp, i],
        "lqcd_eo_hop": [vp, vp, vp, vp, i, i],
        "lqcd_eo_rhs": [vp, vp, d, vp, vp, i],
        "lqcd_eo_reconstruct": [vp, vp, d, vp, vp, vp, i],
        "lqcd_eo_full_eigenpairs": [vp, vp, d, vp, vp, i, d, vp, vp],
        "lqcd_probe_classes": [C.POINTER(C.c_int), i, C.POINTER(C.c_int), vp],
        "lqcd_probe_depth": [C.POINTER(C.c_int), i, i, C.POINTER(C.c_int)],
        "lqcd_autotune_block": [vp, vp, d, vp, C.POINTER(KrylovOpts), C.POINTER(C.c_int), i, C.POINTER(C.c_int),
                                C.POINTER(C.c_double)],
        "lqcd_batch_loop_estimate": [i, C.POINTER(vp), C.POINTER(vp), C.POINTER(d), C.POINTER(EstOpts),
                                     C.POINTER(Estimate), C.POINTER(C.c_int)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.lqcd_last_error_string.argtypes = [vp]
    lib.lqcd_last_error_string.restype = C.c_char_p
    lib.lqcd_version.argtypes = []
    lib.lqcd_version.restype = C.c_char_p
    lib.lqcd_kernel_launches.argtypes = [vp]
    lib.lqcd_kernel_launches.restype = C.c_long
    lib.lqcd_timing_enable.argtypes = [vp, i]
    lib.lqcd_timing_enable.restype = C.c_int
    lib.lqcd_timing_reset.argtypes = [vp]
    lib.lqcd_timing_reset.restype = C.c_int
    lib.lqcd_timing_read.argtypes = [vp, i, C.POINTER(C.c_double), C.POINTER(C.c_long), C.POINTER(C.c_double)]
    lib.lqcd_timing_read.restype = C.c_int
    lib.lqcd_timing_bytes.argtypes = [vp, i, C.POINTER(C.c_double)]
    lib.lqcd_timing_bytes.restype = C.c_int
    _LIB = lib
    return lib


def _torch():
    import torch
    return torch


def _ptr(t, dtype=None):
    if t is None:
        return None
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    want = torch.complex128 if dtype is None else dtype
    if not t.is_cuda or t.dtype != want or not t.is_contiguous():
        raise ValueError("tensors must be contiguous %s CUDA tensors" % want)
    return C.c_void_p(t.data_ptr())


def _host_c(arr):
    a = np.ascontiguousarray(np.asarray(arr, dtype=np.complex128))
    return a, a.ctypes.data_as(C.c_void_p)


def _set_poly(o, poly):
    """Fill the polynomial-preconditioner fields of KrylovOpts o; returns the buffer to keep alive."""
    if poly is None:
        return None
    a, ap = _host_c(poly)
    o.poly_degree = len(a) - 1
    o.poly_coeffs = ap
    return a


class Defl:
    """A deflation space made by a solver (V_{k+1}, Hbar_k, Ritz pairs) or imported eigenpairs."""

    def __init__(self, ctx, handle):
        self.ctx = ctx
        self.h = handle

    @property
    def k(self):
        k, herm = C.c_int(), C.c_int()
        self.ctx._check(self.ctx.lib.lqcd_defl_info(self.h, C.byref(k), C.byref(herm)))
        return k.value

    def export(self, basis=True, eigvecs=True):
        torch = _torch()
        k = self.k
        N = self.ctx.N
        V = torch.empty((k + 1, N), dtype=torch.complex128, device=self.ctx.device) if basis else None
        E = torch.empty((k, N), dtype=torch.complex128, device=self.ctx.device) if eigvecs else None
        H = np.zeros((k + 1, k), dtype=np.complex128) if basis else None
        lam = np.zeros(k, dtype=np.complex128)
        eres = np.zeros(k, dtype=np.float64)
        self.ctx._check(self.ctx.lib.lqcd_defl_export(
            self.h, _ptr(V), H.ctypes.data_as(C.c_void_p) if H is not None else None,
            lam.ctypes.data_as(C.c_void_p), _ptr(E), eres.ctypes.data_as(C.c_void_p)))
        return dict(V=V, Hbar=H, lam=lam, E=E, eig_resid=eres)

    def close(self):
        if self.h:
            self.ctx.lib.lqcd_defl_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Loop:
    """The per-configuration setup of a loop estimate (lqcd_loop): noises can then be run in batches."""

    def __init__(self, ctx, handle, opts, keep=()):
        self.ctx = ctx
        self.h = handle
        self.opts = opts
        self._keep = keep          # deflation objects the setup borrows

    def noises(self, links, first, count):
        """Noise terms [6 modes][count][9 ops][Lt] (complex) of noises first .. first+count-1, and the
        lqcd_noise_info as a dict (with the call's status)."""
        out = np.zeros((NMODES, count, NOPS, self.ctx.dims[3]), dtype=np.complex128)
        info = NoiseInfo()
        st = self.ctx.lib.lqcd_loop_noises(self.h, _ptr(links), first, count, out.ctypes.data_as(C.c_void_p),
                                           C.byref(info))
        if st not in (OK, ERR_NOT_CONVERGED):
            self.ctx._check(st)
        d = info.as_dict()
        d["status"] = st
        return out, d

    def set_noise_opts(self, prec, inner_tol=0.0, block=0):
        """Precision (and block width, 0 = unchanged) of the noise solves from now on."""
        self.ctx._check(self.ctx.lib.lqcd_loop_set_noise_opts(self.h, prec, inner_tol, block))

    def noises_host(self, links_host, first, count):
        """lqcd_loop_noises_host: as noises(), with the gauge field in host memory (a CPU tensor or a
        numpy array, copied to the device by the call)."""
        out = np.zeros((NMODES, count, NOPS, self.ctx.dims[3]), dtype=np.complex128)
        info = NoiseInfo()
        nlink = 4 * int(np.prod(self.ctx.dims)) * 9
        if isinstance(links_host, np.ndarray):
            if links_host.dtype != np.complex128 or not links_host.flags.c_contiguous or links_host.size != nlink:
                raise ValueError("host links: contiguous complex128, 4 x V x 3 x 3")
            ptr = links_host.ctypes.data_as(C.c_void_p)
        else:
            torch = _torch()
            if (links_host.is_cuda or links_host.dtype != torch.complex128 or not links_host.is_contiguous()
                    or links_host.numel() != nlink):
                raise ValueError("host links: contiguous complex128 CPU tensor, 4 x V x 3 x 3")
            ptr = C.c_void_p(links_host.data_ptr())
        st = self.ctx.lib.lqcd_loop_noises_host(self.h, ptr, first, count, out.ctypes.data_as(C.c_void_p),
                                                C.byref(info))
        if st not in (OK, ERR_NOT_CONVERGED):
            self.ctx._check(st)
        d = info.as_dict()
        d["status"] = st
        return out, d

    def set_inner_restart(self, m_inner):
        """GMRES-Proj cycle length of the noise solves from now on (0 = m - k)."""
        self.ctx._check(self.ctx.lib.lqcd_loop_set_inner_restart(self.h, m_inner))

    def info(self):
        lt = self.ctx.dims[3]
        q = self.opts.k
        bufs = dict(addback=np.zeros((NMODES, NOPS, lt), dtype=np.complex128), lam=np.zeros(4096, dtype=np.complex128),
                    poly_a=np.zeros(self.opts.npoly + 1, dtype=np.complex128),
                    xi_pert=np.zeros(4096, dtype=np.complex128), xi_poly=np.zeros(4096, dtype=np.complex128))
        as_dp = lambda a: a.ctypes.data_as(_dp)
        li = LoopInfo(*[as_dp(bufs[n]) for n in ("addback", "lam", "poly_a", "xi_pert", "xi_poly")], 0, 0, 0, 0.0, 0.0)
        self.ctx._check(self.ctx.lib.lqcd_loop_get(self.h, C.byref(li)))
        q = li.Q
        for n in ("lam", "xi_pert", "xi_poly"):
            bufs[n] = bufs[n][:q].copy()
        bufs.update(Q=q, block=li.block, matvecs_setup=li.matvecs_setup, seconds_setup=li.seconds_setup,
                    eig_resid_max=li.eig_resid_max)
        return bufs

    def close(self):
        if self.h:
            self.ctx.lib.lqcd_loop_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """An lqcd_ctx bound to the current CUDA device and torch's current stream."""

    def __init__(self, dims, stream=None, recon=18):
        torch = _torch()
        self.lib = load()
        self.dims = tuple(int(d) for d in dims)
        self.V = int(np.prod(self.dims))
        self.N = 12 * self.V
        self.device = torch.device("cuda", torch.cuda.current_device())
        s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        h = C.c_void_p()
        dd = (C.c_int * 4)(*self.dims)
        st = self.lib.lqcd_ctx_create(C.byref(h), dd, recon, C.c_void_p(s))
        if st != OK:
            raise LqcdError(st, "lqcd_ctx_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.lqcd_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != OK:
            raise LqcdError(st, self.lib.lqcd_last_error_string(self.h).decode())
        return st

    @property
    def launches(self):
        return self.lib.lqcd_kernel_launches(self.h)

    def timing(self, enable):
        """Bracket every kernel launch with CUDA events (diagnostics)."""
        self._check(self.lib.lqcd_timing_enable(self.h, 1 if enable else 0))

    def timing_reset(self):
        self._check(self.lib.lqcd_timing_reset(self.h))

    def timing_read(self):
        """{class: (total device ms, launches, work units)} since the last reset."""
        out = {}
        for i, name in enumerate(KERNEL_CLASSES):
            ms, n, u = C.c_double(), C.c_long(), C.c_double()
            self._check(self.lib.lqcd_timing_read(self.h, i, C.byref(ms), C.byref(n), C.byref(u)))
            out[name] = (ms.value, n.value, u.value)
        return out

    def timing_bytes(self):
        """{class: compulsory device-memory bytes of the timed launches} since the last reset."""
        out = {}
        for i, name in enumerate(KERNEL_CLASSES):
            v = C.c_double()
            self._check(self.lib.lqcd_timing_bytes(self.h, i, C.byref(v)))
            out[name] = v.value
        return out

    def set_stream(self, stream):
        self._check(self.lib.lqcd_set_stream(self.h, C.c_void_p(stream)))

    def field(self, nrhs=None):
        torch = _torch()
        lx, ly, lz, lt = self.dims
        shp = (lt, lz, ly, lx, 4, 3) if nrhs is None else (nrhs, lt, lz, ly, lx, 4, 3)
        return torch.empty(shp, dtype=torch.complex128, device=self.device)

    def _nrhs(self, t):
        n = t.numel() // self.N
        if n * self.N != t.numel():
            raise ValueError("field size %d is not a multiple of 12 V = %d" % (t.numel(), self.N))
        return n

    # Z(4) noise
    def noise_z4(self, seed, first, nrhs, out=None):
        out = self.field(nrhs) if out is None else out
        self._check(self.lib.lqcd_noise_z4(self.h, seed, first, nrhs, _ptr(out)))
        return out

    # Wilson operator
    def wilson_apply(self, links, kappa, inp, out=None, flags=APPLY_M, prec=PREC_F64):
        out = _torch().empty_like(inp) if out is None else out
        self._check(self.lib.lqcd_wilson_apply(self.h, _ptr(links), kappa, _ptr(inp), _ptr(out),
                                               self._nrhs(inp), prec, flags))
        return out

    def to_f32(self, t):
        """complex128 device tensor -> complex64 copy (FP32 storage), converted on the device."""
        out = _torch().empty(t.shape, dtype=_torch().complex64, device=self.device)
        self._check(self.lib.lqcd_to_f32(self.h, _ptr(t), _ptr(out, _torch().complex64), t.numel()))
        return out

    def pack_f32(self, x):
        """canonical complex128 block (nrhs fields) -> packed FP32 (float32 tensor, nrhs x 24 V)."""
        n = self._nrhs(x)
        out = _torch().empty((n, 24 * self.V), dtype=_torch().float32, device=self.device)
        self._check(self.lib.lqcd_pack_f32(self.h, _ptr(x), _ptr(out, _torch().float32), n))
        return out

    def unpack_f32(self, p):
        n = p.numel() // (24 * self.V)
        out = self.field(n)
        self._check(self.lib.lqcd_unpack_f32(self.h, _ptr(p, _torch().float32), _ptr(out), n))
        return out

    def pack_links_f32(self, links, recon=12):
        nc = 12 if recon == 12 else 20
        out = _torch().empty((4, nc * self.V), dtype=_torch().float32, device=self.device)
        self._check(self.lib.lqcd_pack_links_f32(self.h, _ptr(links), _ptr(out, _torch().float32), recon))
        return out

    def wilson_apply_packed(self, links_p, recon, kappa, inp, out=None, flags=APPLY_M, rhs_per_thread=0):
        f32 = _torch().float32
        out = _torch().empty_like(inp) if out is None else out
        self._check(self.lib.lqcd_wilson_apply_packed(self.h, _ptr(links_p, f32), recon, kappa, _ptr(inp, f32),
                                                      _ptr(out, f32), inp.numel() // (24 * self.V), flags,
                                                      rhs_per_thread))
        return out

    def pack_half(self, x, prec=PREC_F16):
        """canonical complex128 block -> packed FP16 / BF16 (int16 tensor of raw halves, nrhs x 24 V),
        stored scaled by 2^floor(log2(sqrt(12 V)))."""
        n = self._nrhs(x)
        out = _torch().empty((n, 24 * self.V), dtype=_torch().int16, device=self.device)
        self._check(self.lib.lqcd_pack_half(self.h, prec, _ptr(x), _ptr(out, _torch().int16), n))
        return out

    def unpack_half(self, p, prec=PREC_F16):
        n = p.numel() // (24 * self.V)
        out = self.field(n)
        self._check(self.lib.lqcd_unpack_half(self.h, prec, _ptr(p, _torch().int16), _ptr(out), n))
        return out

    def wilson_apply_half(self, links_p, recon, kappa, inp, out=None, flags=APPLY_M, prec=PREC_F16):
        i16 = _torch().int16
        out = _torch().empty_like(inp) if out is None else out
        self._check(self.lib.lqcd_wilson_apply_half(self.h, prec, _ptr(links_p, _torch().float32), recon, kappa,
                                                    _ptr(inp, i16), _ptr(out, i16), inp.numel() // (24 * self.V),
                                                    flags))
        return out

    def wilson_apply_f32(self, links32, kappa, inp, out=None, flags=APPLY_M):
        c64 = _torch().complex64
        out = _torch().empty_like(inp) if out is None else out
        self._check(self.lib.lqcd_wilson_apply_f32(self.h, _ptr(links32, c64), kappa, _ptr(inp, c64),
                                                   _ptr(out, c64), inp.numel() // self.N, flags))
        return out

    # GMRES-DR / MINRES-DR
    def _krylov(self, fn, links, kappa, b, m, k, tol, max_cycles, system, want_defl, prec, eig_tol=0.0, poly=None):
        x = _torch().empty_like(b)
        o = KrylovOpts(m, k, tol, max_cycles, system, prec, 0.0, eig_tol)
        keep = _set_poly(o, poly)
        info = SolveInfo()
        dh = C.c_void_p()
        st = fn(self.h, _ptr(links), kappa, _ptr(b), _ptr(x), self._nrhs(b), C.byref(o), C.byref(info),
                C.byref(dh) if want_defl else None)
        if st not in (OK, ERR_NOT_CONVERGED):
            self._check(st)
        defl = Defl(self, dh) if (want_defl and dh.value) else None
        return x, info.as_dict(), defl

    def gmresdr_solve(self, links, kappa, b, m, k, tol, max_cycles=1000, system=SYS_M, want_defl=False,
                      prec=PREC_F64, eig_tol=0.0, poly=None):
        """poly: coefficients a_0..a_d of a polynomial right preconditioner p (Krylov on A p(A))."""
        return self._krylov(self.lib.lqcd_gmresdr_solve, links, kappa, b, m, k, tol, max_cycles, system,
                            want_defl, prec, eig_tol, poly)

    def minresdr_solve(self, links, kappa, b, m, k, tol, max_cycles=1000, want_defl=False, prec=PREC_F64,
                       eig_tol=0.0, poly=None):
        return self._krylov(self.lib.lqcd_minresdr_solve, links, kappa, b, m, k, tol, max_cycles, SYS_MG5,
                            want_defl, prec, eig_tol, poly)

    # deflated multi-RHS solves
    def proj_solve(self, links, kappa, defl, b, m, tol, max_cycles=1000, system=SYS_M, prec=PREC_F64,
                   inner_tol=0.0, poly=None):
        x = _torch().empty_like(b)
        o = KrylovOpts(m, 0, tol, max_cycles, system, prec, inner_tol)
        keep = _set_poly(o, poly)
        info = SolveInfo()
        st = self.lib.lqcd_proj_solve(self.h, _ptr(links), kappa, defl.h, _ptr(b), _ptr(x), self._nrhs(b),
                                      C.byref(o), C.byref(info))
        if st not in (OK, ERR_NOT_CONVERGED):
            self._check(st)
        return x, info.as_dict()

    def defl_import(self, E, lam):
        lamh, lp = _host_c(lam)
        dh = C.c_void_p()
        self._check(self.lib.lqcd_defl_import(self.h, len(lamh), _ptr(E), lp, C.byref(dh)))
        return Defl(self, dh)

    def defl_import_space(self, V, Hbar, hermitian=False):
        """Deflation space from a (k+1)-vector basis V (device) and its (k+1) x k Hbar (host)."""
        k = Hbar.shape[1]
        H = np.ascontiguousarray(Hbar, dtype=np.complex128)
        dh = C.c_void_p()
        self._check(self.lib.lqcd_defl_import_space(self.h, k, _ptr(V), H.ctypes.data_as(C.c_void_p),
                                                    1 if hermitian else 0, C.byref(dh)))
        return Defl(self, dh)

    # loop estimate in two phases
    @staticmethod
    def _est_opts(seed, nnoise, block, m, k, K, npoly, tol, tol_special, m_inner=0, max_cycles=2000, modes=SUB_ALL,
                  prec=PREC_F64, inner_tol=0.0, eig_tol=0.0, system=SYS_M, prec_degree=0, evenodd=0):
        return EstOpts(seed, nnoise, block, m, k, m_inner, K, npoly, tol, tol_special, max_cycles, modes, prec,
                       inner_tol, eig_tol, system, prec_degree, evenodd)

    def loop_setup(self, links, kappa, seed, nnoise, block, m, k, K, npoly, tol, tol_special, **kw):
        """lqcd_loop_setup: special solves, polynomial, hopping traces, 1/xi', add-backs."""
        o = self._est_opts(seed, nnoise, block, m, k, K, npoly, tol, tol_special, **kw)
        h = C.c_void_p()
        self._check(self.lib.lqcd_loop_setup(self.h, _ptr(links), kappa, C.byref(o), C.byref(h)))
        return Loop(self, h, o)

    def loop_setup_from(self, links, kappa, proj, eig, a, seed, nnoise, block, m, k, K, npoly, tol, tol_special, **kw):
        """lqcd_loop_setup_from: the setup from given spaces (proj: Krylov space of M, eig: eigenpairs
        of M') and Min-Res coefficients a (None: computed)."""
        o = self._est_opts(seed, nnoise, block, m, k, K, npoly, tol, tol_special, **kw)
        h = C.c_void_p()
        ap = None
        if a is not None:
            ah, ap = _host_c(a)
        self._check(self.lib.lqcd_loop_setup_from(self.h, _ptr(links), kappa, C.byref(o), proj.h, eig.h, ap,
                                                  C.byref(h)))
        return Loop(self, h, o, keep=(proj, eig))

    # deflation projection
    def deflate_project(self, defl, eta, d):
        out = _torch().empty_like(eta)
        dh, dp = _host_c(d)
        self._check(self.lib.lqcd_deflate_project(self.h, defl.h, _ptr(eta), _ptr(out), self._nrhs(eta), dp))
        return out

    def set_defl_engine(self, engine):
        """DEFL_FP64 (CUDA-core FP64) or DEFL_TENSOR (split-precision tcgen05) deflation projections."""
        self._check(self.lib.lqcd_set_defl_engine(self.h, engine))

    def set_wait_limit(self, seconds):
        """Bound of the tensor-core kernels' device-side waits (LQCD_ERR_TIMEOUT when one runs out)."""
        self._check(self.lib.lqcd_set_wait_limit(self.h, seconds))

    def inject_tc_stall(self, chunks):
        """Failure injection (tests): the next tensor-core launch stops loading after `chunks` chunks."""
        self._check(self.lib.lqcd_inject_tc_stall(self.h, chunks))

    def tc_vdag_x(self, E, X):
        """G[q, r] = <E_q, X_r> on the tensor cores; E (k, ...) and X (nrhs, ...) complex128 fields."""
        k, nrhs = E.shape[0], X.shape[0]
        G = _torch().empty((k, nrhs), dtype=_torch().complex128, device=X.device)
        self._check(self.lib.lqcd_tc_vdag_x(self.h, _ptr(E), k, _ptr(X), nrhs, _ptr(G)))
        return G

    def tc_v_c(self, E, Cm):
        """Y_r = sum_q E_q C[q, r] on the tensor cores; E (k, ...) fields, C (k, nrhs) complex128."""
        k, nrhs = Cm.shape
        Y = _torch().empty((nrhs,) + tuple(E.shape[1:]), dtype=_torch().complex128, device=E.device)
        self._check(self.lib.lqcd_tc_v_c(self.h, _ptr(E), k, _ptr(Cm.contiguous()), nrhs, _ptr(Y)))
        return Y

    # perturbative and polynomial series
    def hop_series(self, links, kappa, eta, K, c=None):
        out = _torch().empty_like(eta)
        if c is not None:
            ch, cp = _host_c(c)
        else:
            cp = None
        self._check(self.lib.lqcd_hop_series(self.h, _ptr(links), kappa, _ptr(eta), _ptr(out), self._nrhs(eta),
                                             K, cp))
        return out

    def poly_apply(self, links, kappa, eta, a):
        out = _torch().empty_like(eta)
        ah, ap = _host_c(a)
        self._check(self.lib.lqcd_poly_apply(self.h, _ptr(links), kappa, _ptr(eta), _ptr(out), self._nrhs(eta),
                                             len(ah) - 1, ap))
        return out

    def poly_coeffs(self, links, kappa, seed, n):
        a = np.zeros(n + 1, dtype=np.complex128)
        self._check(self.lib.lqcd_poly_coeffs(self.h, _ptr(links), kappa, seed, n, a.ctypes.data_as(C.c_void_p)))
        return a

    # hopping traces
    def hop_traces(self, links, kappa, K):
        t = np.zeros((K, NOPS, self.dims[3]), dtype=np.complex128)
        self._check(self.lib.lqcd_hop_traces(self.h, _ptr(links), kappa, K, t.ctypes.data_as(C.c_void_p)))
        return t

    # 1/xi'
    def xi_inverse(self, links, kappa, defl, sub, K, coeffs=None):
        xi = np.zeros(defl.k, dtype=np.complex128)
        if coeffs is not None:
            ch, cp = _host_c(coeffs)
        else:
            cp = None
        self._check(self.lib.lqcd_xi_inverse(self.h, _ptr(links), kappa, defl.h, sub, K, cp,
                                             xi.ctypes.data_as(C.c_void_p)))
        return xi

    # contractions
    def contract(self, links, kappa, eta, w):
        n = self._nrhs(eta)
        out = np.zeros((n, NOPS, self.dims[3]), dtype=np.complex128)
        self._check(self.lib.lqcd_contract(self.h, _ptr(links), kappa, _ptr(eta), _ptr(w), n,
                                           out.ctypes.data_as(C.c_void_p)))
        return out

    # whole path
    def loop_estimate(self, links, kappa, seed, nnoise, block, m, k, K, npoly, tol, tol_special,
                      m_inner=0, max_cycles=2000, modes=SUB_ALL, prec=PREC_F64, inner_tol=0.0, eig_tol=0.0,
                      system=SYS_M, prec_degree=0, evenodd=0):
        """lqcd_loop_estimate; block = 0 lets the autotuner pick the block width."""
        o = EstOpts(seed, nnoise, block, m, k, m_inner, K, npoly, tol, tol_special, max_cycles, modes, prec,
                    inner_tol, eig_tol, system, prec_degree, evenodd)
        bufs, est = _estimate_buffers(self.dims[3], nnoise, k, npoly)
        st = self.lib.lqcd_loop_estimate(self.h, _ptr(links), kappa, C.byref(o), C.byref(est))
        if st not in (OK, ERR_NOT_CONVERGED):
            self._check(st)
        return _estimate_result(bufs, est, st)

    # batching
    def set_rhs_per_thread(self, nr):
        self._check(self.lib.lqcd_set_rhs_per_thread(self.h, nr))

    def set_graphs(self, enable):
        self._check(self.lib.lqcd_set_graphs(self.h, 1 if enable else 0))

    def set_inner_window(self, window):
        """lqcd_set_inner_window: Lanczos window of Hermitian mixed-precision inner cycles (0 = full)."""
        self._check(self.lib.lqcd_set_inner_window(self.h, window))

    def set_probe_depth(self, depth):
        """lqcd_set_probe_depth: full applications of P per probe in the hopping traces (0 = by cost)."""
        self._check(self.lib.lqcd_set_probe_depth(self.h, depth))

    def set_inner_gs_passes(self, passes):
        """lqcd_set_inner_gs_passes: Gram-Schmidt passes (0 = by storage, 1 or 2) of mixed-precision
        inner cycles."""
        self._check(self.lib.lqcd_set_inner_gs_passes(self.h, passes))

    def autotune_block(self, links, kappa, defl, m, candidates=(8, 16, 32), prec=PREC_F64, inner_tol=0.0):
        """lqcd_autotune_block: (best width, {width: seconds per right-hand side and cycle})."""
        o = KrylovOpts(m, 0, 1e-10, 1, SYS_M, prec, inner_tol)
        cand = (C.c_int * len(candidates))(*candidates)
        secs = (C.c_double * len(candidates))()
        best = C.c_int()
        self._check(self.lib.lqcd_autotune_block(self.h, _ptr(links), kappa, defl.h, C.byref(o), cand,
                                                 len(candidates), C.byref(best), secs))
        return best.value, dict(zip(candidates, list(secs)))



class EvenOddContext(Context):
    """lqcd_ctx_create_evenodd: the reduced (even-site) system of a full lattice (Sec. 7).  Its fields
    are (nrhs, V/2, 4, 3) complex128 (even sites in lexicographic order), wilson_apply applies
    hat M = 1 - kappa^2 P_eo P_oe, and the Krylov solvers of Context solve the reduced system."""

    def __init__(self, dims, stream=None, recon=18):
        torch = _torch()
        self.lib = load()
        self.full_dims = tuple(int(d) for d in dims)
        self.dims = (self.full_dims[0] // 2,) + self.full_dims[1:]
        self.V = int(np.prod(self.dims))
        self.N = 12 * self.V
        self.device = torch.device("cuda", torch.cuda.current_device())
        s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        h = C.c_void_p()
        dd = (C.c_int * 4)(*self.full_dims)
        st = self.lib.lqcd_ctx_create_evenodd(C.byref(h), dd, recon, C.c_void_p(s))
        if st != OK:
            raise LqcdError(st, "lqcd_ctx_create_evenodd failed")
        self.h = h

    def field(self, nrhs=None):
        torch = _torch()
        shp = (self.V, 4, 3) if nrhs is None else (nrhs, self.V, 4, 3)
        return torch.empty(shp, dtype=torch.complex128, device=self.device)

    def full_field(self, nrhs):
        torch = _torch()
        lx, ly, lz, lt = self.full_dims
        return torch.empty((nrhs, lt, lz, ly, lx, 4, 3), dtype=torch.complex128, device=self.device)

    def split(self, full):
        n = full.numel() // (2 * self.N)
        e, o = self.field(n), self.field(n)
        self._check(self.lib.lqcd_eo_split(self.h, _ptr(full), _ptr(e), _ptr(o), n))
        return e, o

    def join(self, even, odd):
        n = self._nrhs(even)
        out = self.full_field(n)
        self._check(self.lib.lqcd_eo_join(self.h, _ptr(even), _ptr(odd), _ptr(out), n))
        return out

    def hop(self, links, inp, parity_out):
        """P_eo inp (parity_out 0) or P_oe inp (parity_out 1)."""
        out = _torch().empty_like(inp)
        self._check(self.lib.lqcd_eo_hop(self.h, _ptr(links), _ptr(inp), _ptr(out), self._nrhs(inp), parity_out))
        return out

    def rhs(self, links, kappa, b):
        n = b.numel() // (2 * self.N)
        out = self.field(n)
        self._check(self.lib.lqcd_eo_rhs(self.h, _ptr(links), kappa, _ptr(b), _ptr(out), n))
        return out

    def reconstruct(self, links, kappa, xe, b):
        n = self._nrhs(xe)
        out = self.full_field(n)
        self._check(self.lib.lqcd_eo_reconstruct(self.h, _ptr(links), kappa, _ptr(xe), _ptr(b), _ptr(out), n))
        return out

    def full_eigenpairs(self, links, kappa, mu, Ve, tol=1e-8):
        """(lam (2Q,), E (2Q, T, Z, Y, X, 4, 3)) of M from reduced pairs (mu (Q,), Ve (Q, V/2, 4, 3))."""
        q = len(mu)
        m, mp = _host_c(mu)
        lam = np.zeros(2 * q, dtype=np.complex128)
        E = self.full_field(2 * q)
        self._check(self.lib.lqcd_eo_full_eigenpairs(self.h, _ptr(links), kappa, mp, _ptr(Ve.contiguous()), q, tol,
                                                     lam.ctypes.data_as(C.c_void_p), _ptr(E)))
        return lam, E

def probe_classes(dims, K):
    """lqcd_probe_classes (host only): (number of classes, class of every site as an int array of
    shape (T, Z, Y, X))."""
    lib = load()
    d = (C.c_int * 4)(*dims)
    n = C.c_int()
    cls = np.zeros(int(np.prod(dims)), dtype=np.int32)
    st = lib.lqcd_probe_classes(d, K, C.byref(n), cls.ctypes.data_as(C.c_void_p))
    if st != OK:
        raise LqcdError(st, "probe_classes: bad arguments")
    return n.value, cls.reshape(dims[3], dims[2], dims[1], dims[0])


def probe_depth(dims, K, fixed=0):
    """lqcd_probe_depth (host only): full applications of P per probe that lqcd_hop_traces uses."""
    lib = load()
    d = (C.c_int * 4)(*dims)
    out = C.c_int()
    st = lib.lqcd_probe_depth(d, K, fixed, C.byref(out))
    if st != OK:
        raise LqcdError(st, "probe_depth: bad arguments")
    return out.value


def _estimate_buffers(lt, nnoise, k, npoly):
    bufs = dict(per_noise=np.zeros((NMODES, nnoise, NOPS), dtype=np.complex128),
                per_t=np.zeros((NMODES, NOPS, lt), dtype=np.complex128),
                addback=np.zeros((NMODES, NOPS, lt), dtype=np.complex128),
                mean=np.zeros((NMODES, NOPS), dtype=np.complex128),
                stderr=np.zeros((NMODES, NOPS), dtype=np.float64),
                lam=np.zeros(k, dtype=np.complex128),
                poly_a=np.zeros(npoly + 1, dtype=np.complex128))
    as_dp = lambda a: a.ctypes.data_as(_dp)
    est = Estimate(*[as_dp(bufs[n]) for n in ("per_noise", "per_t", "addback", "mean", "stderr", "lam", "poly_a")],
                   0, 0, 0.0, 0.0, 0.0, 0, 0)
    return bufs, est


def _estimate_result(bufs, est, st):
    return dict(bufs, matvecs_setup=est.matvecs_setup, matvecs_noise=est.matvecs_noise,
                seconds_setup=est.seconds_setup, seconds_noise=est.seconds_noise,
                max_true_resid=est.max_true_resid, converged=bool(est.converged), block=est.block, status=st)


def batch_loop_estimate(problems):
    """lqcd_batch_loop_estimate: loop estimates of several problems (distinct contexts, lattices of any
    size) run concurrently.  problems: list of dicts with ctx, links, kappa and the keyword arguments of
    Context.loop_estimate (seed, nnoise, block, m, k, K, npoly, tol, tol_special, and optional m_inner,
    max_cycles, modes, prec, inner_tol).  Returns the list of result dicts (each with its status)."""
    n = len(problems)
    opts = (EstOpts * n)()
    ests = (Estimate * n)()
    keep = []
    for i, p in enumerate(problems):
        opts[i] = EstOpts(p["seed"], p["nnoise"], p["block"], p["m"], p["k"], p.get("m_inner", 0), p["K"], p["npoly"],
                          p["tol"], p["tol_special"], p.get("max_cycles", 2000), p.get("modes", SUB_ALL),
                          p.get("prec", PREC_F64), p.get("inner_tol", 0.0), p.get("eig_tol", 0.0),
                          p.get("system", SYS_M), p.get("prec_degree", 0))
        bufs, est = _estimate_buffers(p["ctx"].dims[3], p["nnoise"], p["k"], p["npoly"])
        ests[i] = est
        keep.append(bufs)
    ctxs = (C.c_void_p * n)(*[p["ctx"].h.value for p in problems])
    links = (C.c_void_p * n)(*[_ptr(p["links"]).value for p in problems])
    kappas = (C.c_double * n)(*[p["kappa"] for p in problems])
    status = (C.c_int * n)()
    problems[0]["ctx"].lib.lqcd_batch_loop_estimate(n, ctxs, links, kappas, opts, ests, status)
    out = []
    for i, p in enumerate(problems):
        if status[i] not in (OK, ERR_NOT_CONVERGED):
            p["ctx"]._check(status[i])
        out.append(_estimate_result(keep[i], ests[i], status[i]))
    return out


def _link_grad_buffers(ctx, want_links):
    torch = _torch()
    lx, ly, lz, lt = ctx.dims
    g = torch.zeros((4, lt, lz, ly, lx, 8), dtype=torch.complex128, device=ctx.device)
    gl = torch.zeros((4, lt, lz, ly, lx, 3, 3), dtype=torch.complex128, device=ctx.device) if want_links else None
    return g, gl


def link_grad(ctx, links, kappa, z, x, scale=1.0, want_links=True):
    """dT/dw (4, T, Z, Y, X, 8) and the torch-convention gradient of Re T (4, T, Z, Y, X, 3, 3), summed
    over the right-hand sides of z and x and multiplied by scale (lqcd_link_grad)."""
    g, gl = _link_grad_buffers(ctx, want_links)
    ctx._check(ctx.lib.lqcd_link_grad(ctx.h, _ptr(links), kappa, _ptr(z), _ptr(x), ctx._nrhs(x), scale, _ptr(g),
                                      _ptr(gl)))
    return g, gl


def loop_derivs(ctx, links, kappa, seed, nnoise, block, m, k, K, tol, tol_special, m_inner=0, max_cycles=2000,
                prec=PREC_F64, want_grad=True, grad_scale=1.0, inner_tol=0.0, eig_tol=0.0, system=SYS_M):
    """lqcd_loop_derivs: d/dkappa of the NS and PS estimates of the nine operators, and the link
    gradient of the NS scalar estimate."""
    o = EstOpts(seed, nnoise, block, m, k, m_inner, K, 0, tol, tol_special, max_cycles, SUB_NONE | SUB_PERT, prec,
                inner_tol, eig_tol, system)
    dk = np.zeros((2, NOPS), dtype=np.complex128)
    err = np.zeros((2, NOPS), dtype=np.float64)
    per = np.zeros((2, nnoise, NOPS), dtype=np.complex128)
    g, gl = _link_grad_buffers(ctx, want_grad) if want_grad else (None, None)
    as_dp = lambda a: a.ctypes.data_as(_dp)
    out = Derivs(grad_scale, as_dp(dk), as_dp(err), as_dp(per), C.c_void_p(g.data_ptr()) if g is not None else None,
                 C.c_void_p(gl.data_ptr()) if gl is not None else None, 0, 0.0, 0.0, 0)
    st = ctx.lib.lqcd_loop_derivs(ctx.h, _ptr(links), kappa, C.byref(o), C.byref(out))
    if st not in (OK, ERR_NOT_CONVERGED):
        ctx._check(st)
    return dict(dkappa=dk, dkappa_err=err, per_noise=per, link_grad=g, grad_links=gl, matvecs=out.matvecs,
                seconds=out.seconds, max_true_resid=out.max_true_resid, converged=bool(out.converged))


def tc_slice_bytes(dims, k):
    """Device bytes of the tensor-core slices of k vectors on a lattice of dims (Lx, Ly, Lz, Lt);
    host only (no GPU needed)."""
    lib = load()
    out = C.c_size_t()
    st = lib.lqcd_tc_slice_bytes((C.c_int * 4)(*dims), k, C.byref(out))
    if st != OK:
        raise LqcdError(st, "tc_slice_bytes: bad arguments")
    return out.value


def header_functions(header=None):
    """Names of the functions declared in include/lqcd.h (for the ABI export check)."""
    import re
    header = header or os.path.join(_build.ROOT, "include", "lqcd.h")
    txt = open(header).read()
    return sorted(set(re.findall(r"\b(lqcd_[a-z0-9_]+)\s*\(", txt)))
