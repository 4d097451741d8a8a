"""Thin ctypes binding of libhelk.so (include/helk.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Functions carry the C names; ``Context`` wraps them for torch
tensors (device memory and streams come from PyTorch).  There is no CPU
fallback: if the library cannot be loaded, importing this module raises.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhelk.so")

HELK_OK = 0
HELK_ERR_INVALID_ARG = -1
HELK_ERR_OOM = -2
HELK_ERR_CUDA = -3
HELK_ERR_STATE = -4
HELK_ERR_TIMEOUT = -5
HELK_ERR_UNSUPPORTED = -6
STATUS_NAMES = {0: "HELK_OK", -1: "HELK_ERR_INVALID_ARG", -2: "HELK_ERR_OOM", -3: "HELK_ERR_CUDA",
                -4: "HELK_ERR_STATE", -5: "HELK_ERR_TIMEOUT", -6: "HELK_ERR_UNSUPPORTED"}

HELK_CUT_ABS, HELK_CUT_LORENTZ, HELK_CUT_NONE = 0, 1, 2
HELK_PROBE_FFMA, HELK_PROBE_DFMA, HELK_PROBE_MUFU_RCP, HELK_PROBE_MUFU_EX2 = 0, 1, 2, 3
HELK_PREC_F64, HELK_PREC_F32_KAHAN = 0, 1


class helk_grid(ctypes.Structure):
    _fields_ = [("nu_min", ctypes.c_double), ("dnu", ctypes.c_double), ("n", ctypes.c_int64)]


class helk_cutoff(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("value", ctypes.c_double), ("cap", ctypes.c_double)]


class helk_lines(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in
                ("nu0", "S0", "E_lower", "gamma_air", "gamma_self", "n_coll", "delta", "mass",
                 "weight")]


class helk_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("accumulate", ctypes.c_int32),
                ("weight", ctypes.c_double), ("q_ratio", ctypes.c_double),
                ("count_regions", ctypes.c_int32), ("surrogate", ctypes.c_int32)]


LINE_FIELDS = ("nu0", "S0", "E_lower", "gamma_air", "gamma_self", "n_coll", "delta", "mass",
               "weight")

# (name, restype, argtypes) of every exported entry point of include/helk.h
_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_D = ctypes.c_double
SIGNATURES = [
    ("helk_create", ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, _P]),
    ("helk_destroy", None, [_P]),
    ("helk_last_error", ctypes.c_char_p, [_P]),
    ("helk_set_stream", ctypes.c_int, [_P, _P]),
    ("helk_sync", ctypes.c_int, [_P]),
    ("helk_lines_upload", ctypes.c_int, [_P, ctypes.POINTER(helk_lines), _I64, _I32]),
    ("helk_opacity", ctypes.c_int, [_P, _D, _D, _D, ctypes.POINTER(helk_cutoff),
                                    ctypes.POINTER(helk_grid), ctypes.POINTER(helk_opts), _P]),
    ("helk_opacity_stats", ctypes.c_int, [_P, ctypes.POINTER(_I64), _P]),
    ("helk_kdist", ctypes.c_int, [_P, _P, _I64, _I32, _I32, _D, _P, _P, _I32, _P]),
    ("helk_set_profiling", ctypes.c_int, [_P, _I32]),
    ("helk_stage_times", ctypes.c_int, [_P, _P, _P]),
    ("helk_kdist_static", ctypes.c_int, [_P, _I64, _I32, _I32, _D, _P, _P, _P, _P]),
    ("helk_opacity_batch", ctypes.c_int, [_P, _I32, _P, _P, _P, _D, ctypes.POINTER(helk_cutoff),
                                          ctypes.POINTER(helk_grid), ctypes.POINTER(helk_opts), _P]),
    ("helk_opacity_batch_stats", ctypes.c_int, [_P, _I32, _P, _P]),
    ("helk_transmission", ctypes.c_int, [_P, _I32, _I64, _P, _P, _I32, _I32, _I32, _P, _P, _P]),
    ("helk_selftest_timeout", ctypes.c_int, [_P, _I32]),
    ("helk_surrogate_init", ctypes.c_int, [_P, ctypes.c_uint64]),
    ("helk_surrogate_params", ctypes.c_int, [_P, _P, _P]),
    ("helk_surrogate_samples", ctypes.c_int, [_P, _I64, ctypes.c_uint64, _P, _P, _P, _P]),
    ("helk_surrogate_grad", ctypes.c_int, [_P, _I64, _P, _P, _P, _P]),
    ("helk_surrogate_train", ctypes.c_int, [_P, _I64, ctypes.c_uint64, _I32, _I32, _D, _P]),
    ("helk_surrogate_eval", ctypes.c_int, [_P, _I64, _P, _P, _P]),
    ("helk_surrogate_validate", ctypes.c_int, [_P, _I32, _I32, _I32, _D, _P, _P]),
    ("helk_autotune", ctypes.c_int, [_P, _D, _D, _D, ctypes.POINTER(helk_cutoff),
                                     ctypes.POINTER(helk_grid), ctypes.POINTER(helk_opts),
                                     ctypes.POINTER(_I32)]),
    ("helk_tile_candidates", _I32, [_I32, _P, _I32]),
    ("helk_tile_shape", ctypes.c_int, [_I32, _I32, _P, _P, _P]),
    ("helk_launch_count", _I64, [_P]),
    ("helk_set_tile", ctypes.c_int, [_P, _I32, _I64, _I32]),
    ("helk_peak_probe", ctypes.c_int, [_P, _I32, _P, _P]),
    ("helk_set_batch_budget", ctypes.c_int, [_P, _I64]),
]
HELK_NSTAGES = 4
MLP_NPARAMS = 8577
STAGE_NAMES = ("lineprep", "voigt", "kdist", "setup")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libhelk.so is not built (run __graft_entry__.build() or "
                          "python paper_1503_03806_gb300/build.py); there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


class HelkError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


# ----------------------------------------------- C-named thin wrappers ---
def helk_create(device=0, stream=None):
    h = _P()
    st = lib.helk_create(ctypes.byref(h), int(device), stream)
    if st != HELK_OK:
        raise HelkError(st, "helk_create failed")
    return h


def helk_destroy(ctx):
    lib.helk_destroy(ctx)


def helk_last_error(ctx):
    s = lib.helk_last_error(ctx)
    return s.decode() if s else ""


def _check(ctx, st):
    if st != HELK_OK:
        raise HelkError(st, helk_last_error(ctx))
    return st


def helk_set_stream(ctx, stream):
    return _check(ctx, lib.helk_set_stream(ctx, stream))


def helk_sync(ctx):
    return _check(ctx, lib.helk_sync(ctx))


def helk_lines_upload(ctx, lines_struct, n, on_device):
    return lib.helk_lines_upload(ctx, ctypes.byref(lines_struct), int(n), int(on_device))


def helk_opacity(ctx, T, P, mass, cut, grid, opts, kappa_ptr):
    return lib.helk_opacity(ctx, float(T), float(P), float(mass), ctypes.byref(cut),
                            ctypes.byref(grid), None if opts is None else ctypes.byref(opts),
                            kappa_ptr)


def helk_opacity_stats(ctx, with_regions=False):
    ev = _I64(0)
    reg = np.zeros(4, dtype=np.int64)
    st = lib.helk_opacity_stats(ctx, ctypes.byref(ev),
                                reg.ctypes.data_as(_P) if with_regions else None)
    _check(ctx, st)
    return int(ev.value), (reg if with_regions else None)


def helk_kdist(ctx, kappa_ptr, n, nbins, ncheb, kappa_floor, coeffs_ptr, mean_ptr, out_on_host,
               kg_ptr):
    return lib.helk_kdist(ctx, kappa_ptr, int(n), int(nbins), int(ncheb), float(kappa_floor),
                          coeffs_ptr, mean_ptr, int(out_on_host), kg_ptr)


def helk_set_profiling(ctx, on):
    return _check(ctx, lib.helk_set_profiling(ctx, int(bool(on))))


def helk_stage_times(ctx):
    ms = np.zeros(HELK_NSTAGES)
    cnt = np.zeros(HELK_NSTAGES, dtype=np.int64)
    _check(ctx, lib.helk_stage_times(ctx, ms.ctypes.data_as(_P), cnt.ctypes.data_as(_P)))
    return {n: (float(ms[i]), int(cnt[i])) for i, n in enumerate(STAGE_NAMES)}


# -------------------------------------------------------------- Context --
def helk_tile_candidates(precision):
    """The shape codes of a precision's Voigt kernel that the autotuner times."""
    out = (_I32 * 32)()
    n = lib.helk_tile_candidates(int(precision), out, 32)
    return [int(out[i]) for i in range(min(n, 32))]


def helk_tile_shape(precision, code):
    """A shape code decoded: {"points": per CTA tile, "warps": per CTA,
    "lines_per_stage": candidate lines per pipeline stage}."""
    p, w, l = _I32(0), _I32(0), _I32(0)
    st = lib.helk_tile_shape(int(precision), int(code), ctypes.byref(p), ctypes.byref(w), ctypes.byref(l))
    if st != HELK_OK:
        raise HelkError(st, "tile_shape: unknown precision or shape code %r" % (code,))
    return {"points": int(p.value), "warps": int(w.value), "lines_per_stage": int(l.value)}


def _cut(cut):
    """cut: ("abs", C) | ("lorentz", multiple, cap) | ("none",)"""
    kind = cut[0]
    if kind == "abs":
        return helk_cutoff(HELK_CUT_ABS, float(cut[1]), 0.0)
    if kind == "lorentz":
        return helk_cutoff(HELK_CUT_LORENTZ, float(cut[1]), float(cut[2]))
    if kind == "none":
        return helk_cutoff(HELK_CUT_NONE, 0.0, 0.0)
    raise ValueError("unknown cutoff %r" % (cut,))


class Context:
    """A libhelk context bound to one CUDA device and (optionally) a torch
    stream.  Tensors passed in must live on that device."""

    def __init__(self, device=0, stream=None):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        self._stream = stream
        sp = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        self.h = helk_create(self.device.index or 0, sp)
        self.nlines = 0

    def close(self):
        if self.h:
            helk_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        self._stream = stream
        helk_set_stream(self.h, None if stream is None else ctypes.c_void_p(stream.cuda_stream))

    def sync(self):
        helk_sync(self.h)

    # lines: dict of numpy arrays (host) or torch cuda tensors (device)
    def upload(self, lines):
        torch = self.torch
        keep = {}
        on_device = None
        n = None
        s = helk_lines()
        for k in LINE_FIELDS:
            v = lines.get(k)
            if v is None:
                continue
            if isinstance(v, torch.Tensor):
                dev = v.is_cuda
                v = v.contiguous().to(torch.float64)
                ptr = v.data_ptr()
            else:
                dev = False
                v = np.ascontiguousarray(v, dtype=np.float64)
                ptr = v.ctypes.data
            if on_device is None:
                on_device = dev
            elif on_device != dev:
                raise ValueError("all line fields must be on the same side (host or device)")
            keep[k] = v
            setattr(s, k, ptr)
            n = v.shape[0] if n is None else n
            if v.shape[0] != n:
                raise ValueError("line fields differ in length")
        _check(self.h, helk_lines_upload(self.h, s, n or 0, 1 if on_device else 0))
        self.nlines = n or 0

    def opacity(self, T, P, mass, cut, grid, out=None, precision=HELK_PREC_F64, accumulate=False,
                weight=1.0, q_ratio=1.0, count_regions=False, surrogate=False):
        """grid = (nu_min, dnu, n).  Returns the kappa tensor (float64)."""
        torch = self.torch
        g = helk_grid(float(grid[0]), float(grid[1]), int(grid[2]))
        if out is None:
            out = torch.empty(int(grid[2]), dtype=torch.float64, device=self.device)
        assert out.dtype == torch.float64 and out.is_cuda and out.is_contiguous()
        o = helk_opts(int(precision), int(bool(accumulate)), float(weight), float(q_ratio),
                      int(bool(count_regions)), int(bool(surrogate)))
        _check(self.h, helk_opacity(self.h, T, P, mass, _cut(cut), g, o, ctypes.c_void_p(out.data_ptr())))
        return out

    def opacity_batch(self, T, P, mass, cut, grid, out=None, precision=HELK_PREC_F64, q_ratio=None,
                      accumulate=False, weight=1.0, count_regions=False, surrogate=False):
        """n_cond conditions (T[k], P[k]) in one graph-captured persistent launch;
        returns kappa as a (n_cond, n) float64 tensor."""
        torch = self.torch
        T = np.ascontiguousarray(T, dtype=np.float64)
        P = np.ascontiguousarray(P, dtype=np.float64)
        nc = T.shape[0]
        q = None if q_ratio is None else np.ascontiguousarray(q_ratio, dtype=np.float64)
        g = helk_grid(float(grid[0]), float(grid[1]), int(grid[2]))
        if out is None:
            out = torch.empty((nc, int(grid[2])), dtype=torch.float64, device=self.device)
        assert out.dtype == torch.float64 and out.is_cuda and out.is_contiguous()
        o = helk_opts(int(precision), int(bool(accumulate)), float(weight), 1.0, int(bool(count_regions)),
                      int(bool(surrogate)))
        _check(self.h, lib.helk_opacity_batch(self.h, nc, T.ctypes.data_as(_P), P.ctypes.data_as(_P),
                                              None if q is None else q.ctypes.data_as(_P), float(mass),
                                              ctypes.byref(_cut(cut)), ctypes.byref(g), ctypes.byref(o),
                                              ctypes.c_void_p(out.data_ptr())))
        return out

    def transmission(self, nbins, m, sorted_k=None, coeffs=None, ng=None):
        """Per-bin transmission for column masses m: (direct, fit), each a
        (nbins, nm) tensor or None."""
        torch = self.torch
        m = np.ascontiguousarray(np.atleast_1d(m), dtype=np.float64)
        nm = m.shape[0]
        nb = 0 if sorted_k is None else sorted_k.numel() // nbins
        ncheb = 0 if coeffs is None else coeffs.shape[-1]
        if ng is None:
            ng = max(nb, 1)
        direct = None if sorted_k is None else torch.empty((nbins, nm), dtype=torch.float64, device=self.device)
        fit = None if coeffs is None else torch.empty((nbins, nm), dtype=torch.float64, device=self.device)
        p = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
        _check(self.h, lib.helk_transmission(self.h, int(nbins), int(nb), p(sorted_k), p(coeffs), int(ncheb),
                                             int(ng), int(nm), m.ctypes.data_as(_P), p(direct), p(fit)))
        return direct, fit

    def set_batch_budget(self, nbytes):
        """Line-record bytes one chunk of opacity_batch may use (0: default)."""
        _check(self.h, lib.helk_set_batch_budget(self.h, int(nbytes)))

    def batch_stats(self, n_cond, with_regions=False):
        ev = np.zeros(n_cond, dtype=np.int64)
        reg = np.zeros((n_cond, 4), dtype=np.int64)
        _check(self.h, lib.helk_opacity_batch_stats(self.h, int(n_cond), ev.ctypes.data_as(_P),
                                                    reg.ctypes.data_as(_P) if with_regions else None))
        return ev, (reg if with_regions else None)

    def autotune(self, T, P, mass, cut, grid, precision=HELK_PREC_F64, q_ratio=1.0):
        """Time the candidate Voigt kernel shapes on this condition; keep the
        fastest for later calls with the same precision and grid size.
        Returns its shape code (helk_tile_shape decodes it)."""
        g = helk_grid(float(grid[0]), float(grid[1]), int(grid[2]))
        o = helk_opts(int(precision), 0, 1.0, float(q_ratio), 0, 0)
        t = _I32(0)
        _check(self.h, lib.helk_autotune(self.h, float(T), float(P), float(mass), ctypes.byref(_cut(cut)),
                                         ctypes.byref(g), ctypes.byref(o), ctypes.byref(t)))
        return int(t.value)

    def launch_count(self):
        """Kernels this context has launched so far."""
        return int(lib.helk_launch_count(self.h))

    def set_tile(self, precision, n, tile):
        """Fix the Voigt kernel shape (a code from helk_tile_candidates) for
        grids of n points (0: built-in choice)."""
        _check(self.h, lib.helk_set_tile(self.h, int(precision), int(n), int(tile)))

    # ------------------------------------------------------ surrogate --
    def surrogate_init(self, seed=0):
        _check(self.h, lib.helk_surrogate_init(self.h, int(seed)))

    def surrogate_params(self, new=None):
        """Current parameters (numpy float32, 8577); replaces them first if new."""
        out = np.empty(MLP_NPARAMS, dtype=np.float32)
        src = None if new is None else np.ascontiguousarray(new, dtype=np.float32)
        _check(self.h, lib.helk_surrogate_params(self.h, out.ctypes.data_as(_P),
                                                 None if src is None else src.ctypes.data_as(_P)))
        return out

    def surrogate_samples(self, n, seed):
        torch = self.torch
        feat = torch.empty((n, 2), dtype=torch.float32, device=self.device)
        tgt = torch.empty(n, dtype=torch.float32, device=self.device)
        x = torch.empty(n, dtype=torch.float64, device=self.device)
        y = torch.empty(n, dtype=torch.float64, device=self.device)
        _check(self.h, lib.helk_surrogate_samples(self.h, int(n), int(seed), ctypes.c_void_p(feat.data_ptr()),
                                                  ctypes.c_void_p(tgt.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                                  ctypes.c_void_p(y.data_ptr())))
        return feat, tgt, x, y

    def surrogate_grad(self, feat, tgt):
        g = np.empty(MLP_NPARAMS, dtype=np.float32)
        loss = ctypes.c_double(0.0)
        _check(self.h, lib.helk_surrogate_grad(self.h, int(tgt.numel()), ctypes.c_void_p(feat.data_ptr()),
                                               ctypes.c_void_p(tgt.data_ptr()), g.ctypes.data_as(_P),
                                               ctypes.byref(loss)))
        return g, loss.value

    def surrogate_train(self, n_samples, seed, epochs, batch=4096, lr=2e-3):
        loss = ctypes.c_double(0.0)
        _check(self.h, lib.helk_surrogate_train(self.h, int(n_samples), int(seed), int(epochs), int(batch),
                                                float(lr), ctypes.byref(loss)))
        return loss.value

    def surrogate_eval(self, x, y):
        torch = self.torch
        k = torch.empty_like(x)
        _check(self.h, lib.helk_surrogate_eval(self.h, int(x.numel()), ctypes.c_void_p(x.data_ptr()),
                                               ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(k.data_ptr())))
        return k

    def surrogate_validate(self, nx=32, ny=32, per_cell=6, tol=1e-4):
        mask = np.zeros(nx * ny, dtype=np.uint8)
        err = np.zeros(nx * ny)
        _check(self.h, lib.helk_surrogate_validate(self.h, nx, ny, per_cell, float(tol),
                                                   mask.ctypes.data_as(_P), err.ctypes.data_as(_P)))
        return mask.reshape(ny, nx), err.reshape(ny, nx)

    def peak_probe(self, kind):
        """Measured throughput of one arithmetic unit (HELK_PROBE_*):
        (ops per second, ms per launch)."""
        ops, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
        _check(self.h, lib.helk_peak_probe(self.h, int(kind), ctypes.byref(ops), ctypes.byref(ms)))
        return ops.value, ms.value

    def set_profiling(self, on):
        helk_set_profiling(self.h, on)

    def stage_times(self):
        return helk_stage_times(self.h)

    def stats(self, with_regions=False):
        return helk_opacity_stats(self.h, with_regions)

    def kdist(self, kappa, nbins, ncheb=20, kappa_floor=1e-250, want_sorted=False, on_host=False):
        """Returns (coeffs[nbins, ncheb], mean[nbins], sorted or None)."""
        torch = self.torch
        n = int(kappa.shape[0])
        kg = torch.empty_like(kappa) if want_sorted else None
        if on_host:
            coef = np.empty((nbins, ncheb))
            mean = np.empty(nbins)
            cp, mp = coef.ctypes.data, mean.ctypes.data
        else:
            coef = torch.empty((nbins, ncheb), dtype=torch.float64, device=self.device)
            mean = torch.empty(nbins, dtype=torch.float64, device=self.device)
            cp, mp = coef.data_ptr(), mean.data_ptr()
        _check(self.h, helk_kdist(self.h, ctypes.c_void_p(kappa.data_ptr()), n, nbins, ncheb, kappa_floor,
                                  ctypes.c_void_p(cp), ctypes.c_void_p(mp), 1 if on_host else 0,
                                  None if kg is None else ctypes.c_void_p(kg.data_ptr())))
        return coef, mean, kg
