"""Thin ctypes binding of libfourphonon (same names as include/fourphonon.h).

Argument marshalling only: every step of the rate path runs in the library's CUDA
kernels.  Loading fails loudly when the library has not been built; there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

FP_OK = 0
FP_EINVAL = -1
FP_ENOMEM = -2
FP_ECUDA = -3
FP_EUNSTABLE = -4
FP_ESTATE = -6
FP_PREC_FP64 = 0
FP_PREC_MIXED = 1
FP_PREC_DOUBLE_FLOAT = 2


class fp_fc2(ctypes.Structure):
    _fields_ = [("i", ctypes.c_int), ("j", ctypes.c_int), ("Rj", ctypes.c_int * 3), ("fc", ctypes.c_double * 9)]


class fp_fc4(ctypes.Structure):
    _fields_ = [("i", ctypes.c_int), ("j", ctypes.c_int), ("k", ctypes.c_int), ("l", ctypes.c_int),
                ("Rj", ctypes.c_int * 3), ("Rk", ctypes.c_int * 3), ("Rl", ctypes.c_int * 3),
                ("fc", ctypes.c_double * 81)]


class fp_fc3(ctypes.Structure):
    _fields_ = [("i", ctypes.c_int), ("j", ctypes.c_int), ("k", ctypes.c_int),
                ("Rj", ctypes.c_int * 3), ("Rk", ctypes.c_int * 3), ("fc", ctypes.c_double * 27)]


class fp_rates_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("window", ctypes.c_double), ("sigma_min", ctypes.c_double),
                ("dq_mode", ctypes.c_int), ("mode_mask", ctypes.POINTER(ctypes.c_ubyte)),
                ("q_begin", ctypes.c_int), ("q_end", ctypes.c_int), ("block_j0", ctypes.c_int),
                ("k1_tile", ctypes.c_int), ("threads", ctypes.c_int), ("no_graph", ctypes.c_int),
                ("process_mask", ctypes.c_int), ("nu_select", ctypes.c_int), ("no_time_reversal", ctypes.c_int),
                ("tensor_cores", ctypes.c_int)]


class fp_stats(ctypes.Structure):
    _fields_ = [("candidates", ctypes.c_double), ("accepted", ctypes.c_double * 3), ("flops", ctypes.c_double),
                ("ms", ctypes.c_double), ("tile", ctypes.c_int * 4), ("candidates_executed", ctypes.c_double),
                ("vertex_entries", ctypes.c_double), ("terms_executed", ctypes.c_double)]

    def as_dict(self):
        return {"candidates": self.candidates, "accepted": list(self.accepted), "flops": self.flops,
                "ms": self.ms, "tile": list(self.tile), "candidates_executed": self.candidates_executed,
                "vertex_entries": self.vertex_entries, "terms_executed": self.terms_executed}


EXPORTS = ["fp_version", "fp_default_opts", "fp_init", "fp_set_stream", "fp_modes", "fp_set_modes", "fp_rates4",
           "fp_rates4_channels", "fp_rates4_nu", "fp_set_fc3", "fp_rates3", "fp_kappa_rta", "fp_rates4_irreducible",
           "fp_star_table", "fp_rates4_device", "fp_rates4_noalloc", "fp_autotune", "fp_phase3", "fp_phase4",
           "fp_mlp_params_size", "fp_mlp_loss_grad", "fp_surrogate_default_opts", "fp_surrogate_fit",
           "fp_surrogate_rates", "fp_free", "fp_last_error", "fp_phase_space4", "fp_surrogate_sweep", "fp_write_fc4",
           "fp_read_fc4", "fp_write_fc3", "fp_read_fc3"]


class fp_surrogate_opts(ctypes.Structure):
    _fields_ = [("train_frac", ctypes.c_double), ("holdout_frac", ctypes.c_double), ("tol", ctypes.c_double),
                ("seed", ctypes.c_ulonglong), ("epochs", ctypes.c_int), ("batch", ctypes.c_int),
                ("lr", ctypes.c_double), ("precision", ctypes.c_int)]


class fp_surrogate_report(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in ("n_modes", "n_train", "n_holdout", "n_fallback_modes", "n_bins",
                                            "n_bins_fallback")] + \
               [(n, ctypes.c_double) for n in ("final_loss", "holdout_median_rel_err", "holdout_p90_rel_err",
                                               "holdout_max_rel_err", "ms_exact", "ms_features", "ms_train",
                                               "ms_predict", "ms_fallback", "ms_total")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


_LIB = None


class FourPhononError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libfourphonon error {code}: {msg}")
        self.code = code


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libfourphonon.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or library_path()
    if not os.path.exists(path):
        raise FileNotFoundError(f"libfourphonon.so is not built ({path}); run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    L.fp_version.restype = ctypes.c_int
    L.fp_default_opts.argtypes = [ctypes.POINTER(fp_rates_opts)]
    L.fp_default_opts.restype = None
    L.fp_init.argtypes = [ctypes.POINTER(vp), dp, ctypes.c_int, dp, dp, ctypes.c_int, ctypes.POINTER(fp_fc2),
                          ctypes.c_int, ctypes.POINTER(fp_fc4), ctypes.POINTER(ctypes.c_int), ctypes.c_int]
    L.fp_init.restype = ctypes.c_int
    L.fp_set_stream.argtypes = [vp, vp]
    L.fp_set_stream.restype = ctypes.c_int
    L.fp_modes.argtypes = [vp, vp, vp, vp]
    L.fp_modes.restype = ctypes.c_int
    L.fp_set_modes.argtypes = [vp, dp, dp, dp]
    L.fp_set_modes.restype = ctypes.c_int
    L.fp_rates4.argtypes = [vp, ctypes.c_int, dp, ctypes.c_double, ctypes.POINTER(fp_rates_opts), dp,
                            ctypes.POINTER(fp_stats)]
    L.fp_rates4.restype = ctypes.c_int
    L.fp_rates4_device.argtypes = [vp, ctypes.c_int, dp, ctypes.c_double, ctypes.POINTER(fp_rates_opts), vp,
                                   ctypes.POINTER(fp_stats)]
    L.fp_rates4_channels.argtypes = [vp, ctypes.c_int, dp, ctypes.c_double, ctypes.POINTER(fp_rates_opts), dp,
                                     ctypes.POINTER(fp_stats)]
    L.fp_rates4_channels.restype = ctypes.c_int
    L.fp_set_fc3.argtypes = [vp, ctypes.c_int, ctypes.POINTER(fp_fc3)]
    L.fp_set_fc3.restype = ctypes.c_int
    L.fp_rates3.argtypes = L.fp_rates4_channels.argtypes
    L.fp_rates3.restype = ctypes.c_int
    L.fp_kappa_rta.argtypes = [vp, ctypes.c_int, dp, dp, dp]
    L.fp_kappa_rta.restype = ctypes.c_int
    L.fp_rates4_nu.argtypes = L.fp_rates4_channels.argtypes
    L.fp_rates4_nu.restype = ctypes.c_int
    ip = ctypes.POINTER(ctypes.c_int)
    L.fp_star_table.argtypes = [ip, ctypes.c_int, ip, ip, ip]
    L.fp_star_table.restype = ctypes.c_int
    L.fp_rates4_irreducible.argtypes = [vp, ctypes.c_int, ip, ctypes.c_int, dp, ctypes.c_double,
                                        ctypes.POINTER(fp_rates_opts), dp, ctypes.POINTER(fp_stats), ip]
    L.fp_rates4_irreducible.restype = ctypes.c_int
    L.fp_rates4_device.restype = ctypes.c_int
    L.fp_rates4_noalloc.argtypes = [vp, ctypes.c_int, dp, ctypes.c_double, ctypes.POINTER(fp_rates_opts), vp,
                                    ctypes.POINTER(fp_stats)]
    L.fp_rates4_noalloc.restype = ctypes.c_int
    L.fp_autotune.argtypes = [vp, ctypes.c_int, dp, ctypes.c_double, ctypes.POINTER(fp_rates_opts), dp]
    L.fp_autotune.restype = ctypes.c_int
    L.fp_phase3.argtypes = [vp, ctypes.c_int, dp, ctypes.c_double, ctypes.POINTER(fp_rates_opts), dp, dp]
    L.fp_phase3.restype = ctypes.c_int
    L.fp_phase4.argtypes = [vp, ctypes.c_int, dp, ctypes.c_double, ctypes.c_int, dp]
    L.fp_phase4.restype = ctypes.c_int
    L.fp_mlp_params_size.argtypes = [ctypes.c_int]
    L.fp_mlp_params_size.restype = ctypes.c_int
    fpp = ctypes.POINTER(ctypes.c_float)
    L.fp_mlp_loss_grad.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, fpp, fpp, fpp, fpp, fpp]
    L.fp_mlp_loss_grad.restype = ctypes.c_int
    L.fp_surrogate_default_opts.argtypes = [ctypes.POINTER(fp_surrogate_opts)]
    L.fp_surrogate_default_opts.restype = None
    L.fp_surrogate_fit.argtypes = [vp, ctypes.c_int, dp, ctypes.c_double, ctypes.POINTER(fp_surrogate_opts),
                                   ctypes.POINTER(fp_surrogate_report)]
    L.fp_surrogate_fit.restype = ctypes.c_int
    L.fp_surrogate_rates.argtypes = [vp, dp, ctypes.POINTER(ctypes.c_ubyte)]
    L.fp_surrogate_sweep.argtypes = [vp, ctypes.c_int, dp, ctypes.c_int, dp, ctypes.c_double,
                                     ctypes.POINTER(fp_surrogate_opts), dp, ctypes.POINTER(ctypes.c_ubyte),
                                     ctypes.POINTER(fp_surrogate_report)]
    L.fp_surrogate_sweep.restype = ctypes.c_int
    L.fp_surrogate_rates.restype = ctypes.c_int
    L.fp_phase_space4.argtypes = [vp, ctypes.c_int, dp, ctypes.c_double, ctypes.POINTER(fp_rates_opts), ctypes.c_int,
                                  dp, dp, dp]
    L.fp_phase_space4.restype = ctypes.c_int
    cp = ctypes.c_char_p
    L.fp_write_fc4.argtypes = [cp, dp, ctypes.c_int, ctypes.POINTER(fp_fc4)]
    L.fp_write_fc4.restype = ctypes.c_int
    L.fp_read_fc4.argtypes = [cp, dp, ctypes.POINTER(fp_fc4), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.fp_read_fc4.restype = ctypes.c_int
    L.fp_write_fc3.argtypes = [cp, dp, ctypes.c_int, ctypes.POINTER(fp_fc3)]
    L.fp_write_fc3.restype = ctypes.c_int
    L.fp_read_fc3.argtypes = [cp, dp, ctypes.POINTER(fp_fc3), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.fp_read_fc3.restype = ctypes.c_int
    L.fp_free.argtypes = [vp]
    L.fp_free.restype = None
    L.fp_last_error.argtypes = [vp]
    L.fp_last_error.restype = ctypes.c_char_p
    _LIB = L
    return L


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(L, ctx, rc):
    if rc != FP_OK:
        msg = L.fp_last_error(ctx)
        raise FourPhononError(rc, msg.decode() if msg else "")


def pack_fc2(idx, val):
    arr = (fp_fc2 * max(1, len(idx)))()
    for b, (ix, v) in enumerate(zip(idx, val)):
        arr[b].i, arr[b].j = int(ix[0]), int(ix[1])
        for d in range(3):
            arr[b].Rj[d] = int(ix[2 + d])
        ctypes.memmove(arr[b].fc, np.ascontiguousarray(v, np.float64).ctypes.data, 72)
    return arr


def pack_fc3(idx, val):
    arr = (fp_fc3 * max(1, len(idx)))()
    for b, (ix, v) in enumerate(zip(idx, val)):
        arr[b].i, arr[b].j, arr[b].k = (int(x) for x in ix[:3])
        for d in range(3):
            arr[b].Rj[d] = int(ix[3 + d])
            arr[b].Rk[d] = int(ix[6 + d])
        ctypes.memmove(arr[b].fc, np.ascontiguousarray(v, np.float64).ctypes.data, 216)
    return arr


def pack_fc4(idx, val):
    arr = (fp_fc4 * max(1, len(idx)))()
    for b, (ix, v) in enumerate(zip(idx, val)):
        arr[b].i, arr[b].j, arr[b].k, arr[b].l = (int(x) for x in ix[:4])
        for d in range(3):
            arr[b].Rj[d] = int(ix[4 + d])
            arr[b].Rk[d] = int(ix[7 + d])
            arr[b].Rl[d] = int(ix[10 + d])
        ctypes.memmove(arr[b].fc, np.ascontiguousarray(v, np.float64).ctypes.data, 648)
    return arr


class Context:
    """One fp_ctx: a crystal, its q-grid and its device memory."""

    def __init__(self, lattice, frac, mass, fc2_idx, fc2_val, fc4_idx, fc4_val, grid, device=0):
        self.L = load()
        self.nb = 3 * len(mass)
        self.grid = tuple(int(g) for g in grid)
        self.N = int(np.prod(self.grid))
        lat = np.ascontiguousarray(lattice, np.float64).reshape(9)
        fr = np.ascontiguousarray(frac, np.float64).reshape(-1)
        m = np.ascontiguousarray(mass, np.float64)
        g = (ctypes.c_int * 3)(*self.grid)
        f2 = pack_fc2(fc2_idx, fc2_val)
        f4 = pack_fc4(fc4_idx, fc4_val)
        h = ctypes.c_void_p()
        rc = self.L.fp_init(ctypes.byref(h), _dp(lat), len(m), _dp(fr), _dp(m), len(fc2_idx), f2, len(fc4_idx), f4,
                            g, int(device))
        _check(self.L, None, rc)
        self.h = h

    @classmethod
    def from_crystal(cls, cr, device=0):
        ctx = cls(cr.lattice, cr.frac, cr.mass, cr.fc2_idx, cr.fc2_val, cr.fc4_idx, cr.fc4_val, cr.grid, device)
        if getattr(cr, "fc3_idx", None) is not None:
            ctx.set_fc3(cr.fc3_idx, cr.fc3_val)
        return ctx

    def set_fc3(self, idx, val):
        """fp_set_fc3: triplets idx (n3, 9) = i, j, k, Rj[3], Rk[3] and values (n3, 27) in eV/A^3."""
        idx = np.asarray(idx)
        _check(self.L, self.h, self.L.fp_set_fc3(self.h, len(idx), pack_fc3(idx, np.asarray(val, np.float64))))

    def phase_space4(self, temps, scalebroad=1.0, stride=1, **opts):
        """fp_phase_space4: (numprocess (N*nb), p4 (N*nb), wp4 (nT, N*nb)), the onlyharmonic outputs."""
        T = np.ascontiguousarray(temps, np.float64).reshape(-1)
        o, keep = self.make_opts(**opts)
        npr = np.zeros(self.N * self.nb)
        p4 = np.zeros(self.N * self.nb)
        wp4 = np.zeros((len(T), self.N * self.nb))
        _check(self.L, self.h, self.L.fp_phase_space4(self.h, len(T), _dp(T), float(scalebroad), ctypes.byref(o),
                                                      int(stride), _dp(npr), _dp(p4), _dp(wp4)))
        del keep
        return npr, p4, wp4

    def kappa_rta(self, temps, rates):
        """fp_kappa_rta: kappa (nT, 3, 3) in W/(m K) from rates (nT, N, nb) in ps^-1."""
        T = np.ascontiguousarray(temps, np.float64).reshape(-1)
        r = np.ascontiguousarray(rates, np.float64).reshape(len(T), -1)
        k = np.zeros((len(T), 3, 3))
        _check(self.L, self.h, self.L.fp_kappa_rta(self.h, len(T), _dp(T), _dp(r), _dp(k)))
        return k

    def rates3(self, temps, scalebroad=1.0, **opts):
        """fp_rates3: three-phonon rates (nT, N, nb) and stats."""
        T = np.ascontiguousarray(temps, np.float64).reshape(-1)
        o, keep = self.make_opts(**opts)
        out = np.zeros((len(T), self.N, self.nb))
        st = fp_stats()
        rc = self.L.fp_rates3(self.h, len(T), _dp(T), float(scalebroad), ctypes.byref(o), _dp(out), ctypes.byref(st))
        _check(self.L, self.h, rc)
        del keep
        return out, st.as_dict()

    def close(self):
        if getattr(self, "h", None):
            self.L.fp_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_stream(self, stream_handle: int | None):
        _check(self.L, self.h, self.L.fp_set_stream(self.h, ctypes.c_void_p(stream_handle or 0)))

    def modes(self, copy=True):
        if not copy:
            _check(self.L, self.h, self.L.fp_modes(self.h, None, None, None))
            return None
        om = np.zeros((self.N, self.nb))
        ev = np.zeros((self.N, self.nb, self.nb, 2))
        ve = np.zeros((self.N, self.nb, 3))
        rc = self.L.fp_modes(self.h, om.ctypes.data, ev.ctypes.data, ve.ctypes.data)
        _check(self.L, self.h, rc)
        return om, ev[..., 0] + 1j * ev[..., 1], ve

    def set_modes(self, omega, evec, vel):
        om = np.ascontiguousarray(omega, np.float64)
        if np.iscomplexobj(evec):
            ev = np.ascontiguousarray(np.stack([evec.real, evec.imag], axis=-1))
        else:
            ev = np.ascontiguousarray(evec, np.float64)
        ve = np.ascontiguousarray(vel, np.float64)
        _check(self.L, self.h, self.L.fp_set_modes(self.h, _dp(om), _dp(ev), _dp(ve)))

    @staticmethod
    def make_opts(precision=FP_PREC_FP64, window=2.0, sigma_min=1e-10, dq_mode=0, mode_mask=None, q_begin=0,
                  q_end=0, block_j0=0, k1_tile=0, threads=0, no_graph=0, process_mask=0, nu_select=0,
                  no_time_reversal=0, tensor_cores=0):
        o = fp_rates_opts()
        o.precision, o.window, o.sigma_min, o.dq_mode = int(precision), float(window), float(sigma_min), int(dq_mode)
        o.q_begin, o.q_end, o.block_j0, o.k1_tile, o.threads = int(q_begin), int(q_end), int(block_j0), \
            int(k1_tile), int(threads)
        o.no_graph = int(no_graph)
        o.process_mask = int(process_mask)
        o.nu_select = int(nu_select)
        o.no_time_reversal = int(no_time_reversal)
        o.tensor_cores = int(tensor_cores)
        keep = None
        if mode_mask is not None:
            keep = np.ascontiguousarray(mode_mask, np.uint8)
            o.mode_mask = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))
        return o, keep

    def rates4(self, temps, scalebroad=1.0, **opts):
        T = np.ascontiguousarray(temps, np.float64).reshape(-1)
        o, keep = self.make_opts(**opts)
        out = np.zeros((len(T), self.N, self.nb))
        st = fp_stats()
        rc = self.L.fp_rates4(self.h, len(T), _dp(T), float(scalebroad), ctypes.byref(o), _dp(out), ctypes.byref(st))
        _check(self.L, self.h, rc)
        del keep
        return out, st.as_dict()

    def rates4_irreducible(self, ops, temps, scalebroad=1.0, **opts):
        """fp_rates4_irreducible: rates (nT, N, nb) from one q per star of the integer point-group ops
        (nops, 3, 3) on reciprocal fractional coordinates; returns (rates, stats, number of stars)."""
        R = np.ascontiguousarray(ops, np.int32).reshape(-1, 9)
        T = np.ascontiguousarray(temps, np.float64).reshape(-1)
        o, keep = self.make_opts(**opts)
        out = np.zeros((len(T), self.N, self.nb))
        st = fp_stats()
        nirr = ctypes.c_int(0)
        rc = self.L.fp_rates4_irreducible(self.h, len(R), R.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), len(T),
                                          _dp(T), float(scalebroad), ctypes.byref(o), _dp(out), ctypes.byref(st),
                                          ctypes.byref(nirr))
        _check(self.L, self.h, rc)
        del keep
        return out, st.as_dict(), nirr.value

    def rates4_nu(self, temps, scalebroad=1.0, **opts):
        """fp_rates4_nu: rates (nT, 2, N, nb) of normal and Umklapp processes."""
        T = np.ascontiguousarray(temps, np.float64).reshape(-1)
        o, keep = self.make_opts(**opts)
        out = np.zeros((len(T), 2, self.N, self.nb))
        st = fp_stats()
        rc = self.L.fp_rates4_nu(self.h, len(T), _dp(T), float(scalebroad), ctypes.byref(o), _dp(out), ctypes.byref(st))
        _check(self.L, self.h, rc)
        del keep
        return out, st.as_dict()

    def rates4_channels(self, temps, scalebroad=1.0, **opts):
        """fp_rates4_channels: rates (nT, 3, N, nb) of the ++, +- and -- processes."""
        T = np.ascontiguousarray(temps, np.float64).reshape(-1)
        o, keep = self.make_opts(**opts)
        out = np.zeros((len(T), 3, self.N, self.nb))
        st = fp_stats()
        rc = self.L.fp_rates4_channels(self.h, len(T), _dp(T), float(scalebroad), ctypes.byref(o), _dp(out),
                                       ctypes.byref(st))
        _check(self.L, self.h, rc)
        del keep
        return out, st.as_dict()

    def rates4_device(self, temps, d_rates_ptr: int, scalebroad=1.0, **opts):
        T = np.ascontiguousarray(temps, np.float64).reshape(-1)
        o, keep = self.make_opts(**opts)
        st = fp_stats()
        rc = self.L.fp_rates4_device(self.h, len(T), _dp(T), float(scalebroad), ctypes.byref(o),
                                     ctypes.c_void_p(d_rates_ptr), ctypes.byref(st))
        _check(self.L, self.h, rc)
        del keep
        return st.as_dict()

    def autotune(self, temps, scalebroad=1.0, **opts):
        """Tile autotuning (fp_autotune); returns (tiles dict, best ms) and remembers the tiles in the context."""
        T = np.ascontiguousarray(temps, np.float64).reshape(-1)
        o, keep = self.make_opts(**opts)
        best = ctypes.c_double(0.0)
        _check(self.L, self.h, self.L.fp_autotune(self.h, len(T), _dp(T), float(scalebroad), ctypes.byref(o),
                                                  ctypes.byref(best)))
        del keep
        return {"block_j0": o.block_j0, "k1_tile": o.k1_tile, "threads": o.threads}, best.value

    def phase3(self, temps, scalebroad=1.0, **opts):
        """Three-phonon-like phase space (fp_phase3): p3 (N*nb), wp3 (nT, N*nb)."""
        T = np.ascontiguousarray(temps, np.float64).reshape(-1)
        o, keep = self.make_opts(**opts)
        p3 = np.zeros(self.N * self.nb)
        wp3 = np.zeros((len(T), self.N * self.nb))
        _check(self.L, self.h, self.L.fp_phase3(self.h, len(T), _dp(T), float(scalebroad), ctypes.byref(o),
                                                _dp(p3), _dp(wp3)))
        del keep
        return p3, wp3

    def phase4(self, temps, scalebroad=1.0, stride=1):
        """Four-phonon weighted phase space (fp_phase4), (nT, N*nb)."""
        T = np.ascontiguousarray(temps, np.float64).reshape(-1)
        wp4 = np.zeros((len(T), self.N * self.nb))
        _check(self.L, self.h, self.L.fp_phase4(self.h, len(T), _dp(T), float(scalebroad), int(stride), _dp(wp4)))
        return wp4

    def surrogate_fit(self, temps, scalebroad=1.0, **sopts):
        """Learned rates (fp_surrogate_fit); returns the report as a dict."""
        T = np.ascontiguousarray(temps, np.float64).reshape(-1)
        so = fp_surrogate_opts()
        self.L.fp_surrogate_default_opts(ctypes.byref(so))
        for k, v in sopts.items():
            setattr(so, k, v)
        rep = fp_surrogate_report()
        _check(self.L, self.h, self.L.fp_surrogate_fit(self.h, len(T), _dp(T), float(scalebroad), ctypes.byref(so),
                                                       ctypes.byref(rep)))
        self._sur_nT = len(T)
        return rep.as_dict()

    def surrogate_sweep(self, anchors, temps, scalebroad=1.0, **sopts):
        """Learned rates at new temperatures (fp_surrogate_sweep): (rates (nT, N, nb), used_exact (nT, N, nb),
        report dict) from exact rates at the anchor temperatures and on a seeded subset at `temps`."""
        A = np.ascontiguousarray(anchors, np.float64).reshape(-1)
        T = np.ascontiguousarray(temps, np.float64).reshape(-1)
        so = fp_surrogate_opts()
        self.L.fp_surrogate_default_opts(ctypes.byref(so))
        for k, v in sopts.items():
            setattr(so, k, v)
        rep = fp_surrogate_report()
        r = np.zeros((len(T), self.N, self.nb))
        u = np.zeros((len(T), self.N, self.nb), np.uint8)
        _check(self.L, self.h, self.L.fp_surrogate_sweep(self.h, len(A), _dp(A), len(T), _dp(T), float(scalebroad),
                                                         ctypes.byref(so), _dp(r),
                                                         u.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)),
                                                         ctypes.byref(rep)))
        return r, u, rep.as_dict()

    def surrogate_rates(self):
        """Rates of the last surrogate fit (nT, N, nb) and the exact-evaluation flags (same shape)."""
        nT = self._sur_nT
        r = np.zeros((nT, self.N, self.nb))
        u = np.zeros((nT, self.N, self.nb), np.uint8)
        _check(self.L, self.h, self.L.fp_surrogate_rates(self.h, _dp(r),
                                                         u.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))))
        return r, u


def mlp_loss_grad(X, y, params, device=0):
    """Loss and gradient of the surrogate network on one batch (fp_mlp_loss_grad, FP32 kernels)."""
    L = load()
    X = np.ascontiguousarray(X, np.float32)
    y = np.ascontiguousarray(y, np.float32)
    p = np.ascontiguousarray(params, np.float32)
    B, F = X.shape
    if L.fp_mlp_params_size(F) != p.size:
        raise ValueError("parameter vector has the wrong size")
    g = np.zeros_like(p)
    loss = np.zeros(1, np.float32)
    fpp = ctypes.POINTER(ctypes.c_float)
    rc = L.fp_mlp_loss_grad(int(device), F, B, X.ctypes.data_as(fpp), y.ctypes.data_as(fpp), p.ctypes.data_as(fpp),
                            g.ctypes.data_as(fpp), loss.ctypes.data_as(fpp))
    if rc != FP_OK:
        raise FourPhononError(rc, "fp_mlp_loss_grad failed")
    return float(loss[0]), g


def star_table(grid, ops):
    """fp_star_table (host only): (rep (N,), number of stars) for the integer ops (nops, 3, 3)."""
    L = load()
    g = np.ascontiguousarray(grid, np.int32).reshape(3)
    R = np.ascontiguousarray(ops, np.int32).reshape(-1, 9)
    rep = np.zeros(int(np.prod(g)), np.int32)
    n = ctypes.c_int(0)
    ip = ctypes.POINTER(ctypes.c_int)
    rc = L.fp_star_table(g.ctypes.data_as(ip), len(R), R.ctypes.data_as(ip), rep.ctypes.data_as(ip), ctypes.byref(n))
    if rc != FP_OK:
        raise FourPhononError(rc, "fp_star_table rejected the operations")
    return rep, n.value


def _lat(lattice):
    return np.ascontiguousarray(lattice, np.float64).reshape(9)


def write_fc4(path, lattice, idx, val):
    """fp_write_fc4: quartets idx (n, 13) = i, j, k, l, Rj[3], Rk[3], Rl[3] (0-based atoms), val (n, 81) eV/A^4."""
    L = load()
    lat = _lat(lattice)
    _check(L, None, L.fp_write_fc4(os.fsencode(path), _dp(lat), len(idx), pack_fc4(idx, val)))


def read_fc4(path, lattice):
    """fp_read_fc4: (idx (n, 13) int32, val (n, 81)) in the layout of write_fc4."""
    L = load()
    lat = _lat(lattice)
    n = ctypes.c_int(0)
    _check(L, None, L.fp_read_fc4(os.fsencode(path), _dp(lat), None, 0, ctypes.byref(n)))
    arr = (fp_fc4 * max(1, n.value))()
    _check(L, None, L.fp_read_fc4(os.fsencode(path), _dp(lat), arr, n.value, ctypes.byref(n)))
    idx = np.array([[a.i, a.j, a.k, a.l, *a.Rj, *a.Rk, *a.Rl] for a in arr[:n.value]], np.int32).reshape(-1, 13)
    val = np.array([list(a.fc) for a in arr[:n.value]], np.float64).reshape(-1, 81)
    return idx, val


def write_fc3(path, lattice, idx, val):
    """fp_write_fc3: triplets idx (n, 9) = i, j, k, Rj[3], Rk[3] (0-based atoms), val (n, 27) eV/A^3."""
    L = load()
    lat = _lat(lattice)
    _check(L, None, L.fp_write_fc3(os.fsencode(path), _dp(lat), len(idx), pack_fc3(idx, val)))


def read_fc3(path, lattice):
    """fp_read_fc3: (idx (n, 9) int32, val (n, 27)) in the layout of write_fc3."""
    L = load()
    lat = _lat(lattice)
    n = ctypes.c_int(0)
    _check(L, None, L.fp_read_fc3(os.fsencode(path), _dp(lat), None, 0, ctypes.byref(n)))
    arr = (fp_fc3 * max(1, n.value))()
    _check(L, None, L.fp_read_fc3(os.fsencode(path), _dp(lat), arr, n.value, ctypes.byref(n)))
    idx = np.array([[a.i, a.j, a.k, *a.Rj, *a.Rk] for a in arr[:n.value]], np.int32).reshape(-1, 9)
    val = np.array([list(a.fc) for a in arr[:n.value]], np.float64).reshape(-1, 27)
    return idx, val
