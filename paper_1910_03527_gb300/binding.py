"""Python binding of the C ABI in include/mbe.h (argument marshalling only).

Every computation runs in the CUDA kernels of libmbe_gb300.so.  This module
only checks tensor placement, dtype and contiguity, passes raw pointers and
sizes through ctypes, and allocates output tensors with PyTorch on the
context's device.  There is no CPU fallback: without the library or a CUDA
device every call raises.
"""

from __future__ import annotations

import ctypes
import functools
import os
from dataclasses import dataclass
from typing import List, Optional, Sequence

import torch

from . import _build

MBE_OK = 0
MBE_PREC_FP64 = 0
MBE_PREC_MIXED = 1
MBE_SKIP_NO_OCC_OR_VIRT = 1
MBE_MAX_CAS = 12
MBE_MAX_LARGE_CAS = 16
STATUS_NAMES = {0: "OK", 1: "MAXITER", 2: "NONFINITE", 3: "BADINPUT", 4: "DEGENERATE"}

EXPORTS = ("mbe_default_opts", "mbe_ctx_create", "mbe_ctx_set_stream", "mbe_ctx_destroy",
           "mbe_last_error", "mbe_ctx_sync", "mbe_ctx_launches", "mbe_ctx_set_timing",
           "mbe_ctx_timings", "mbe_tuples", "mbe_string_table", "mbe_phi_energy",
           "casci_batch", "casci_sigma", "casci_sigma_noalloc", "mbe_increments", "mbe_total",
           "mbe_weights", "casci_rdm_batch", "mbe_phi_gradient", "casci_sigma_large", "casci_solve",
           "mbe_screen", "casci_batch_routed", "mbe_fma_peak", "mbe_ctx_set_tuning", "mbe_ctx_get_tuning",
           "mbe_autotune")


class MbeOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("tol", ctypes.c_double),
                ("tol_switch", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("fp64_final_iters", ctypes.c_int), ("sectors", ctypes.c_int),
                ("s2_penalty", ctypes.c_double)]


class MbeTiming(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int), ("solver", ctypes.c_int), ("dpl", ctypes.c_int),
                ("ms", ctypes.c_float)]


class MbeTuning(ctypes.Structure):
    _fields_ = [("warp_max_ndet", ctypes.c_int), ("warp_warps", ctypes.c_int), ("block_basis", ctypes.c_int)]


class MbeTuneRecord(ctypes.Structure):
    _fields_ = [("tuning", MbeTuning), ("ms", ctypes.c_float)]


class MbeError(RuntimeError):
    pass


def library_path() -> str:
    return _build.LIB


@functools.lru_cache(maxsize=1)
def lib() -> ctypes.CDLL:
    """Load libmbe_gb300.so (it must have been built: __graft_entry__.build())."""
    path = library_path()
    if not os.path.exists(path):
        raise MbeError(f"{path} is missing; build it first (python -c 'import __graft_entry__ as g; "
                       "g.build()')")
    L = ctypes.CDLL(path)
    P, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    L.mbe_default_opts.restype = None
    L.mbe_default_opts.argtypes = [ctypes.POINTER(MbeOpts)]
    L.mbe_ctx_create.restype = i32
    L.mbe_ctx_create.argtypes = [ctypes.POINTER(P), i32, P]
    L.mbe_ctx_set_stream.restype = i32
    L.mbe_ctx_set_stream.argtypes = [P, P]
    L.mbe_ctx_destroy.restype = None
    L.mbe_ctx_destroy.argtypes = [P]
    L.mbe_last_error.restype = ctypes.c_char_p
    L.mbe_last_error.argtypes = []
    L.mbe_ctx_sync.restype = i32
    L.mbe_ctx_sync.argtypes = [P]
    L.mbe_ctx_launches.restype = i32
    L.mbe_ctx_launches.argtypes = [P, ctypes.POINTER(i64)]
    L.mbe_ctx_set_timing.restype = i32
    L.mbe_ctx_set_timing.argtypes = [P, i32]
    L.mbe_ctx_timings.restype = i32
    L.mbe_ctx_timings.argtypes = [P, i32, ctypes.POINTER(MbeTiming), ctypes.POINTER(i32)]
    L.mbe_tuples.restype = i32
    L.mbe_tuples.argtypes = [P, i32, P, i32, P, i32, P, i32, i32, ctypes.POINTER(i64), P]
    L.mbe_string_table.restype = i32
    L.mbe_string_table.argtypes = [P, i32, i32, P, P]
    L.mbe_phi_energy.restype = i32
    L.mbe_phi_energy.argtypes = [P, i32, P, P, P, P]
    L.casci_batch.restype = i32
    L.casci_batch.argtypes = [P, i32, P, P, P, i32, P, dbl, i32, i64, P, ctypes.POINTER(MbeOpts),
                              P, P, P]
    L.casci_sigma.restype = i32
    L.casci_sigma.argtypes = [P, i32, P, P, P, i32, P, P, P, P]
    L.casci_sigma_noalloc.restype = i32
    L.casci_sigma_noalloc.argtypes = [i32, P, i32, P, P, P, i32, P, i32, P, P, P]
    L.mbe_increments.restype = i32
    L.mbe_increments.argtypes = [P, i32, i64, P, P, i32, P, P, P, P]
    L.mbe_total.restype = i32
    L.mbe_total.argtypes = [P, i32, P, P, P, dbl, P, P]
    L.mbe_weights.restype = i32
    L.mbe_weights.argtypes = [P, i32, P, P, i32, P, dbl, P, P]
    L.casci_rdm_batch.restype = i32
    L.casci_rdm_batch.argtypes = [P, i32, P, P, P, i32, P, i32, i64, P, ctypes.POINTER(MbeOpts), P, P, P, P]
    L.mbe_phi_gradient.restype = i32
    L.mbe_phi_gradient.argtypes = [P, i32, P, dbl, P, P]
    L.casci_sigma_large.restype = i32
    L.casci_sigma_large.argtypes = [P, i32, P, P, P, i32, P, i32, P, P, P]
    L.casci_solve.restype = i32
    L.casci_solve.argtypes = [P, i32, P, P, P, i32, P, ctypes.POINTER(MbeOpts), P, P, P]
    L.casci_batch_routed.restype = i32
    L.casci_batch_routed.argtypes = [P, i32, P, P, P, i32, P, dbl, i32, i64, P, ctypes.POINTER(MbeOpts), i64,
                                     P, P, P]
    L.mbe_ctx_set_tuning.restype = i32
    L.mbe_ctx_set_tuning.argtypes = [P, i32, i32, ctypes.POINTER(MbeTuning)]
    L.mbe_ctx_get_tuning.restype = i32
    L.mbe_ctx_get_tuning.argtypes = [P, i32, i32, ctypes.POINTER(MbeTuning)]
    L.mbe_autotune.restype = i32
    L.mbe_autotune.argtypes = [P, i32, P, P, P, i32, P, dbl, i32, i64, P, ctypes.POINTER(MbeOpts),
                               ctypes.POINTER(MbeTuning), ctypes.POINTER(MbeTuneRecord), i32, ctypes.POINTER(i32)]
    L.mbe_fma_peak.restype = i32
    L.mbe_fma_peak.argtypes = [P, i32, i32, ctypes.POINTER(dbl)]
    L.mbe_screen.restype = i32
    L.mbe_screen.argtypes = [P, i32, P, i32, P, i32, P, i32, i64, P, P, dbl, i32, dbl, i32, i64,
                             ctypes.POINTER(i64), P]
    return L


def _check(rc: int, what: str) -> None:
    if rc != MBE_OK:
        msg = lib().mbe_last_error().decode(errors="replace")
        raise MbeError(f"{what} failed ({rc}): {msg}")


def _i32_host(values: Sequence[int]):
    arr = (ctypes.c_int32 * max(len(values), 1))(*[int(v) for v in values])
    return arr


def _u8_host(values: Sequence[int]):
    return (ctypes.c_uint8 * max(len(values), 1))(*[int(v) for v in values])


@dataclass
class Opts:
    """Davidson options of casci_batch (see mbe_opts in include/mbe.h)."""

    precision: str = "fp64"  # "fp64" or "mixed"
    tol: float = 1e-7
    tol_switch: float = 1e-5
    max_iter: int = 2000
    fp64_final_iters: int = 2
    even_only: bool = False  # only the even sector of the alpha-beta string exchange
    s2_penalty: float = 0.0  # mu of H + mu S^2 (state targeting by total spin; 0: off)

    def to_c(self) -> MbeOpts:
        o = MbeOpts()
        o.precision = {"fp64": MBE_PREC_FP64, "mixed": MBE_PREC_MIXED}[self.precision]
        o.tol = self.tol
        o.tol_switch = self.tol_switch
        o.max_iter = self.max_iter
        o.fp64_final_iters = self.fp64_final_iters
        o.sectors = 1 if self.even_only else 0
        o.s2_penalty = self.s2_penalty
        return o


class Context:
    """An mbe_ctx bound to one CUDA device; work is issued on `stream`."""

    def __init__(self, device: int = 0, stream: Optional[torch.cuda.Stream] = None):
        if not torch.cuda.is_available():
            raise MbeError("no CUDA device: the MBE-FCI engine has no CPU path")
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        _check(lib().mbe_ctx_create(ctypes.byref(h), device, ctypes.c_void_p(self.stream.cuda_stream)),
               "mbe_ctx_create")
        self._h = h

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().mbe_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream: torch.cuda.Stream) -> None:
        self.stream = stream
        _check(lib().mbe_ctx_set_stream(self._h, ctypes.c_void_p(stream.cuda_stream)), "mbe_ctx_set_stream")

    def sync(self) -> None:
        _check(lib().mbe_ctx_sync(self._h), "mbe_ctx_sync")

    def launches(self) -> int:
        """Kernels launched by this context so far."""
        n = ctypes.c_int64()
        _check(lib().mbe_ctx_launches(self._h, ctypes.byref(n)), "mbe_ctx_launches")
        return n.value

    def set_timing(self, enable: bool) -> None:
        _check(lib().mbe_ctx_set_timing(self._h, 1 if enable else 0), "mbe_ctx_set_timing")

    def take_timings(self, max_records: int = 4096):
        """[(order, solver, dpl, ms)] of the timed solver launches since the last read."""
        buf = (MbeTiming * max_records)()
        cnt = ctypes.c_int()
        _check(lib().mbe_ctx_timings(self._h, max_records, buf, ctypes.byref(cnt)), "mbe_ctx_timings")
        return [(buf[i].order, buf[i].solver, buf[i].dpl, buf[i].ms) for i in range(min(cnt.value,
                                                                                       max_records))]

    def fma_peak(self, kind: str, reps: int = 5) -> float:
        """Measured fused multiply-add throughput (TFLOP/s) of the float64 or float32 pipe."""
        out = ctypes.c_double()
        _check(lib().mbe_fma_peak(self._h, {"fp64": 0, "fp32": 1}[kind], int(reps), ctypes.byref(out)),
               "mbe_fma_peak")
        return out.value

    @staticmethod
    def _tuning_dict(t: MbeTuning) -> dict:
        return dict(warp_max_ndet=t.warp_max_ndet, warp_warps=t.warp_warps, block_basis=t.block_basis)

    def set_tuning(self, precision: str, n_cas: int, warp_max_ndet: int, warp_warps: int, block_basis: int) -> None:
        """Launch choices of later casci_batch calls (n_cas 0: every active-space size)."""
        t = MbeTuning(warp_max_ndet, warp_warps, block_basis)
        _check(lib().mbe_ctx_set_tuning(self._h, {"fp64": MBE_PREC_FP64, "mixed": MBE_PREC_MIXED}[precision],
                                        int(n_cas), ctypes.byref(t)), "mbe_ctx_set_tuning")

    def get_tuning(self, precision: str, n_cas: int) -> dict:
        t = MbeTuning()
        _check(lib().mbe_ctx_get_tuning(self._h, {"fp64": MBE_PREC_FP64, "mixed": MBE_PREC_MIXED}[precision],
                                        int(n_cas), ctypes.byref(t)), "mbe_ctx_get_tuning")
        return self._tuning_dict(t)

    def autotune(self, h1, eri, occ, ref: Sequence[int], e_ref_corr: float, order: int, tuples: torch.Tensor,
                 opts: Optional[Opts] = None):
        """mbe_autotune on `tuples`: the chosen tuning (set on the context for this
        precision and |R| + order) and the timed candidates [(tuning, ms)]."""
        norb = h1.shape[0]
        self._dev(tuples, torch.int32, "tuples")
        o = (opts or Opts()).to_c()
        best = MbeTuning()
        recs = (MbeTuneRecord * 16)()
        nrec = ctypes.c_int()
        _check(lib().mbe_autotune(self._h, norb, self._p(self._dev(h1, torch.float64, "h1")),
                                  self._p(self._dev(eri, torch.float64, "eri")),
                                  self._p(self._dev(occ, torch.uint8, "occ")), len(ref), _i32_host(ref),
                                  float(e_ref_corr), order, int(tuples.shape[0]), self._p(tuples), ctypes.byref(o),
                                  ctypes.byref(best), recs, 16, ctypes.byref(nrec)), "mbe_autotune")
        return (self._tuning_dict(best),
                [(self._tuning_dict(recs[i].tuning), recs[i].ms) for i in range(min(nrec.value, 16))])

    # ---------------------------------------------------------------- helpers
    def _dev(self, t: torch.Tensor, dtype: torch.dtype, name: str) -> torch.Tensor:
        if not isinstance(t, torch.Tensor) or t.device != self.device or t.dtype != dtype:
            raise MbeError(f"{name}: expected a {dtype} tensor on {self.device}")
        if not t.is_contiguous():
            raise MbeError(f"{name}: must be contiguous")
        return t

    @staticmethod
    def _p(t: Optional[torch.Tensor]):
        return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else None

    def _empty(self, shape, dtype):
        return torch.empty(shape, dtype=dtype, device=self.device)

    # ---------------------------------------------------------------- ABI calls
    def mbe_tuples(self, norb: int, occ: Sequence[int], exp: Sequence[int], ref: Sequence[int],
                   order: int, skip: bool) -> torch.Tensor:
        n = ctypes.c_int64()
        flags = MBE_SKIP_NO_OCC_OR_VIRT if skip else 0
        occ_h, exp_h, ref_h = _u8_host(occ), _i32_host(exp), _i32_host(ref)
        _check(lib().mbe_tuples(self._h, norb, occ_h, len(exp), exp_h, len(ref), ref_h, order, flags,
                                ctypes.byref(n), None), "mbe_tuples(count)")
        out = self._empty((n.value, order), torch.int32)
        if n.value > 0:
            _check(lib().mbe_tuples(self._h, norb, occ_h, len(exp), exp_h, len(ref), ref_h, order,
                                    flags, ctypes.byref(n), self._p(out)), "mbe_tuples")
        return out

    def mbe_screen(self, norb: int, occ: Sequence[int], exp: Sequence[int], ref: Sequence[int], order: int,
                   parents: torch.Tensor, parent_incs: torch.Tensor, t_init: float, m_init: int, a: float,
                   skip: bool) -> torch.Tensor:
        """Order-(order+1) children spawned from the order-`order` tuples and increments."""
        n = ctypes.c_int64()
        flags = MBE_SKIP_NO_OCC_OR_VIRT if skip else 0
        occ_h, exp_h, ref_h = _u8_host(occ), _i32_host(exp), _i32_host(ref)
        n_par = int(parents.shape[0])
        args = (self._h, norb, occ_h, len(exp), exp_h, len(ref), ref_h, order, n_par,
                self._p(self._dev(parents, torch.int32, "parents")),
                self._p(self._dev(parent_incs, torch.float64, "parent increments")),
                float(t_init), int(m_init), float(a), flags)
        _check(lib().mbe_screen(*args, 0, ctypes.byref(n), None), "mbe_screen(count)")
        out = self._empty((n.value, order + 1), torch.int32)
        if n.value > 0:
            _check(lib().mbe_screen(*args, n.value, ctypes.byref(n), self._p(out)), "mbe_screen")
        return out

    def mbe_string_table(self, n_orb: int, n_el: int):
        import math
        ns = math.comb(n_orb, n_el)
        r = n_el * (n_orb - n_el + 1)
        strings = self._empty((ns,), torch.int32)
        table = self._empty((ns, r), torch.int32)
        _check(lib().mbe_string_table(self._h, n_orb, n_el, self._p(strings), self._p(table)),
               "mbe_string_table")
        return strings, table

    def mbe_phi_energy(self, h1, eri, occ) -> torch.Tensor:
        norb = h1.shape[0]
        out = self._empty((1,), torch.float64)
        _check(lib().mbe_phi_energy(self._h, norb, self._p(self._dev(h1, torch.float64, "h1")),
                                    self._p(self._dev(eri, torch.float64, "eri")),
                                    self._p(self._dev(occ, torch.uint8, "occ")), self._p(out)),
               "mbe_phi_energy")
        return out

    def casci_batch(self, h1, eri, occ, ref: Sequence[int], e_ref_corr: float, order: int,
                    tuples: Optional[torch.Tensor], opts: Optional[Opts] = None, n_tuples=None,
                    out=None):
        norb = h1.shape[0]
        if tuples is not None:
            self._dev(tuples, torch.int32, "tuples")
            n_t = tuples.shape[0] if n_tuples is None else n_tuples
        else:
            n_t = 1 if n_tuples is None else n_tuples
        if out is None:
            eps = self._empty((n_t,), torch.float64)
            status = self._empty((n_t,), torch.int32)
            iters = self._empty((n_t,), torch.int32)
        else:
            eps, status, iters = out
        o = (opts or Opts()).to_c()
        ref_h = _i32_host(ref)
        _check(lib().casci_batch(self._h, norb, self._p(self._dev(h1, torch.float64, "h1")),
                                 self._p(self._dev(eri, torch.float64, "eri")),
                                 self._p(self._dev(occ, torch.uint8, "occ")), len(ref), ref_h,
                                 float(e_ref_corr), order, n_t, self._p(tuples), ctypes.byref(o),
                                 self._p(eps), self._p(status), self._p(iters)), "casci_batch")
        return eps, status, iters

    def casci_batch_routed(self, h1, eri, occ, ref: Sequence[int], e_ref_corr: float, order: int,
                           tuples: Optional[torch.Tensor], opts: Optional[Opts] = None, large_ndet: int = 0):
        """casci_batch for active spaces of up to MBE_MAX_LARGE_CAS orbitals: tuples above
        MBE_MAX_CAS orbitals or above large_ndet determinants (if > 0) are solved one at a
        time with the whole GPU."""
        norb = h1.shape[0]
        if tuples is not None:
            self._dev(tuples, torch.int32, "tuples")
        n_t = tuples.shape[0] if tuples is not None else 1
        eps = self._empty((n_t,), torch.float64)
        status = self._empty((n_t,), torch.int32)
        iters = self._empty((n_t,), torch.int32)
        o = (opts or Opts()).to_c()
        _check(lib().casci_batch_routed(self._h, norb, self._p(self._dev(h1, torch.float64, "h1")),
                                        self._p(self._dev(eri, torch.float64, "eri")),
                                        self._p(self._dev(occ, torch.uint8, "occ")), len(ref), _i32_host(ref),
                                        float(e_ref_corr), order, n_t, self._p(tuples), ctypes.byref(o),
                                        int(large_ndet), self._p(eps), self._p(status), self._p(iters)),
               "casci_batch_routed")
        return eps, status, iters

    def casci_sigma(self, h1, eri, occ, cas: Sequence[int], c: torch.Tensor, want_diag: bool = True):
        norb = h1.shape[0]
        self._dev(c, torch.float64, "c")
        sigma = torch.empty_like(c)
        diag = torch.empty_like(c) if want_diag else None
        cas_h = _i32_host(cas)
        _check(lib().casci_sigma(self._h, norb, self._p(self._dev(h1, torch.float64, "h1")),
                                 self._p(self._dev(eri, torch.float64, "eri")),
                                 self._p(self._dev(occ, torch.uint8, "occ")), len(cas), cas_h,
                                 self._p(c), self._p(sigma), self._p(diag)), "casci_sigma")
        return sigma, diag

    def mbe_increments(self, order: int, tuples: torch.Tensor, eps: torch.Tensor,
                       lower_tuples: List[torch.Tensor], lower_incs: List[torch.Tensor],
                       out: Optional[torch.Tensor] = None) -> torch.Tensor:
        n_t = tuples.shape[0]
        inc = self._empty((n_t,), torch.float64) if out is None else out
        nl = len(lower_tuples)
        counts = (ctypes.c_int64 * max(nl, 1))(*[int(t.shape[0]) for t in lower_tuples])
        tp = (ctypes.c_void_p * max(nl, 1))(*[self._p(t) for t in lower_tuples])
        ip = (ctypes.c_void_p * max(nl, 1))(*[self._p(t) for t in lower_incs])
        for t in lower_tuples:
            self._dev(t, torch.int32, "lower tuples")
        for t in lower_incs:
            self._dev(t, torch.float64, "lower increments")
        _check(lib().mbe_increments(self._h, order, n_t, self._p(self._dev(tuples, torch.int32, "tuples")),
                                    self._p(self._dev(eps, torch.float64, "eps")), nl, counts, tp, ip,
                                    self._p(inc)), "mbe_increments")
        return inc

    def mbe_total(self, incs: List[torch.Tensor], e_phi: Optional[torch.Tensor], e_ref_corr: float,
                  out=None):
        n = len(incs)
        e_order = self._empty((max(n, 1),), torch.float64) if out is None else out[0]
        e_total = self._empty((1,), torch.float64) if out is None else out[1]
        counts = (ctypes.c_int64 * max(n, 1))(*[int(t.shape[0]) for t in incs])
        ip = (ctypes.c_void_p * max(n, 1))(*[self._p(t) for t in incs])
        _check(lib().mbe_total(self._h, n, counts, ip, self._p(e_phi), float(e_ref_corr),
                               self._p(e_order), self._p(e_total)), "mbe_total")
        return e_order[:n], e_total

    def mbe_weights(self, tuples: List[torch.Tensor], exp: Sequence[int], scale: float = 1.0):
        """Adjoint weights scale * w(S) of every tuple of orders 1..len(tuples), and
        scale * w(R), w(R) = 1 - sum_S w(S), of the reference-space CASCI (a device
        tensor of one element), all computed by the library."""
        n = len(tuples)
        out = [self._empty((t.shape[0],), torch.float64) for t in tuples]
        ref_w = self._empty((1,), torch.float64)
        counts = (ctypes.c_int64 * max(n, 1))(*[int(t.shape[0]) for t in tuples])
        tp = (ctypes.c_void_p * max(n, 1))(*[self._p(t) for t in tuples])
        wp = (ctypes.c_void_p * max(n, 1))(*[self._p(t) for t in out])
        for t in tuples:
            self._dev(t, torch.int32, "tuples")
        _check(lib().mbe_weights(self._h, n, counts, tp, len(exp), _i32_host(exp), float(scale), wp,
                                 self._p(ref_w)), "mbe_weights")
        return out, ref_w

    def casci_rdm_batch(self, h1, eri, occ, ref: Sequence[int], order: int, tuples: Optional[torch.Tensor],
                        weights: Optional[torch.Tensor], grad_h1: torch.Tensor,
                        grad_eri: Optional[torch.Tensor] = None, opts: Optional[Opts] = None,
                        n_tuples=None) -> torch.Tensor:
        norb = h1.shape[0]
        if tuples is not None:
            self._dev(tuples, torch.int32, "tuples")
            n_t = tuples.shape[0] if n_tuples is None else n_tuples
        else:
            n_t = 1 if n_tuples is None else n_tuples
        status = self._empty((n_t,), torch.int32)
        o = (opts or Opts()).to_c()
        if weights is not None:
            self._dev(weights, torch.float64, "weights")
        self._dev(grad_h1, torch.float64, "grad_h1")
        if grad_eri is not None:
            self._dev(grad_eri, torch.float64, "grad_eri")
        _check(lib().casci_rdm_batch(self._h, norb, self._p(self._dev(h1, torch.float64, "h1")),
                                     self._p(self._dev(eri, torch.float64, "eri")),
                                     self._p(self._dev(occ, torch.uint8, "occ")), len(ref), _i32_host(ref),
                                     order, n_t, self._p(tuples), ctypes.byref(o), self._p(weights),
                                     self._p(grad_h1), self._p(grad_eri), self._p(status)), "casci_rdm_batch")
        return status

    def mbe_phi_gradient(self, occ, scale: float, grad_h1, grad_eri=None) -> None:
        _check(lib().mbe_phi_gradient(self._h, grad_h1.shape[0], self._p(self._dev(occ, torch.uint8, "occ")),
                                      float(scale), self._p(grad_h1), self._p(grad_eri)), "mbe_phi_gradient")

    def casci_sigma_large(self, h1, eri, occ, cas: Sequence[int], c: torch.Tensor, precision: str = "fp64",
                          want_diag: bool = False):
        norb = h1.shape[0]
        self._dev(c, torch.float64, "c")
        sigma = torch.empty_like(c)
        diag = torch.empty_like(c) if want_diag else None
        prec = {"fp64": MBE_PREC_FP64, "mixed": MBE_PREC_MIXED}[precision]
        _check(lib().casci_sigma_large(self._h, norb, self._p(self._dev(h1, torch.float64, "h1")),
                                       self._p(self._dev(eri, torch.float64, "eri")),
                                       self._p(self._dev(occ, torch.uint8, "occ")), len(cas), _i32_host(cas),
                                       prec, self._p(c), self._p(sigma), self._p(diag)), "casci_sigma_large")
        return sigma, diag

    def casci_solve(self, h1, eri, occ, cas: Sequence[int], opts: Optional[Opts] = None, want_vector=False):
        """Lowest eigenpair of one large active space: dict(lambda, eps, rnorm, status, n64, n32[, c])."""
        norb = h1.shape[0]
        res = (ctypes.c_double * 3)()
        info = (ctypes.c_int32 * 3)()
        o = (opts or Opts()).to_c()
        cvec = None
        if want_vector:
            import math
            occ_h = occ.cpu().tolist()
            k = sum(int(occ_h[p]) for p in cas)
            cvec = self._empty((math.comb(len(cas), k) ** 2,), torch.float64)
        _check(lib().casci_solve(self._h, norb, self._p(self._dev(h1, torch.float64, "h1")),
                                 self._p(self._dev(eri, torch.float64, "eri")),
                                 self._p(self._dev(occ, torch.uint8, "occ")), len(cas), _i32_host(cas),
                                 ctypes.byref(o), res, info, self._p(cvec)), "casci_solve")
        out = dict(lam=res[0], eps=res[1], rnorm=res[2], status=info[0], n64=info[1], n32=info[2])
        if cvec is not None:
            out["c"] = cvec
        return out


def mbe_gradient(ctx: Context, h1, eri, occ, ref: Sequence[int], exp: Sequence[int], orders: Sequence[int],
                 skip: bool, opts: Optional[Opts] = None, two_body: bool = True, forward=None,
                 occ_host: Optional[Sequence[int]] = None, scale: float = 1.0):
    """Gradient of the MBE energy with respect to h1 and (pq|rs), on the device.

    E_MBE = E_CAS(R) + sum_S w(S) eps(S) with the adjoint weights of Eq. 2, so
        dE = dE_Phi + (1 - sum_S w(S)) (dE_CAS(R) - dE_Phi)
                    + sum_S w(S) (dE_CAS(R u S) - dE_Phi),
    every term a Hellmann-Feynman density-matrix contraction.  `forward` is the
    dict of a previous run_mbe (its tuple lists are reused); opts should carry a
    tight residual tolerance (default here 1e-9).  `scale` multiplies the
    gradient (the library folds it into the adjoint weights).
    Returns (grad_h1 [norb, norb], grad_eri [norb]*4 or None, forward dict).
    """
    opts = opts or Opts(tol=1e-9)
    if forward is None:
        forward = run_mbe(ctx, h1, eri, occ, ref, exp, orders, skip, opts, occ_host=occ_host)
    norb = h1.shape[0]
    gh = torch.zeros((norb, norb), dtype=torch.float64, device=ctx.device)
    ge = torch.zeros((norb,) * 4, dtype=torch.float64, device=ctx.device) if two_body else None
    w, r_w = ctx.mbe_weights(forward["tuples"], exp, scale)
    ctx.mbe_phi_gradient(occ, scale, gh, ge)
    if len(ref) > 0:
        ctx.casci_rdm_batch(h1, eri, occ, ref, 0, None, r_w, gh, ge, opts)
    for n, tup, wt in zip(orders, forward["tuples"], w):
        if tup.shape[0] > 0:
            ctx.casci_rdm_batch(h1, eri, occ, ref, n, tup, wt, gh, ge, opts)
    return gh, ge, forward


class MBEEnergy(torch.autograd.Function):
    """E_MBE(h1, eri) with a hand-written adjoint (density matrices + Eq. 2 weights)."""

    @staticmethod
    def forward(fctx, h1, eri, ctx, occ, ref, exp, orders, skip, opts, two_body):
        out = run_mbe(ctx, h1, eri, occ, ref, exp, orders, skip, opts)
        fctx.save_for_backward(h1, eri, occ)
        fctx.cfg = (ctx, ref, exp, orders, skip, opts, two_body, out)
        return out["e_total"].clone()

    @staticmethod
    def backward(fctx, grad_out):
        h1, eri, occ = fctx.saved_tensors
        ctx, ref, exp, orders, skip, opts, two_body, out = fctx.cfg
        # the upstream derivative of the scalar output, read back and handed to the library
        gh, ge, _ = mbe_gradient(ctx, h1, eri, occ, ref, exp, orders, skip, opts, two_body, forward=out,
                                 scale=float(grad_out.reshape(()).item()))
        return gh, ge, None, None, None, None, None, None, None, None


EXPANSION_TYPES = ("type1", "type2", "type3")


def expansion_spaces(occ: Sequence[int], kind: str, active: Sequence[int] = ()):
    """(ref, exp) of the three expansion types of Sec. 1 (Fig. 1), as sorted lists.

    * type1 (Bethe-Goldstone): the expansion space is the occupied orbitals, and
      the reference space is every virtual orbital, so an order-k tuple
      correlates 2k electrons in k + M_vir orbitals.  `active` must be empty.
    * type2: the reference space is every occupied orbital plus the virtual
      orbitals in `active`; the expansion space is the other virtuals.  Every
      tuple correlates all electrons.
    * type3: the reference space is `active` (empty: the vacuum reference
      space); the expansion space is every other orbital.

    Host-side choice of orbital lists only; run_mbe and run_mbe_screened take
    the result as their ref and exp.  Raises ValueError on an unknown kind, on
    an orbital index out of range or repeated, on occupied orbitals in a type2
    `active`, and on a type1 call with a non-empty `active`.
    """
    occ_h = [int(v) for v in occ]
    norb = len(occ_h)
    act = sorted(int(p) for p in active)
    if kind not in EXPANSION_TYPES:
        raise ValueError(f"expansion_spaces: kind must be one of {EXPANSION_TYPES}, got {kind!r}")
    if any(p < 0 or p >= norb for p in act) or len(set(act)) != len(act):
        raise ValueError("expansion_spaces: active orbitals out of range or repeated")
    occupied = [p for p in range(norb) if occ_h[p]]
    virtual = [p for p in range(norb) if not occ_h[p]]
    if kind == "type1":
        if act:
            raise ValueError("expansion_spaces: type1 takes no active orbitals")
        return virtual, occupied
    if kind == "type2":
        if any(occ_h[p] for p in act):
            raise ValueError("expansion_spaces: type2 active orbitals must be virtual")
        return sorted(occupied + act), [p for p in virtual if p not in act]
    return act, [p for p in range(norb) if p not in act]


def _order_casci(ctx: Context, h1, eri, occ, ref, e_ref, order, tup, opts, large_ndet):
    """casci_batch, or casci_batch_routed when the active spaces exceed MBE_MAX_CAS
    orbitals or a determinant limit for the batched solvers is given."""
    if len(ref) + order <= MBE_MAX_CAS and not large_ndet:
        return ctx.casci_batch(h1, eri, occ, ref, e_ref, order, tup, opts)
    return ctx.casci_batch_routed(h1, eri, occ, ref, e_ref, order, tup, opts, large_ndet or 0)


def run_mbe(ctx: Context, h1, eri, occ, ref: Sequence[int], exp: Sequence[int],
            orders: Sequence[int], skip: bool, opts: Optional[Opts] = None,
            occ_host: Optional[Sequence[int]] = None, large_ndet: Optional[int] = None):
    """One pass of the whole hot path through the C ABI: tuples, tuple CASCI,
    increments (Eq. 2) and the order sums and total (Eq. 1), all on the device.

    h1, eri, occ are device tensors.  Returns a dict of device tensors (per-order
    tuples, eps, status, iters, increments; e_order, e_total, e_phi) and the
    reference-space correlation energy used.  Active spaces R u Omega of more than
    MBE_MAX_CAS (up to MBE_MAX_LARGE_CAS) orbitals, as in Type-1 and Type-2
    expansions, and with large_ndet set the tuples above that many determinants,
    go through casci_batch_routed.
    """
    occ_h = [int(v) for v in (occ_host if occ_host is not None else occ.cpu().tolist())]
    norb = h1.shape[0]
    e_phi = ctx.mbe_phi_energy(h1, eri, occ)
    e_ref = 0.0
    if len(ref) > 0:
        eps_r, st_r, _ = _order_casci(ctx, h1, eri, occ, ref, 0.0, 0, None, opts, large_ndet)
        e_ref = float(eps_r.item())
    out = dict(tuples=[], eps=[], status=[], iters=[], inc=[], e_phi=e_phi, e_ref_corr=e_ref)
    for n in orders:
        tup = ctx.mbe_tuples(norb, occ_h, exp, ref, n, skip)
        eps, status, iters = _order_casci(ctx, h1, eri, occ, ref, e_ref, n, tup, opts, large_ndet)
        inc = ctx.mbe_increments(n, tup, eps, out["tuples"], out["inc"]) if n == len(out["inc"]) + 1 \
            else None
        if inc is None:
            raise MbeError("orders must be 1, 2, ..., n without gaps")
        out["tuples"].append(tup)
        out["eps"].append(eps)
        out["status"].append(status)
        out["iters"].append(iters)
        out["inc"].append(inc)
    e_order, e_total = ctx.mbe_total(out["inc"], e_phi, e_ref)
    out["e_order"] = e_order
    out["e_total"] = e_total
    return out


def run_mbe_screened(ctx: Context, h1, eri, occ, ref: Sequence[int], exp: Sequence[int], max_order: int,
                     skip: bool, t_init: float = 1e-10, m_init: int = 3, a: float = 5.0,
                     opts: Optional[Opts] = None, occ_host: Optional[Sequence[int]] = None,
                     large_ndet: Optional[int] = None):
    """The screened expansion through the C ABI: orders up to the first computed
    one (order 2 for an empty reference space with the skip rule, else 1) are
    complete; every later order holds the children mbe_screen spawns from the
    order below, until max_order or until no child is spawned.  Returns the
    dict of run_mbe plus "orders" (the orders with tuples)."""
    occ_h = [int(v) for v in (occ_host if occ_host is not None else occ.cpu().tolist())]
    norb = h1.shape[0]
    e_phi = ctx.mbe_phi_energy(h1, eri, occ)
    e_ref = 0.0
    if len(ref) > 0:
        eps_r, st_r, _ = _order_casci(ctx, h1, eri, occ, ref, 0.0, 0, None, opts, large_ndet)
        e_ref = float(eps_r.item())
    k0 = 2 if (skip and len(ref) == 0) else 1
    out = dict(tuples=[], eps=[], status=[], iters=[], inc=[], e_phi=e_phi, e_ref_corr=e_ref, orders=[])
    for n in range(1, max_order + 1):
        if n <= k0:
            tup = ctx.mbe_tuples(norb, occ_h, exp, ref, n, skip)
        else:
            tup = ctx.mbe_screen(norb, occ_h, exp, ref, n - 1, out["tuples"][-1], out["inc"][-1],
                                 t_init, m_init, a, skip)
        if tup.shape[0] == 0 and n >= k0:
            break
        eps, status, iters = _order_casci(ctx, h1, eri, occ, ref, e_ref, n, tup, opts, large_ndet)
        inc = ctx.mbe_increments(n, tup, eps, out["tuples"], out["inc"])
        out["tuples"].append(tup)
        out["eps"].append(eps)
        out["status"].append(status)
        out["iters"].append(iters)
        out["inc"].append(inc)
        if tup.shape[0] > 0:
            out["orders"].append(n)
    e_order, e_total = ctx.mbe_total(out["inc"], e_phi, e_ref)
    out["e_order"] = e_order
    out["e_total"] = e_total
    return out
