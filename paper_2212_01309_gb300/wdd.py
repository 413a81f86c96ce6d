"""Python binding of libwdd.so (the C ABI in include/wdd.h).

Argument marshalling only: every step of the reconstruction runs in the library's CUDA kernels.
PyTorch is used for device memory and streams.  If the shared library is missing this module
raises at load time; there is no CPU fallback.
"""
from __future__ import annotations

import collections
import ctypes
import os
from typing import Any

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libwdd.so")

# ---- enums (mirror include/wdd.h) -------------------------------------------------------------
OK, ERR_INVALID_ARG, ERR_OUT_OF_MEMORY, ERR_CUDA, ERR_SCAN_INDEX, ERR_STATE, ERR_TIMEOUT, \
    ERR_UNSUPPORTED = range(8)
BASIS = {"fourier_full": 0, "hg_tensor": 1, "hg_energy": 2}
PRECISION = {"fp32": 0, "split": 1}
FRAME_DTYPE = {"u16": 0, "f32": 1, "f64": 2}
ACCUM_MODE = {"direct": 0, "separable": 1}
ACCUM_KERNEL = {0: "accumulate_fp32_kernel", 1: "rowdft_kernel", 2: "accumulate_narrow_kernel",
                3: "accumulate_tc_kernel<128>", 4: "accumulate_tc_kernel<64>"}
PROJ_ENGINE = {"auto": 0, "tensor": 1, "simt": 2, "stream": 3}
ARRAY = {"weights": 0, "chi": 1, "accum": 2, "coeff": 3, "spectrum": 4, "basis_y": 5,
         "basis_x": 6, "mask": 7, "coeff_index": 8}


class WddError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        super().__init__(f"{where}: {_status_name(status)}: {detail}")


class Params(ctypes.Structure):
    _fields_ = [
        ("scan_y", ctypes.c_int32), ("scan_x", ctypes.c_int32),
        ("scan_step_m", ctypes.c_double),
        ("det_y", ctypes.c_int32), ("det_x", ctypes.c_int32),
        ("det_px_inv_m", ctypes.c_double),
        ("voltage_v", ctypes.c_double),
        ("semiconv_rad", ctypes.c_double),
        ("defocus_m", ctypes.c_double),
        ("epsilon", ctypes.c_double),
        ("rank_k", ctypes.c_int32),
        ("basis", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("frame_dtype", ctypes.c_int32),
        ("max_batch", ctypes.c_int32),
        ("accum_depth", ctypes.c_int32),
        ("det_center_y", ctypes.c_double),
        ("det_center_x", ctypes.c_double),
        ("eps_absolute", ctypes.c_int32),
        ("proj_cluster", ctypes.c_int32),
        ("hbm_budget_bytes", ctypes.c_int64),
        ("overlap_pushes", ctypes.c_int32),
        ("accum_segment", ctypes.c_int32),
        ("accum_mode", ctypes.c_int32), ("coalesce_frames", ctypes.c_int32),
        ("scan_rotation_rad", ctypes.c_double),
        ("proj_engine", ctypes.c_int32),
    ]


class Result(ctypes.Structure):
    _fields_ = [("obj", ctypes.c_void_p), ("phase", ctypes.c_void_p),
                ("frames_seen", ctypes.c_int64), ("positions_covered", ctypes.c_int64)]


class PlanInfo(ctypes.Structure):
    _fields_ = [
        ("rank_k", ctypes.c_int32), ("basis_ly", ctypes.c_int32), ("basis_lx", ctypes.c_int32),
        ("n_active", ctypes.c_int32),
        ("eps_eff", ctypes.c_double), ("wavelength_m", ctypes.c_double),
        ("bf_radius_px", ctypes.c_double), ("hg_sigma_px", ctypes.c_double),
        ("device_bytes", ctypes.c_int64), ("frames_seen", ctypes.c_int64),
        ("positions_covered", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
        ("staged", ctypes.c_int32), ("finished", ctypes.c_int32),
        ("proj_tensor", ctypes.c_int32), ("accum_mode", ctypes.c_int32),
        ("pending", ctypes.c_int32), ("proj_engine", ctypes.c_int32),
        ("accum_kernel", ctypes.c_int32), ("spectrum_cols", ctypes.c_int32),
    ]


# Exported entry points and their signatures.
_SIGS: dict[str, tuple[Any, list[Any]]] = {
    "wdd_version": (ctypes.c_int32, []),
    "wdd_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "wdd_last_error": (ctypes.c_char_p, []),
    "wdd_params_default": (ctypes.c_int, [ctypes.POINTER(Params)]),
    "wdd_plan_create": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_void_p)]),
    "wdd_plan_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "wdd_plan_set_probe": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "wdd_merge_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_int64]),
    "wdd_plan_footprint": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_int64)]),
    "wdd_flush": (ctypes.c_int, [ctypes.c_void_p]),
    "wdd_flush_group": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32,
                                       ctypes.c_void_p]),
    "wdd_flush_group_max": (ctypes.c_int32, []),
    "wdd_push_frames": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_int64, ctypes.c_void_p]),
    "wdd_snapshot": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Result)]),
    "wdd_finalize": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Result)]),
    "wdd_reset": (ctypes.c_int, [ctypes.c_void_p]),
    "wdd_set_stream": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "wdd_plan_get_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(PlanInfo)]),
    "wdd_set_stage_timing": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "wdd_get_stage_times": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "wdd_check_device": (ctypes.c_int, [ctypes.c_void_p]),
    "wdd_selftest_bounded_wait": (ctypes.c_int, [ctypes.c_int64]),
    "wdd_reconstruct_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                               ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_void_p]),
    "wdd_detector_center": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                           ctypes.c_int32, ctypes.c_int32,
                                           ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "wdd_offline_plan_create": (ctypes.c_int, [ctypes.POINTER(Params),
                                               ctypes.POINTER(ctypes.c_void_p)]),
    "wdd_offline_probe_plan_create": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_void_p,
                                                     ctypes.POINTER(ctypes.c_void_p)]),
    "wdd_offline_footprint": (ctypes.c_int, [ctypes.POINTER(Params),
                                             ctypes.POINTER(ctypes.c_int64)]),
    "wdd_offline_reconstruct": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.POINTER(Result), ctypes.c_void_p]),
    "wdd_offline_copy_array": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                              ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "wdd_offline_get_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                            ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(ctypes.c_double)]),
    "wdd_offline_plan_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "wdd_get_hit_counts": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    "wdd_copy_array": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                      ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
}

_lib = None


def lib() -> ctypes.CDLL:
    """Loads libwdd.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2212_01309_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _status_name(s: int) -> str:
    try:
        return lib().wdd_status_string(s).decode()
    except Exception:  # pragma: no cover - only when the library itself is unusable
        return str(s)


def _check(status: int, where: str) -> None:
    if status != OK:
        raise WddError(status, where, lib().wdd_last_error().decode())


def exported_symbols() -> list[str]:
    return sorted(_SIGS)


def make_params(*, scan_y, scan_x, scan_step_m, det_y, det_x, det_px_inv_m, voltage_v,
                semiconv_rad, defocus_m=0.0, epsilon=1e-3, rank_k, basis="hg_tensor",
                precision="fp32", frame_dtype="f32", max_batch=256, accum_depth=0,
                det_center_y=-1.0, det_center_x=-1.0, eps_absolute=False,
                hbm_budget_bytes=0, proj_cluster=0, overlap_pushes=False,
                accum_segment=0, accum_mode="direct", coalesce_frames=0,
                scan_rotation_rad=0.0, proj_engine="auto") -> Params:
    p = Params()
    _check(lib().wdd_params_default(ctypes.byref(p)), "wdd_params_default")
    p.scan_y, p.scan_x, p.scan_step_m = scan_y, scan_x, scan_step_m
    p.det_y, p.det_x, p.det_px_inv_m = det_y, det_x, det_px_inv_m
    p.voltage_v, p.semiconv_rad, p.defocus_m = voltage_v, semiconv_rad, defocus_m
    p.epsilon, p.rank_k = epsilon, rank_k
    p.basis = BASIS[basis] if isinstance(basis, str) else int(basis)
    p.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    p.frame_dtype = FRAME_DTYPE[frame_dtype] if isinstance(frame_dtype, str) else int(frame_dtype)
    p.max_batch, p.accum_depth = max_batch, accum_depth
    p.det_center_y, p.det_center_x = det_center_y, det_center_x
    p.eps_absolute = 1 if eps_absolute else 0
    p.hbm_budget_bytes = hbm_budget_bytes
    p.proj_cluster = proj_cluster
    p.overlap_pushes = 1 if overlap_pushes else 0
    p.accum_segment = accum_segment
    p.accum_mode = ACCUM_MODE[accum_mode] if isinstance(accum_mode, str) else int(accum_mode)
    p.coalesce_frames = coalesce_frames
    p.scan_rotation_rad = scan_rotation_rad
    p.proj_engine = PROJ_ENGINE[proj_engine] if isinstance(proj_engine, str) else int(proj_engine)
    return p


def params_from_acquisition(acq, *, basis, rank_k, epsilon=1e-3, **kw) -> Params:
    return make_params(scan_y=acq.scan_y, scan_x=acq.scan_x, scan_step_m=acq.scan_step_m,
                       det_y=acq.det, det_x=acq.det, det_px_inv_m=acq.det_px_inv_m,
                       voltage_v=acq.voltage_v, semiconv_rad=acq.semiconv_rad,
                       defocus_m=acq.defocus_m, epsilon=epsilon, rank_k=rank_k, basis=basis,
                       frame_dtype=acq.dtype, **kw)


def plan_footprint(params: Params) -> int:
    """Device bytes a plan with these parameters would hold (no GPU work)."""
    b = ctypes.c_int64()
    _check(lib().wdd_plan_footprint(ctypes.byref(params), ctypes.byref(b)), "wdd_plan_footprint")
    return int(b.value)


def _ptr(x) -> int:
    """Address of a torch tensor or numpy array's data (no copy)."""
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if isinstance(x, np.ndarray):
        return int(x.ctypes.data)
    raise TypeError(f"unsupported buffer type {type(x)}")


class Plan:
    """A live-WDD plan on the current CUDA device (owns its device buffers)."""

    def __init__(self, params: Params):
        import torch  # noqa: F401  (device context, memory and streams)
        self.params = params
        h = ctypes.c_void_p()
        _check(lib().wdd_plan_create(ctypes.byref(params), ctypes.byref(h)), "wdd_plan_create")
        self._h = h
        self.S = params.scan_y * params.scan_x
        self.K = params.rank_k
        self._keep: collections.deque = collections.deque(maxlen=64)

    # -- lifetime --------------------------------------------------------------------------
    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            _check(lib().wdd_plan_destroy(self._h), "wdd_plan_destroy")
            self._h = ctypes.c_void_p()
        self._keep.clear()

    def __del__(self):  # pragma: no cover - best effort
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- streaming -------------------------------------------------------------------------
    def push(self, frames, scan_idx, stream=None) -> None:
        """Enqueues frames (torch tensor on the GPU or in pinned memory, or a numpy array)."""
        import torch
        idx = np.ascontiguousarray(np.asarray(scan_idx, dtype=np.int32))
        n = int(idx.shape[0])
        if stream is None:
            stream = torch.cuda.current_stream()
        sh = ctypes.c_void_p(int(stream.cuda_stream))
        if hasattr(frames, "is_contiguous") and not frames.is_contiguous():
            raise ValueError("frames must be contiguous")
        _check(lib().wdd_push_frames(self._h, ctypes.c_void_p(_ptr(frames)),
                                     ctypes.c_void_p(idx.ctypes.data), n, sh), "wdd_push_frames")
        # The library borrows the frames until the stream has passed this push; keeping the most
        # recent ones referenced here covers callers that drop them right after the call.
        self._keep.append(frames)

    def _result(self, fn, obj=None, phase=None):
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        if obj is None:
            obj = torch.empty((self.params.scan_y, self.params.scan_x), dtype=torch.complex64,
                              device=dev)
        if phase is None:
            phase = torch.empty((self.params.scan_y, self.params.scan_x), dtype=torch.float32,
                                device=dev)
        r = Result(obj=_ptr(obj), phase=_ptr(phase) if phase is not False else None)
        _check(fn(self._h, ctypes.byref(r)), fn.__name__)
        return obj, (phase if phase is not False else None), int(r.frames_seen), \
            int(r.positions_covered)

    def snapshot(self, obj=None, phase=None, stream=None):
        """(object complex64 [S_y, S_x], phase f32, frames_seen, positions_covered)."""
        if stream is not None:
            self.set_stream(stream)
        return self._result(lib().wdd_snapshot, obj, phase)

    def finalize(self, obj=None, phase=None, stream=None):
        if stream is not None:
            self.set_stream(stream)
        return self._result(lib().wdd_finalize, obj, phase)

    def set_probe(self, probe) -> None:
        """Rebuilds the Wiener filter from a recovered probe (complex64 [scan_y, scan_x] on the
        scan grid, e.g. the output of OfflinePlan(params, obj=...).reconstruct); the
        accumulated frames are kept."""
        import torch
        if (not isinstance(probe, torch.Tensor) or probe.dtype != torch.complex64
                or probe.numel() != self.params.scan_y * self.params.scan_x
                or not probe.is_contiguous()):
            raise ValueError("probe must be a contiguous complex64 tensor of scan_y * scan_x")
        _check(lib().wdd_plan_set_probe(self._h, ctypes.c_void_p(_ptr(probe))),
               "wdd_plan_set_probe")

    def flush(self, stream=None) -> None:
        """Accumulates the staged frames now (a later snapshot then only reconstructs)."""
        if stream is not None:
            self.set_stream(stream)
        _check(lib().wdd_flush(self._h), "wdd_flush")

    def set_stream(self, stream) -> None:
        _check(lib().wdd_set_stream(self._h, ctypes.c_void_p(int(stream.cuda_stream))),
               "wdd_set_stream")

    def reset(self, stream=None) -> None:
        if stream is not None:
            self.set_stream(stream)
        _check(lib().wdd_reset(self._h), "wdd_reset")

    # -- inspection ------------------------------------------------------------------------
    def info(self) -> dict:
        pi = PlanInfo()
        _check(lib().wdd_plan_get_info(self._h, ctypes.byref(pi)), "wdd_plan_get_info")
        return {name: getattr(pi, name) for name, _ in PlanInfo._fields_}

    def check_device(self) -> None:
        """Raises WddError(ERR_TIMEOUT) if a kernel of this plan gave up a bounded wait."""
        _check(lib().wdd_check_device(self._h), "wdd_check_device")

    STAGES = ("project", "accumulate", "deconvolve", "idft")

    def set_stage_timing(self, enable: bool) -> None:
        _check(lib().wdd_set_stage_timing(self._h, 1 if enable else 0), "wdd_set_stage_timing")

    def stage_times(self) -> dict:
        """{stage: (total_ms, launches)} since the previous call (synchronises the stream)."""
        ms = np.zeros(4, dtype=np.float64)
        cnt = np.zeros(4, dtype=np.int64)
        _check(lib().wdd_get_stage_times(self._h, ctypes.c_void_p(ms.ctypes.data),
                                         ctypes.c_void_p(cnt.ctypes.data)), "wdd_get_stage_times")
        return {s: (float(ms[i]), int(cnt[i])) for i, s in enumerate(self.STAGES)}

    def hit_counts(self) -> np.ndarray:
        out = np.zeros(self.S, dtype=np.uint32)
        _check(lib().wdd_get_hit_counts(self._h, ctypes.c_void_p(out.ctypes.data), self.S),
               "wdd_get_hit_counts")
        return out

    def _signature(self) -> tuple:
        p = self.params
        return (p.scan_y, p.scan_x, p.det_y, p.det_x, p.rank_k, p.basis)

    def export_state(self) -> dict:
        """The plan's state (accumulator with staged frames accumulated first, hit counters,
        frame count): enough to resume the acquisition or merge it with another partition."""
        return {"accum": self.copy_array("accum"), "hits": self.hit_counts(),
                "frames_seen": int(self.info()["frames_seen"]), "signature": self._signature()}

    def merge_state(self, state: dict, stream=None) -> None:
        """Adds an exported state (of a plan with the same parameters) to this plan, in stream
        order.  ``state["accum"]`` may be a numpy array (copied to pinned memory here) or a
        complex64 torch tensor on the GPU or in pinned memory."""
        import torch
        sig = state.get("signature")
        if sig is not None and tuple(sig) != self._signature():
            raise ValueError("state of a plan with other parameters")
        accum = state["accum"]
        if isinstance(accum, np.ndarray):
            accum = torch.from_numpy(np.ascontiguousarray(accum, dtype=np.complex64)).pin_memory()
        if accum.dtype != torch.complex64 or not accum.is_contiguous():
            raise ValueError("accum must be contiguous complex64")
        hits = np.ascontiguousarray(state["hits"], dtype=np.uint32)
        if accum.numel() != self.S * self.K or hits.size != self.S:
            raise ValueError("state of a plan with other parameters")
        if stream is not None:
            self.set_stream(stream)
        _check(lib().wdd_merge_state(self._h, ctypes.c_void_p(_ptr(accum)),
                                     ctypes.c_void_p(hits.ctypes.data),
                                     int(state["frames_seen"])), "wdd_merge_state")
        # borrowed until the stream has passed the merge
        self._keep.append(accum)

    def copy_array(self, which: str) -> np.ndarray:
        inf = self.info()
        S, K = self.S, self.K
        M = inf["basis_ly"] * inf["basis_lx"]
        p = self.params
        cplx_basis = p.basis == BASIS["fourier_full"]
        shapes = {
            "weights": ((S, K), np.complex64), "chi": ((S, M), np.complex128),
            "accum": ((S, K), np.complex64), "spectrum": ((S,), np.complex64),
            "basis_y": ((p.det_y, inf["basis_ly"]), np.complex128),
            "basis_x": ((p.det_x, inf["basis_lx"]), np.complex128),
            "mask": ((S,), np.uint8), "coeff_index": ((K, 2), np.int32),
            "coeff": ((max(1, p.max_batch), K), np.float32),
        }
        shape, dt = shapes[which]
        out = np.zeros(shape, dtype=dt)
        written = ctypes.c_int64()
        _check(lib().wdd_copy_array(self._h, ARRAY[which], ctypes.c_void_p(out.ctypes.data),
                                    out.nbytes, ctypes.byref(written)), "wdd_copy_array")
        if which == "coeff":
            out = out[: written.value // (4 * K)]
        if which in ("basis_y", "basis_x") and not cplx_basis:
            out = out.real.copy()
        return out


def flush_group_max() -> int:
    """Most plans one flush_group call takes."""
    return int(lib().wdd_flush_group_max())


def flush_group(plans, stream) -> None:
    """Accumulates the staged frames of several SPLIT plans with one coefficient-split launch and
    one tensor-core launch on `stream` (which becomes every plan's stream); wdd_flush_group."""
    plans = list(plans)
    arr = (ctypes.c_void_p * max(1, len(plans)))(*[g._h.value for g in plans])
    _check(lib().wdd_flush_group(arr, len(plans), ctypes.c_void_p(int(stream.cuda_stream))),
           "wdd_flush_group")


def selftest_bounded_wait(wait_ns: int = 50_000_000) -> int:
    """Runs the device bounded-wait self test; returns the status code (ERR_TIMEOUT expected)."""
    return int(lib().wdd_selftest_bounded_wait(int(wait_ns)))


def offline_footprint(params: Params) -> int:
    b = ctypes.c_int64()
    _check(lib().wdd_offline_footprint(ctypes.byref(params), ctypes.byref(b)),
           "wdd_offline_footprint")
    return int(b.value)


class OfflinePlan:
    """Classical WDD on the whole 4-D dataset (wdd_offline_*): the comparison method, on the GPU.

    With ``obj`` (complex64 [scan_y, scan_x] object estimate on the GPU) the plan runs the
    deconvolution with the roles swapped (wdd_offline_probe_plan_create) and ``reconstruct``
    returns the probe on the scan grid instead of the object."""

    def __init__(self, params: Params, obj=None):
        import torch
        self.params = params
        self.S = params.scan_y * params.scan_x
        h = ctypes.c_void_p()
        if obj is None:
            _check(lib().wdd_offline_plan_create(ctypes.byref(params), ctypes.byref(h)),
                   "wdd_offline_plan_create")
        else:
            if (not isinstance(obj, torch.Tensor) or obj.dtype != torch.complex64
                    or obj.numel() != self.S or not obj.is_contiguous()):
                raise ValueError("obj must be a contiguous complex64 tensor of scan_y * scan_x")
            _check(lib().wdd_offline_probe_plan_create(ctypes.byref(params),
                                                       ctypes.c_void_p(_ptr(obj)),
                                                       ctypes.byref(h)),
                   "wdd_offline_probe_plan_create")
        self._h = h

    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            _check(lib().wdd_offline_plan_destroy(self._h), "wdd_offline_plan_destroy")
            self._h = ctypes.c_void_p()

    def __del__(self):  # pragma: no cover - best effort
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def reconstruct(self, frames, obj=None, phase=None, stream=None):
        """frames: [S, det_y, det_x] torch tensor on the GPU or in pinned memory, raster order.
        Returns (object complex64 [S_y, S_x], phase f32)."""
        import torch
        if hasattr(frames, "is_contiguous") and not frames.is_contiguous():
            raise ValueError("frames must be contiguous")
        dev = torch.device("cuda", torch.cuda.current_device())
        shape = (self.params.scan_y, self.params.scan_x)
        if obj is None:
            obj = torch.empty(shape, dtype=torch.complex64, device=dev)
        if phase is None:
            phase = torch.empty(shape, dtype=torch.float32, device=dev)
        if stream is None:
            stream = torch.cuda.current_stream()
        r = Result(obj=_ptr(obj), phase=_ptr(phase) if phase is not False else None)
        _check(lib().wdd_offline_reconstruct(self._h, ctypes.c_void_p(_ptr(frames)),
                                             ctypes.byref(r),
                                             ctypes.c_void_p(int(stream.cuda_stream))),
               "wdd_offline_reconstruct")
        return obj, (phase if phase is not False else None)

    def info(self) -> dict:
        b, n, f, e = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
        _check(lib().wdd_offline_get_info(self._h, ctypes.byref(b), ctypes.byref(n),
                                          ctypes.byref(f), ctypes.byref(e)),
               "wdd_offline_get_info")
        return {"device_bytes": b.value, "n_active": n.value, "fused": f.value,
                "eps_eff": e.value}

    def copy_array(self, which: str) -> np.ndarray:
        p = self.params
        shapes = {"spectrum": (0, np.complex64, (self.S,)),
                  "wiener": (1, np.complex64, (self.S, p.det_y, p.det_x)),
                  "mask": (2, np.uint8, (self.S,))}
        code, dt, shape = shapes[which]
        out = np.empty(shape, dtype=dt)
        w = ctypes.c_int64()
        _check(lib().wdd_offline_copy_array(self._h, code, ctypes.c_void_p(out.ctypes.data),
                                            out.nbytes, ctypes.byref(w)), "wdd_offline_copy_array")
        return out


def detector_center(frames, stream=None) -> tuple[float, float]:
    """Centre of mass (row, column) of frames [n, det_y, det_x] (wdd_detector_center): a torch
    tensor on the GPU or in pinned host memory, of dtype uint16, float32 or float64."""
    import torch
    dt = {torch.uint16: "u16", torch.float32: "f32", torch.float64: "f64"}.get(frames.dtype)
    if dt is None:
        raise TypeError(f"unsupported frame dtype {frames.dtype}")
    if frames.dim() != 3 or not frames.is_contiguous():
        raise ValueError("frames must be a contiguous [n, det_y, det_x] tensor")
    if stream is None:
        stream = torch.cuda.current_stream()
    cy, cx = ctypes.c_double(), ctypes.c_double()
    n, ny, nx = frames.shape
    _check(lib().wdd_detector_center(ctypes.c_void_p(_ptr(frames)), n, ny, nx, FRAME_DTYPE[dt],
                                     ctypes.byref(cy), ctypes.byref(cx),
                                     ctypes.c_void_p(int(stream.cuda_stream))),
           "wdd_detector_center")
    return cy.value, cx.value


def reconstruct_noalloc(weights, accum, scan_y: int, scan_x: int, rank_k: int, obj, phase=None,
                        stream=None) -> None:
    """Reconstruction that allocates no device memory (wdd_reconstruct_noalloc): for callers
    that cannot allocate, such as code running during CUDA graph capture.  All buffers are the
    caller's device tensors; the library's fixed scratch holds the intermediates."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(lib().wdd_reconstruct_noalloc(ctypes.c_void_p(_ptr(weights)), ctypes.c_void_p(_ptr(accum)),
                                         scan_y, scan_x, rank_k, ctypes.c_void_p(_ptr(obj)),
                                         ctypes.c_void_p(_ptr(phase)) if phase is not None else None,
                                         ctypes.c_void_p(int(stream.cuda_stream))),
           "wdd_reconstruct_noalloc")
