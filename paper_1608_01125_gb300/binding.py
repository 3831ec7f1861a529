"""Python binding of the trilens C ABI (``include/trilens.h``).

Argument marshalling only: device memory and streams come from PyTorch, every
step of the collision path runs in the CUDA library ``libtrilens.so``.  There
is no fallback: if the library or a CUDA device is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtrilens.so")

OK = 0
ERR_INVALID = -1
ERR_CAPACITY = -2
ERR_CUDA = -3
ERR_TIMEOUT = -4
ERR_STACK = -5
ERR_NOMEM = -6

FP64 = 0
FP32_BAND = 1
YIELD_EXACT = 0
YIELD_SURROGATE = 1

BEAM_KEYS = ("px", "py", "pz", "dx", "dy", "dz", "E", "w")


class TrilensError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"trilens error {code}: {msg}")
        self.code = code


class Beam(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64)] + [(k, ctypes.c_void_p) for k in BEAM_KEYS]


class Params(ctypes.Structure):
    _fields_ = [("dt_fs", ctypes.c_double), ("kappa", ctypes.c_double),
                ("precision", ctypes.c_int32), ("leaf_bucket", ctypes.c_int32),
                ("stack_depth", ctypes.c_int32), ("block_shape", ctypes.c_int32),
                ("spin_limit", ctypes.c_int64)]


class StepStats(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("count", ctypes.c_int64), ("weighted", ctypes.c_double),
                ("hsum", ctypes.c_uint64), ("hxor", ctypes.c_uint64),
                ("narrow_tests", ctypes.c_int64), ("node_tests", ctypes.c_int64),
                ("leaf_pairs", ctypes.c_int64), ("band", ctypes.c_int64),
                ("retries", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lock = threading.Lock()
_lib = None

#: kernel phases reported by Collider.phase_ms (trilens_debug_phase_ms order)
PHASES = ("propagate", "sort", "gather", "emit", "refit", "expand", "traverse", "band", "yield",
          "narrow")


class SurPairs(ctypes.Structure):
    """trilens_sur_pairs: host arrays of the level-L node pairs of a step."""
    _fields_ = [("cap", ctypes.c_int64), ("n_pairs", ctypes.c_int64),
                ("cloud", ctypes.c_void_p), ("feat", ctypes.c_void_p), ("st", ctypes.c_void_p),
                ("label", ctypes.c_void_p), ("pred", ctypes.c_void_p),
                ("fallback", ctypes.c_void_p), ("net", ctypes.c_void_p),
                ("cloud_of_a", ctypes.c_void_p), ("cloud_of_b", ctypes.c_void_p),
                ("fallback_exact", ctypes.c_double)]


def lib() -> ctypes.CDLL:
    """Load ``libtrilens.so`` (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.trilens_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Beam), ctypes.POINTER(Beam),
                                     ctypes.POINTER(Params), vp]
        L.trilens_create.restype = ctypes.c_int
        L.trilens_build.argtypes = [vp, i64]
        L.trilens_build.restype = ctypes.c_int
        L.trilens_collide_step.argtypes = [vp, i64, vp, i64, ctypes.POINTER(i64)]
        L.trilens_collide_step.restype = ctypes.c_int
        L.trilens_step_stats_get.argtypes = [vp, ctypes.POINTER(StepStats)]
        L.trilens_step_stats_get.restype = ctypes.c_int
        L.trilens_yield.argtypes = [vp, i32, i32, ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
        L.trilens_yield.restype = ctypes.c_int
        L.trilens_reset_yield.argtypes = [vp]
        L.trilens_reset_yield.restype = ctypes.c_int
        L.trilens_run.argtypes = [vp, i64, i64, ctypes.POINTER(StepStats)]
        L.trilens_run.restype = ctypes.c_int
        L.trilens_pair_products.argtypes = [ctypes.POINTER(Beam), ctypes.POINTER(Beam), vp, i64,
                                            ctypes.c_uint64, vp, vp]
        L.trilens_pair_products.restype = ctypes.c_int
        L.trilens_destroy.argtypes = [vp]
        L.trilens_destroy.restype = None
        L.trilens_status_str.argtypes = [ctypes.c_int]
        L.trilens_status_str.restype = ctypes.c_char_p
        L.trilens_last_error.argtypes = [vp]
        L.trilens_last_error.restype = ctypes.c_char_p
        L.trilens_version.argtypes = []
        L.trilens_version.restype = ctypes.c_char_p
        L.trilens_debug_stall_sort.argtypes = [vp, ctypes.c_int]
        L.trilens_debug_stall_sort.restype = ctypes.c_int
        L.trilens_debug_set_spin_limit.argtypes = [vp, i64]
        L.trilens_debug_set_spin_limit.restype = ctypes.c_int
        L.trilens_debug_set_cut_cap.argtypes = [vp, ctypes.c_int32]
        L.trilens_debug_set_cut_cap.restype = ctypes.c_int
        L.trilens_debug_shrink_buffers.argtypes = [vp, i64]
        L.trilens_debug_shrink_buffers.restype = ctypes.c_int
        L.trilens_debug_set_key_bits.argtypes = [vp, ctypes.c_int32]
        L.trilens_debug_set_key_bits.restype = ctypes.c_int
        L.trilens_debug_eval64.argtypes = [vp, vp, i64, i32, vp]
        L.trilens_debug_eval64.restype = ctypes.c_int
        L.trilens_debug_set_parts.argtypes = [vp, i32]
        L.trilens_debug_set_parts.restype = ctypes.c_int
        L.trilens_debug_band_stress.argtypes = [ctypes.c_uint64, i64, ctypes.c_double,
                                                ctypes.c_double, vp, vp, i64, vp]
        L.trilens_debug_band_stress.restype = ctypes.c_int
        L.trilens_debug_narrow_bins.argtypes = [ctypes.c_double, ctypes.c_double, vp, i32,
                                                ctypes.POINTER(ctypes.c_float)]
        L.trilens_debug_narrow_bins.restype = ctypes.c_int
        L.trilens_debug_timing.argtypes = [vp, ctypes.c_int]
        L.trilens_debug_timing.restype = ctypes.c_int
        L.trilens_debug_phase_ms.argtypes = [vp, ctypes.POINTER(dbl), ctypes.POINTER(i64), ctypes.c_int]
        L.trilens_debug_phase_ms.restype = ctypes.c_int
        L.trilens_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Beam),
                                           ctypes.POINTER(Beam), i32, ctypes.POINTER(Params), vp]
        L.trilens_batch_create.restype = ctypes.c_int
        L.trilens_batch_run.argtypes = [vp, i64, i64, vp]
        L.trilens_batch_run.restype = ctypes.c_int
        L.trilens_collide_batch.argtypes = [ctypes.POINTER(Beam), ctypes.POINTER(Beam),
                                            ctypes.POINTER(Params), i32, i64, vp, vp]
        L.trilens_collide_batch.restype = ctypes.c_int
        L.trilens_set_tuning.argtypes = [vp, i32, i32, i32, i32]
        L.trilens_set_tuning.restype = ctypes.c_int
        L.trilens_get_tuning.argtypes = [vp, ctypes.POINTER(i32)]
        L.trilens_get_tuning.restype = ctypes.c_int
        L.trilens_autotune.argtypes = [vp, ctypes.POINTER(i64), i32, ctypes.c_char_p,
                                       ctypes.POINTER(i32)]
        L.trilens_autotune.restype = ctypes.c_int
        L.trilens_mlp_forward.argtypes = [vp, vp, vp, i64, vp, vp]
        L.trilens_mlp_forward.restype = ctypes.c_int
        L.trilens_mlp_grad.argtypes = [vp, vp, vp, vp, vp, ctypes.c_float, i32, i64, vp, vp, vp]
        L.trilens_mlp_grad.restype = ctypes.c_int
        L.trilens_surrogate_collect.argtypes = [vp, ctypes.POINTER(i64), i32, i32]
        L.trilens_surrogate_fit.argtypes = [vp, i32, ctypes.c_uint64]
        L.trilens_surrogate_train.argtypes = [vp, ctypes.POINTER(i64), i32, i32, i32, ctypes.c_uint64]
        L.trilens_surrogate_step.argtypes = [vp, i64, i32, ctypes.c_float, ctypes.POINTER(dbl)]
        L.trilens_surrogate_info.argtypes = [vp, ctypes.POINTER(dbl)]
        L.trilens_surrogate_dataset.argtypes = [vp, vp, vp, vp, i64, ctypes.POINTER(i64)]
        L.trilens_surrogate_save.argtypes = [vp, ctypes.c_char_p]
        L.trilens_surrogate_load.argtypes = [vp, ctypes.c_char_p]
        L.trilens_surrogate_add_samples.argtypes = [vp, vp, vp, vp, i64, i32]
        L.trilens_surrogate_pairs.argtypes = [vp, i64, i32, ctypes.c_float,
                                              ctypes.POINTER(SurPairs)]
        for f in ("collect", "fit", "train", "step", "info", "dataset", "save", "load",
                  "add_samples", "pairs"):
            getattr(L, "trilens_surrogate_" + f).restype = ctypes.c_int
        L.trilens_yield_reduce_noalloc.argtypes = [vp, i64, vp, vp, vp, vp]
        L.trilens_yield_reduce_noalloc.restype = ctypes.c_int
        L.trilens_deplete_step.argtypes = [vp, i64, vp, i64, vp, vp, vp, ctypes.POINTER(i64),
                                           ctypes.POINTER(dbl)]
        L.trilens_deplete_step.restype = ctypes.c_int
        L.trilens_deplete_step_async.argtypes = [vp, i64, vp, i64, vp, vp, vp, vp]
        L.trilens_deplete_step_async.restype = ctypes.c_int
        L.trilens_deplete_rounds.argtypes = [vp, ctypes.POINTER(i64)]
        L.trilens_deplete_rounds.restype = ctypes.c_int
        L.trilens_swarm_mark.argtypes = [ctypes.POINTER(Beam), ctypes.POINTER(Beam), dbl, dbl,
                                         ctypes.POINTER(Params), i64, i64, vp, vp, vp]
        L.trilens_swarm_mark.restype = ctypes.c_int
        L.trilens_swarm_count.argtypes = [ctypes.POINTER(Beam), vp, vp, ctypes.POINTER(i64), vp]
        L.trilens_swarm_count.restype = ctypes.c_int
        L.trilens_swarm_expand.argtypes = [ctypes.POINTER(Beam), dbl, vp, i64,
                                           ctypes.POINTER(vp), vp, vp, vp]
        L.trilens_swarm_expand.restype = ctypes.c_int
        _lib = L
        return L


def status_str(code: int) -> str:
    return lib().trilens_status_str(code).decode()


def _check(rc: int, ctx=None):
    if rc != OK:
        msg = status_str(rc)
        if ctx is not None:
            detail = lib().trilens_last_error(ctx)
            if detail:
                msg += f" ({detail.decode()})"
        raise TrilensError(rc, msg)


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("trilens needs a CUDA device; none is available")
    return torch


def to_device(beam: dict, device="cuda") -> dict:
    """Copy a numpy beam (see synth.py) to contiguous float64 device tensors."""
    torch = _torch()
    return {k: torch.from_numpy(np.ascontiguousarray(beam[k], dtype=np.float64)).to(device)
            for k in BEAM_KEYS}


def beam_struct(t: dict) -> Beam:
    n = int(t["px"].numel())
    ptrs = []
    for k in BEAM_KEYS:
        v = t.get(k)
        if v is None:
            ptrs.append(None)
            continue
        assert v.is_cuda and v.dtype.is_floating_point and v.element_size() == 8
        assert v.is_contiguous() and v.numel() == n
        ptrs.append(v.data_ptr() if n > 0 else None)
    return Beam(n, *ptrs)


class Collider:
    """One context: two resident beams, built and collided step by step."""

    def __init__(self, beam_a: dict, beam_b: dict, dt_fs: float, kappa: float,
                 precision: int = FP32_BAND, leaf_bucket: int = 0, stack_depth: int = 0,
                 block_shape: int = 0, spin_limit: int = 0, stream=None):
        torch = _torch()
        self._torch = torch
        self.a = beam_a if _is_dev(beam_a) else to_device(beam_a)
        self.b = beam_b if _is_dev(beam_b) else to_device(beam_b)
        self.params = Params(float(dt_fs), float(kappa), int(precision), int(leaf_bucket),
                             int(stack_depth), int(block_shape), int(spin_limit))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._ba, self._bb = beam_struct(self.a), beam_struct(self.b)
        h = ctypes.c_void_p()
        _check(lib().trilens_create(ctypes.byref(h), ctypes.byref(self._ba), ctypes.byref(self._bb),
                                    ctypes.byref(self.params), ctypes.c_void_p(self.stream.cuda_stream)))
        self.ctx = h

    def build(self, step: int):
        _check(lib().trilens_build(self.ctx, int(step)), self.ctx)

    def collide(self, step: int, hits=None) -> int:
        """Collide the built step; with a (cap, 2) uint32-sized int32 tensor,
        also return the hit pairs in it.  Returns the step's hit count."""
        n = ctypes.c_int64(0)
        if hits is None:
            rc = lib().trilens_collide_step(self.ctx, int(step), None, 0, ctypes.byref(n))
        else:
            assert hits.is_cuda and hits.element_size() == 4 and hits.is_contiguous()
            cap = hits.numel() // 2
            rc = lib().trilens_collide_step(self.ctx, int(step), ctypes.c_void_p(hits.data_ptr()),
                                            cap, ctypes.byref(n))
        if rc == ERR_CAPACITY:
            err = TrilensError(rc, f"hit buffer too small, need {n.value}")
            err.needed = int(n.value)
            raise err
        _check(rc, self.ctx)
        return int(n.value)

    def step_hits(self, step: int, cap: int | None = None):
        """Build and collide `step`; return (hits[n, 2] int64 numpy, stats)."""
        torch = self._torch
        self.build(step)
        cap = cap or 1 << 16
        while True:
            buf = torch.empty((cap, 2), dtype=torch.int32, device=self.a["px"].device)
            try:
                n = self.collide(step, buf)
                break
            except TrilensError as e:
                if e.code != ERR_CAPACITY:
                    raise
                cap = e.needed + 16
        self.stream.synchronize()
        h = buf[:n].cpu().numpy().view(np.uint32).astype(np.int64)
        return h, self.stats()

    def run(self, first_step: int, steps: int) -> dict:
        """Build and collide steps first_step .. first_step+steps-1 as one
        captured graph (trilens_run); returns the run's totals."""
        s = StepStats()
        _check(lib().trilens_run(self.ctx, int(first_step), int(steps), ctypes.byref(s)),
               self.ctx)
        return s.as_dict()

    def stats(self) -> dict:
        s = StepStats()
        _check(lib().trilens_step_stats_get(self.ctx, ctypes.byref(s)), self.ctx)
        return s.as_dict()

    def yield_(self, mode: int = YIELD_EXACT, level_L: int = 0):
        c, w = ctypes.c_double(), ctypes.c_double()
        _check(lib().trilens_yield(self.ctx, mode, level_L, ctypes.byref(c), ctypes.byref(w)),
               self.ctx)
        return c.value, w.value

    def reset_yield(self):
        _check(lib().trilens_reset_yield(self.ctx), self.ctx)

    def debug_stall_sort(self, on: bool):
        _check(lib().trilens_debug_stall_sort(self.ctx, int(bool(on))), self.ctx)

    def timing(self, on: bool = True):
        _check(lib().trilens_debug_timing(self.ctx, int(bool(on))), self.ctx)

    def phase_ms(self, reset: bool = False) -> tuple[dict, dict]:
        ms = (ctypes.c_double * len(PHASES))()
        ln = (ctypes.c_int64 * len(PHASES))()
        _check(lib().trilens_debug_phase_ms(self.ctx, ms, ln, int(bool(reset))), self.ctx)
        return dict(zip(PHASES, list(ms))), dict(zip(PHASES, list(ln)))

    def set_tuning(self, leaf_bucket: int, stack_depth: int, block_shape: int, budget: int):
        _check(lib().trilens_set_tuning(self.ctx, leaf_bucket, stack_depth, block_shape, budget),
               self.ctx)

    def tuning(self) -> dict:
        v = (ctypes.c_int32 * 4)()
        _check(lib().trilens_get_tuning(self.ctx, v), self.ctx)
        return dict(zip(("leaf_bucket", "stack_depth", "block_shape", "budget"), list(v)))

    def autotune(self, steps, cache_path: str | None = None) -> dict:
        st = (ctypes.c_int64 * len(steps))(*[int(x) for x in steps])
        v = (ctypes.c_int32 * 4)()
        _check(lib().trilens_autotune(self.ctx, st, len(steps),
                                      cache_path.encode() if cache_path else None, v), self.ctx)
        return dict(zip(("leaf_bucket", "stack_depth", "block_shape", "budget"), list(v)))

    # ---- learned statistical regime
    def surrogate_collect(self, steps, level_L: int):
        st = (ctypes.c_int64 * len(steps))(*[int(x) for x in steps])
        _check(lib().trilens_surrogate_collect(self.ctx, st, len(steps), int(level_L)), self.ctx)

    def surrogate_fit(self, epochs: int, seed: int = 0):
        _check(lib().trilens_surrogate_fit(self.ctx, int(epochs), int(seed)), self.ctx)

    def surrogate_train(self, steps, level_L: int, epochs: int, seed: int = 0):
        self.surrogate_collect(steps, level_L)
        self.surrogate_fit(epochs, seed)

    def surrogate_step(self, step: int, level_L: int, tau: float = 1e30) -> dict:
        """Build `step` and return the surrogate estimate and its timings."""
        self.build(step)
        v = (ctypes.c_double * 8)()
        _check(lib().trilens_surrogate_step(self.ctx, int(step), int(level_L), float(tau), v),
               self.ctx)
        return dict(zip(("yield", "st_yield", "pairs", "fallback_pairs", "fallback_yield",
                         "ms", "ms_network", "ms_cut"), list(v)))

    def surrogate_pairs(self, step: int, level_L: int, tau: float | None = None,
                        labels: bool = True, cap: int = 1 << 22) -> dict:
        """Build `step` and return its level-L node pairs (trilens_surrogate_pairs):
        cut node ids, features, ST rates, exact labels (labels=True), and with
        tau given the network's outputs, estimates and fallback flags; plus every
        input photon's cut node in each beam."""
        self.build(step)
        na, nb = self.a["px"].numel(), self.b["px"].numel()
        out = {"cloud": np.zeros((cap, 2), np.uint32), "feat": np.zeros((cap, 24), np.float32),
               "st": np.zeros(cap, np.float32), "cloud_of_a": np.zeros(na, np.uint32),
               "cloud_of_b": np.zeros(nb, np.uint32)}
        if labels:
            out["label"] = np.zeros(cap, np.float64)
        if tau is not None:
            out["pred"] = np.zeros(cap, np.float64)
            out["fallback"] = np.zeros(cap, np.uint8)
            out["net"] = np.zeros((cap, 2), np.float32)
        sp = SurPairs(cap, 0, *[out[k].ctypes.data if k in out else None
                                for k in ("cloud", "feat", "st", "label", "pred", "fallback",
                                          "net", "cloud_of_a", "cloud_of_b")], 0.0)
        _check(lib().trilens_surrogate_pairs(self.ctx, int(step), int(level_L),
                                             float(1e30 if tau is None else tau), ctypes.byref(sp)),
               self.ctx)
        n = int(sp.n_pairs)
        if n > cap:
            return self.surrogate_pairs(step, level_L, tau, labels, n)
        res = {k: (v[:n] if k not in ("cloud_of_a", "cloud_of_b") else v) for k, v in out.items()}
        res["n_pairs"] = n
        res["fallback_exact"] = sp.fallback_exact
        return res

    def surrogate_info(self) -> dict:
        v = (ctypes.c_double * 6)()
        _check(lib().trilens_surrogate_info(self.ctx, v), self.ctx)
        return dict(zip(("samples", "loss", "calib", "st_calib", "level", "total"), list(v)))

    def surrogate_dataset(self):
        n = ctypes.c_int64(0)
        _check(lib().trilens_surrogate_dataset(self.ctx, None, None, None, 0, ctypes.byref(n)),
               self.ctx)
        x = np.zeros((n.value, 24), np.float32)
        lab = np.zeros(n.value, np.float64)
        st = np.zeros(n.value, np.float32)
        _check(lib().trilens_surrogate_dataset(
            self.ctx, x.ctypes.data_as(ctypes.c_void_p), lab.ctypes.data_as(ctypes.c_void_p),
            st.ctypes.data_as(ctypes.c_void_p), n.value, ctypes.byref(n)), self.ctx)
        return x, lab, st

    def surrogate_add_samples(self, x, label, st, level_L: int):
        x = np.ascontiguousarray(x, np.float32)
        label = np.ascontiguousarray(label, np.float64)
        st = np.ascontiguousarray(st, np.float32)
        _check(lib().trilens_surrogate_add_samples(
            self.ctx, x.ctypes.data_as(ctypes.c_void_p), label.ctypes.data_as(ctypes.c_void_p),
            st.ctypes.data_as(ctypes.c_void_p), len(label), int(level_L)), self.ctx)

    def surrogate_save(self, path: str):
        _check(lib().trilens_surrogate_save(self.ctx, path.encode()), self.ctx)

    def surrogate_load(self, path: str):
        _check(lib().trilens_surrogate_load(self.ctx, path.encode()), self.ctx)

    def deplete_step(self, step: int, hits, n_hits: int, rem_a, rem_b, delta=None) -> dict:
        """Depletion in time order of step `step`'s hits (trilens_deplete_step): hits an
        int32 CUDA tensor holding >= 2*n_hits entries ((i, j) pairs as collide wrote them),
        rem_a / rem_b float64 CUDA tensors (one entry per photon of beam a / b, updated in
        place), delta an optional float64 CUDA tensor of >= n_hits entries.  Returns
        {"accepted", "transferred", "rounds"}."""
        n_hits = int(n_hits)
        na, nb = int(self.a["px"].numel()), int(self.b["px"].numel())
        for name, t, n in (("rem_a", rem_a, na), ("rem_b", rem_b, nb)):
            if not (t.is_cuda and t.dtype == self._torch.float64 and t.is_contiguous()
                    and t.numel() == n):
                raise TrilensError(ERR_INVALID, f"{name}: need {n} contiguous float64 on the GPU")
        if n_hits > 0 and not (hits.is_cuda and hits.element_size() == 4 and hits.is_contiguous()
                               and hits.numel() >= 2 * n_hits):
            raise TrilensError(ERR_INVALID, "hits: need >= 2*n_hits contiguous 32-bit entries")
        if delta is not None and not (delta.is_cuda and delta.dtype == self._torch.float64
                                      and delta.is_contiguous() and delta.numel() >= n_hits):
            raise TrilensError(ERR_INVALID, "delta: need >= n_hits contiguous float64")
        acc = ctypes.c_int64(0)
        tr = ctypes.c_double(0.0)
        ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
        _check(lib().trilens_deplete_step(self.ctx, int(step), ptr(hits) if n_hits else None,
                                          n_hits, ptr(rem_a), ptr(rem_b), ptr(delta),
                                          ctypes.byref(acc), ctypes.byref(tr)), self.ctx)
        r = ctypes.c_int64(0)
        _check(lib().trilens_deplete_rounds(self.ctx, ctypes.byref(r)), self.ctx)
        return {"accepted": int(acc.value), "transferred": float(tr.value),
                "rounds": int(r.value) if n_hits else 0}

    def deplete_step_async(self, step: int, hits, n_hits: int, rem_a, rem_b, delta, out):
        """trilens_deplete_step_async: enqueue the depletion of step `step` on the
        context's stream; its record goes to `out`, a CUDA int64 tensor of >= 4
        entries (see deplete_record).  Same arguments as deplete_step."""
        n_hits = int(n_hits)
        if not (out.is_cuda and out.dtype == self._torch.int64 and out.is_contiguous()
                and out.numel() >= 4):
            raise TrilensError(ERR_INVALID, "out: need >= 4 contiguous int64 on the GPU")
        na, nb = int(self.a["px"].numel()), int(self.b["px"].numel())
        for name, t, n in (("rem_a", rem_a, na), ("rem_b", rem_b, nb)):
            if not (t.is_cuda and t.dtype == self._torch.float64 and t.is_contiguous()
                    and t.numel() == n):
                raise TrilensError(ERR_INVALID, f"{name}: need {n} contiguous float64 on the GPU")
        if n_hits > 0 and not (hits.is_cuda and hits.element_size() == 4 and hits.is_contiguous()
                               and hits.numel() >= 2 * n_hits):
            raise TrilensError(ERR_INVALID, "hits: need >= 2*n_hits contiguous 32-bit entries")
        ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
        _check(lib().trilens_deplete_step_async(self.ctx, int(step), ptr(hits) if n_hits else None,
                                                n_hits, ptr(rem_a), ptr(rem_b), ptr(delta),
                                                ptr(out)), self.ctx)

    def debug_set_parts(self, parts: int):
        _check(lib().trilens_debug_set_parts(self.ctx, int(parts)), self.ctx)

    def debug_set_spin_limit(self, limit: int):
        _check(lib().trilens_debug_set_spin_limit(self.ctx, int(limit)), self.ctx)

    def debug_set_cut_cap(self, cap: int):
        _check(lib().trilens_debug_set_cut_cap(self.ctx, int(cap)), self.ctx)

    def debug_set_key_bits(self, bits: int):
        _check(lib().trilens_debug_set_key_bits(self.ctx, int(bits)), self.ctx)

    def debug_shrink_buffers(self, cap: int = 64):
        _check(lib().trilens_debug_shrink_buffers(self.ctx, int(cap)), self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            lib().trilens_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _is_dev(b: dict) -> bool:
    v = b.get("px")
    return hasattr(v, "is_cuda") and v.is_cuda


def eval64(x, which: str = "sigma", stream=None):
    """Device FP64 sigma(s) or ln(x) of the exact decision, element-wise on a
    float64 CUDA tensor (for bit-exact comparison with a CPU implementation)."""
    torch = _torch()
    assert x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()
    out = torch.empty_like(x)
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().trilens_debug_eval64(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                      x.numel(), 0 if which == "sigma" else 1,
                                      ctypes.c_void_p(st.cuda_stream)))
    return out


STRESS_CATEGORIES, STRESS_FIELDS, STRESS_SAMPLE = 8, 7, 17
STRESS_FIELD_NAMES = ("pairs", "fp64_hits", "fp32_sure_hits", "fp32_sure_misses", "fp32_band",
                      "wrong_sure_hits", "wrong_sure_misses")


def band_stress(seed: int, n_pairs: int, dt_fs: float, kappa: float, n_sample: int = 0,
                stream=None):
    """Seeded near-boundary photon pairs decided by the FP32 narrow phase and
    the FP64 definition on the device (trilens_debug_band_stress).  Returns
    (counts[8 categories, 7 fields] as numpy uint64, sample[n_sample, 17] as
    numpy float64 or None)."""
    torch = _torch()
    st = stream if stream is not None else torch.cuda.current_stream()
    counts = torch.zeros(STRESS_CATEGORIES * STRESS_FIELDS, dtype=torch.int64, device="cuda")
    sample = (torch.empty((n_sample, STRESS_SAMPLE), dtype=torch.float64, device="cuda")
              if n_sample > 0 else None)
    _check(lib().trilens_debug_band_stress(
        ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), int(n_pairs), float(dt_fs), float(kappa),
        ctypes.c_void_p(counts.data_ptr()),
        ctypes.c_void_p(sample.data_ptr()) if sample is not None else None, int(n_sample),
        ctypes.c_void_p(st.cuda_stream)))
    torch.cuda.synchronize()
    c = counts.cpu().numpy().view(np.uint64).reshape(STRESS_CATEGORIES, STRESS_FIELDS)
    return c, (sample.cpu().numpy() if sample is not None else None)


NOALLOC_MAX_HITS = 1 << 28


def yield_reduce_noalloc(hits, n_hits: int, w_a=None, w_b=None, out=None, stream=None):
    """Reduce a device hit list (int32 tensor of >= 2*n_hits entries) without
    any device allocation inside the library: returns a 4-element int64 CUDA
    tensor holding (count, weighted as float64 bits, checksum sum, checksum
    xor); pass `out` (4 int64 on the device) to avoid torch allocating it."""
    torch = _torch()
    if n_hits < 0 or n_hits > NOALLOC_MAX_HITS:
        raise TrilensError(ERR_INVALID, f"n_hits={n_hits} outside [0, {NOALLOC_MAX_HITS}]")
    if out is None:
        out = torch.zeros(4, dtype=torch.int64, device=hits.device)
    st = stream if stream is not None else torch.cuda.current_stream()
    ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
    _check(lib().trilens_yield_reduce_noalloc(ptr(hits), int(n_hits), ptr(w_a), ptr(w_b), ptr(out),
                                             ctypes.c_void_p(st.cuda_stream)))
    return out


def pair_products(beam_a: dict, beam_b: dict, hits, seed: int, out=None, stream=None):
    """Electron and positron four-momenta [MeV] of each hit (trilens_pair_products):
    beams as device tensors (to_device), hits an (n, 2) int32 CUDA tensor of
    (i, j); returns an (n, 8) float64 CUDA tensor = electron (E, px, py, pz),
    positron (E, px, py, pz)."""
    torch = _torch()
    n = int(hits.shape[0]) if hits.dim() == 2 else int(hits.numel() // 2)
    if out is None:
        out = torch.empty((n, 8), dtype=torch.float64, device=hits.device)
    st = stream if stream is not None else torch.cuda.current_stream()
    ba, bb = beam_struct(beam_a), beam_struct(beam_b)
    _check(lib().trilens_pair_products(ctypes.byref(ba), ctypes.byref(bb),
                                       ctypes.c_void_p(hits.data_ptr()), n,
                                       ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF),
                                       ctypes.c_void_p(out.data_ptr()),
                                       ctypes.c_void_p(st.cuda_stream)))
    return out


def swarm_mark(mp_a: dict, mp_b: dict, h_a: float, h_b: float, dt_fs: float, kappa: float,
               first_step: int, steps: int, stream=None):
    """trilens_swarm_mark: uint8 CUDA tensors (mark_a, mark_b), 1 for the
    macro-photons of pairs that can collide in the given steps."""
    torch = _torch()
    st = stream if stream is not None else torch.cuda.current_stream()
    ba, bb = beam_struct(mp_a), beam_struct(mp_b)
    dev = mp_a["px"].device
    na, nb = int(mp_a["px"].numel()), int(mp_b["px"].numel())
    mark_a = torch.zeros(max(na, 1), dtype=torch.uint8, device=dev)
    mark_b = torch.zeros(max(nb, 1), dtype=torch.uint8, device=dev)
    params = Params(float(dt_fs), float(kappa), FP32_BAND, 0, 0, 0, 0)
    _check(lib().trilens_swarm_mark(ctypes.byref(ba), ctypes.byref(bb), float(h_a), float(h_b),
                                    ctypes.byref(params), int(first_step), int(steps),
                                    ctypes.c_void_p(mark_a.data_ptr()),
                                    ctypes.c_void_p(mark_b.data_ptr()),
                                    ctypes.c_void_p(st.cuda_stream)))
    return mark_a[:na], mark_b[:nb]


def swarm_split(mp_a: dict, mp_b: dict, h_a: float, h_b: float, dt_fs: float, kappa: float,
                first_step: int, steps: int, stream=None) -> dict:
    """IP regime (trilens_swarm_mark / _count / _expand): the real photons of the
    macro-photons that can collide in the given steps.  mp_a / mp_b: beams of MPs
    (device tensors, integer weights); h_a / h_b: the MPs' cube sides [um].
    Returns {"a", "b": the real-photon beams (device tensors, weight 1),
    "owner_a", "k_a", "owner_b", "k_b": int32 tensors mapping each real photon to
    its MP and its index in the swarm, "mark_a", "mark_b": uint8 tensors}."""
    torch = _torch()
    st = stream if stream is not None else torch.cuda.current_stream()
    sp = ctypes.c_void_p(st.cuda_stream)
    ba, bb = beam_struct(mp_a), beam_struct(mp_b)
    dev = mp_a["px"].device
    mark_a, mark_b = swarm_mark(mp_a, mp_b, h_a, h_b, dt_fs, kappa, first_step, steps, st)
    out = {"mark_a": mark_a, "mark_b": mark_b}
    for side, mp, bs, mark, h in (("a", mp_a, ba, mark_a, h_a), ("b", mp_b, bb, mark_b, h_b)):
        n = int(mp["px"].numel())
        off = torch.empty(n + 1, dtype=torch.int64, device=dev)
        total = ctypes.c_int64(0)
        _check(lib().trilens_swarm_count(ctypes.byref(bs), ctypes.c_void_p(mark.data_ptr()),
                                         ctypes.c_void_p(off.data_ptr()), ctypes.byref(total), sp))
        m = int(total.value)
        beam = {k: torch.empty(m, dtype=torch.float64, device=dev) for k in BEAM_KEYS}
        owner = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
        kof = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
        ptrs = (ctypes.c_void_p * 8)(*[ctypes.c_void_p(beam[k].data_ptr() if m else None)
                                       for k in BEAM_KEYS])
        _check(lib().trilens_swarm_expand(ctypes.byref(bs), float(h), ctypes.c_void_p(off.data_ptr()),
                                          m, ptrs, ctypes.c_void_p(owner.data_ptr()),
                                          ctypes.c_void_p(kof.data_ptr()), sp))
        out[side] = beam
        out["owner_" + side] = owner[:m]
        out["k_" + side] = kof[:m]
    return out


class Batch(Collider):
    """Many independent instances (pairs of beams) in one context.

    ``run(first, steps)`` executes the steps of every instance as one captured
    CUDA graph and returns per-instance (count, sum w w) as an (n_inst, 2)
    numpy array.  ``build``/``collide``/``step_hits`` work on the
    concatenation (photon indices are positions in it)."""

    def __init__(self, beams_a: list, beams_b: list, dt_fs: float, kappa: float,
                 precision: int = FP32_BAND, leaf_bucket: int = 0, stack_depth: int = 0,
                 block_shape: int = 0, spin_limit: int = 0, stream=None):
        torch = _torch()
        self._torch = torch
        assert len(beams_a) == len(beams_b) and len(beams_a) >= 1
        self.n_inst = len(beams_a)
        self.inst_a = [x if _is_dev(x) else to_device(x) for x in beams_a]
        self.inst_b = [x if _is_dev(x) else to_device(x) for x in beams_b]
        self.a, self.b = self.inst_a[0], self.inst_b[0]
        self.params = Params(float(dt_fs), float(kappa), int(precision), int(leaf_bucket),
                             int(stack_depth), int(block_shape), int(spin_limit))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        arr_a = (Beam * self.n_inst)(*[beam_struct(x) for x in self.inst_a])
        arr_b = (Beam * self.n_inst)(*[beam_struct(x) for x in self.inst_b])
        h = ctypes.c_void_p()
        _check(lib().trilens_batch_create(ctypes.byref(h), arr_a, arr_b, self.n_inst,
                                          ctypes.byref(self.params),
                                          ctypes.c_void_p(self.stream.cuda_stream)))
        self.ctx = h
        self.offsets_a = np.cumsum([0] + [int(x["px"].numel()) for x in self.inst_a])
        self.offsets_b = np.cumsum([0] + [int(x["px"].numel()) for x in self.inst_b])
        self.yields = torch.zeros((self.n_inst, 2), dtype=torch.float64,
                                  device=self.inst_a[0]["px"].device)

    def run(self, first_step: int, steps: int):
        _check(lib().trilens_batch_run(self.ctx, int(first_step), int(steps),
                                       ctypes.c_void_p(self.yields.data_ptr())), self.ctx)
        return self.yields.cpu().numpy().copy()


MLP_PARAMS = 36482
MLP_ORDER = (("W1", (128, 24)), ("b1", (128,)), ("W2", (128, 128)), ("b2", (128,)),
             ("W3", (128, 128)), ("b3", (128,)), ("W4", (2, 128)), ("b4", (2,)))


def mlp_flatten(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[k], dtype=np.float64).reshape(-1) for k, _ in MLP_ORDER])


def mlp_unflatten(v) -> dict:
    v = np.asarray(v)
    out, off = {}, 0
    for k, shp in MLP_ORDER:
        n = int(np.prod(shp))
        out[k] = v[off:off + n].reshape(shp)
        off += n
    return out


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def mlp_forward(params, norm, x, stream=None):
    """Network outputs (m, 2) for device FP32 tensors params, norm (48), x (m, 24)."""
    torch = _torch()
    out = torch.empty((x.shape[0], 2), dtype=torch.float32, device=x.device)
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().trilens_mlp_forward(_ptr(params), _ptr(norm), _ptr(x), x.shape[0], _ptr(out),
                                     ctypes.c_void_p(st.cuda_stream)))
    return out


#: bins of s of the narrow phase's sure-miss radii (trilens_debug_narrow_bins)
NARROW_BINS = 193


def narrow_bins(dt_fs: float, kappa: float):
    """(upper bounds of r^2 per bin of s [um^2], as float32, and the bound over every
    s): the table the FP32 narrow phase's quick miss uses (host only)."""
    out = np.zeros(NARROW_BINS, dtype=np.float32)
    r2max = ctypes.c_float(0.0)
    rc = lib().trilens_debug_narrow_bins(float(dt_fs), float(kappa),
                                         ctypes.c_void_p(out.ctypes.data), NARROW_BINS,
                                         ctypes.byref(r2max))
    if rc != NARROW_BINS:
        raise TrilensError(rc, status_str(rc))
    return out, float(r2max.value)


def deplete_record(out) -> dict:
    """The record(s) trilens_deplete_step_async wrote: `out` an int64 tensor of
    shape (4,) or (m, 4) -> dict (or list of dicts) with transferred, accepted,
    rounds and status (0 = OK, else a TRILENS_ERR_* code)."""
    a = np.ascontiguousarray(out.cpu().numpy().astype(np.int64).reshape(-1, 4))
    recs = [{"transferred": float(r[:1].view(np.float64)[0]), "accepted": int(r[1]),
             "rounds": int(r[2]), "status": int(r[3])} for r in a]
    return recs[0] if out.dim() == 1 else recs


def mlp_grad(params, norm, x, y, stream=None, kind=0, baseline=None, scale=1.0):
    """(gradient of the mean loss, summed loss) for device FP32 tensors;
    kind 1 is the surrogate's objective with baseline (m,) and its scale."""
    torch = _torch()
    g = torch.empty(MLP_PARAMS, dtype=torch.float32, device=x.device)
    loss = torch.empty(1, dtype=torch.float32, device=x.device)
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().trilens_mlp_grad(_ptr(params), _ptr(norm), _ptr(x), _ptr(y),
                                  _ptr(baseline) if baseline is not None else None,
                                  float(scale), int(kind), x.shape[0], _ptr(g), _ptr(loss),
                                  ctypes.c_void_p(st.cuda_stream)))
    return g, loss
