"""Python binding of the GB300 cortical-microcircuit library (``include/snn.h``).

Argument marshalling only: every step of the simulation runs in the CUDA
kernels of ``libsnn_gb300.so``.  The functions keep the C names
(``snn_create``, ``snn_step`` ...); :class:`Microcircuit` wraps one network
handle.  There is no CPU fallback: importing the binding without the built
library, or calling it without a CUDA device, raises.

Device memory and streams may come from PyTorch: pass
``torch.cuda.current_stream().cuda_stream`` as the stream, and device
tensors' ``data_ptr()`` where the ABI takes device pointers.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsnn_gb300.so")
MAX_POP = 8
WCODES = 128
RING_DEPTH = 64

SNN_OK, SNN_ERR_INVALID, SNN_ERR_CUDA, SNN_ERR_OOM = 0, 1, 2, 3
SNN_ERR_TIMEOUT, SNN_ERR_OVERFLOW, SNN_ERR_UNSUPPORTED, SNN_ERR_SATURATED = 4, 5, 6, 7
_ERR_NAMES = {1: "INVALID", 2: "CUDA", 3: "OOM", 4: "TIMEOUT", 5: "OVERFLOW", 6: "UNSUPPORTED",
              7: "SATURATED"}


class SnnError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("SNN_ERR_%s: %s" % (_ERR_NAMES.get(code, code), msg))
        self.code = code


class SnnConfig(C.Structure):
    _fields_ = [
        ("n_pop", C.c_int32),
        ("pop_size", C.c_int32 * MAX_POP),
        ("pop_exc", C.c_int32 * MAX_POP),
        ("conn_prob", (C.c_double * MAX_POP) * MAX_POP),
        ("conn_scale", C.c_double),
        ("w_mean", (C.c_double * MAX_POP) * MAX_POP),
        ("w_sd", (C.c_double * MAX_POP) * MAX_POP),
        ("w_scale", C.c_double),
        ("proj_scale", (C.c_double * MAX_POP) * MAX_POP),
        ("d_mean", C.c_double * MAX_POP),
        ("d_sd", C.c_double * MAX_POP),
        ("k_ext", C.c_double * MAX_POP),
        ("nu_bg", C.c_double),
        ("w_ext", C.c_double),
        ("i_dc", C.c_double * MAX_POP),
        ("input_mode", C.c_int32),
        ("tau_m", C.c_double),
        ("c_m", C.c_double),
        ("tau_syn", C.c_double),
        ("t_ref", C.c_double),
        ("theta", C.c_double),
        ("dt", C.c_double),
        ("u0_lo", C.c_double),
        ("u0_hi", C.c_double),
        ("ring_depth", C.c_int32),
    ]


class SnnOptions(C.Structure):
    _fields_ = [("n_part", C.c_int32), ("inject_fault", C.c_int32),
                ("raster_capacity", C.c_int64), ("timeout_s", C.c_double)]


class SnnInfo(C.Structure):
    _fields_ = [("n_neurons", C.c_int64), ("n_synapses", C.c_int64), ("n_part", C.c_int32),
                ("threads", C.c_int32), ("neurons_per_thread", C.c_int32),
                ("ring_in_shared", C.c_int32), ("max_part_neurons", C.c_int32),
                ("n_ref", C.c_int32), ("propagators", C.c_float * 4), ("wext_q", C.c_int32),
                ("shared_bytes", C.c_int32), ("slot_entries", C.c_int32),
                ("slot_bytes", C.c_int64), ("deliver_clusters_active", C.c_int32),
                ("saturation_check", C.c_int32), ("input_bound", C.c_int64)]


class SnnNoallocIO(C.Structure):
    """Device pointers of ``snn_step_noalloc`` (all caller-owned)."""
    _fields_ = [("row_ptr", C.c_void_p), ("words", C.c_void_p), ("wtab", C.c_void_p),
                ("u", C.c_void_p), ("i_syn", C.c_void_p), ("refr", C.c_void_p),
                ("ring", C.c_void_p), ("ras_step", C.c_void_p), ("ras_id", C.c_void_p),
                ("ras_n", C.c_void_p), ("ras_cap", C.c_int64), ("counters", C.c_void_p),
                ("status", C.c_void_p)]


class SnnBatchInfo(C.Structure):
    _fields_ = [("n_instances", C.c_int32), ("n_neurons_total", C.c_int32),
                ("n_neurons", C.c_int32), ("n_synapses", C.c_int64), ("tiling", C.c_int32),
                ("tune_us_warp", C.c_float), ("tune_us_block", C.c_float),
                ("tune_us_flat", C.c_float), ("trial_us_per_step", C.c_float),
                ("blocks", C.c_int32), ("threads", C.c_int32),
                ("neurons_per_thread", C.c_int32), ("graph", C.c_int32),
                ("graph_steps", C.c_int32)]


NOALLOC_MAX_NEURONS = 131072

EXPORTED = ["snn_create", "snn_create_from_rows", "snn_step", "snn_sync", "snn_read_spikes",
            "snn_raster_size", "snn_read_state", "snn_read_ring", "snn_counters", "snn_get_info",
            "snn_export_network", "snn_deliver", "snn_step_noalloc", "snn_record_step_times",
            "snn_record_step_counts",
            "snn_set_realtime", "snn_realtime_stats", "snn_save_state",
            "snn_load_state", "snn_set_params", "snn_grad_forward", "snn_grad_backward",
            "snn_grad_set_trace_budget",
            "snn_batch_create",
            "snn_batch_step", "snn_batch_sync", "snn_batch_read_spikes", "snn_batch_read_state",
            "snn_batch_counters", "snn_batch_get_info", "snn_batch_set_tiling",
            "snn_batch_destroy", "snn_destroy",
            "snn_last_error"]

_lib = None


def lib():
    """Load ``libsnn_gb300.so`` (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libsnn_gb300.so is not built; run "
                              "python -c 'import __graft_entry__ as g; g.build()'")
        L = C.CDLL(LIB_PATH)
        P = C.POINTER
        vp = C.c_void_p
        L.snn_create.argtypes = [P(SnnConfig), C.c_uint64, P(SnnOptions), P(C.c_float), vp, P(vp)]
        L.snn_create_from_rows.argtypes = [P(SnnConfig), C.c_uint64, P(SnnOptions),
                                           P(C.c_uint64), P(C.c_uint32), P(C.c_int32),
                                           P(C.c_float), vp, P(vp)]
        L.snn_step.argtypes = [vp, C.c_int64]
        L.snn_sync.argtypes = [vp]
        L.snn_read_spikes.argtypes = [vp, P(C.c_uint32), P(C.c_uint32), C.c_int64, P(C.c_int64)]
        L.snn_raster_size.argtypes = [vp, P(C.c_int64)]
        L.snn_read_state.argtypes = [vp, P(C.c_float), P(C.c_float), P(C.c_int32)]
        L.snn_read_ring.argtypes = [vp, P(C.c_int32)]
        L.snn_counters.argtypes = [vp, P(C.c_int64), P(C.c_uint64), P(C.c_uint64)]
        L.snn_get_info.argtypes = [vp, P(SnnInfo)]
        L.snn_export_network.argtypes = [vp, P(C.c_uint64), P(C.c_uint32), P(C.c_int32)]
        L.snn_deliver.argtypes = [vp, vp, C.c_int32, C.c_int64, C.c_int32]
        L.snn_step_noalloc.argtypes = [P(SnnConfig), C.c_uint64, P(SnnNoallocIO), C.c_int64,
                                       C.c_int64, vp]
        L.snn_record_step_times.argtypes = [vp, vp, C.c_int64]
        L.snn_record_step_counts.argtypes = [vp, vp, C.c_int64]
        L.snn_set_realtime.argtypes = [vp, C.c_int64]
        L.snn_realtime_stats.argtypes = [vp, P(C.c_int64), P(C.c_int64)]
        L.snn_save_state.argtypes = [vp, vp, C.c_int64, P(C.c_int64)]
        L.snn_load_state.argtypes = [vp, vp, C.c_int64]
        L.snn_set_params.argtypes = [vp, P(C.c_double), C.c_double]
        L.snn_grad_forward.argtypes = [vp, C.c_int64, C.c_int32, P(C.c_double)]
        L.snn_grad_backward.argtypes = [vp, P(C.c_double), P(C.c_double), P(C.c_double)]
        L.snn_grad_set_trace_budget.argtypes = [vp, C.c_int64]
        L.snn_batch_create.argtypes = [P(SnnConfig), P(C.c_uint64), C.c_int32, P(SnnOptions),
                                       vp, P(vp)]
        L.snn_batch_step.argtypes = [vp, C.c_int64]
        L.snn_batch_sync.argtypes = [vp]
        L.snn_batch_read_spikes.argtypes = [vp, C.c_int32, P(C.c_uint32), P(C.c_uint32),
                                            C.c_int64, P(C.c_int64)]
        L.snn_batch_read_state.argtypes = [vp, C.c_int32, P(C.c_float), P(C.c_float),
                                           P(C.c_int32)]
        L.snn_batch_counters.argtypes = [vp, C.c_int32, P(C.c_int64), P(C.c_uint64),
                                         P(C.c_uint64)]
        L.snn_batch_get_info.argtypes = [vp, C.c_int32, P(SnnBatchInfo)]
        L.snn_batch_set_tiling.argtypes = [vp, C.c_int32, C.c_int32]
        L.snn_batch_destroy.argtypes = [vp]
        L.snn_destroy.argtypes = [vp]
        L.snn_last_error.restype = C.c_char_p
        for name in EXPORTED:
            if name != "snn_last_error":
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(rc):
    if rc != SNN_OK:
        raise SnnError(rc, lib().snn_last_error().decode())


def _ptr(a, ctype):
    return None if a is None else a.ctypes.data_as(C.POINTER(ctype))


def make_config(cfg: dict) -> SnnConfig:
    """Fill an ``snn_config`` from a configuration dictionary."""
    c = SnnConfig()
    npop = len(cfg["pop_sizes"])
    if not 1 <= npop <= MAX_POP:
        raise ValueError("1..8 populations")
    c.n_pop = npop
    for p in range(npop):
        c.pop_size[p] = int(cfg["pop_sizes"][p])
        c.pop_exc[p] = int(cfg["pop_exc"][p])
        c.d_mean[p] = float(cfg["d_mean"][p])
        c.d_sd[p] = float(cfg["d_sd"][p])
        c.k_ext[p] = float(cfg["k_ext"][p])
        c.i_dc[p] = float(cfg["i_dc"][p])
        for q in range(npop):
            c.conn_prob[p][q] = float(cfg["conn_prob"][p][q])
            c.w_mean[p][q] = float(cfg["w_mean"][p][q])
            c.w_sd[p][q] = float(cfg["w_sd"][p][q])
            c.proj_scale[p][q] = float(cfg["proj_scale"][p][q])
    c.conn_scale = float(cfg["conn_scale"])
    c.w_scale = float(cfg["w_scale"])
    c.nu_bg = float(cfg["nu_bg"])
    c.w_ext = float(cfg["w_ext"])
    c.input_mode = int(cfg["input_mode"])
    for k in ("tau_m", "c_m", "tau_syn", "t_ref", "theta", "dt", "u0_lo", "u0_hi"):
        setattr(c, k, float(cfg[k]))
    c.ring_depth = int(cfg["ring_depth"])
    return c


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)          # torch.cuda.Stream


class Microcircuit:
    """One simulated network on the current CUDA device."""

    def __init__(self, cfg: dict, seed: int | None = None, u0=None, n_part: int = 0,
                 raster_capacity: int = 0, timeout_s: float = 0.0, stream=None,
                 rows: dict | None = None, inject_fault: int = 0):
        self.cfg = cfg
        self.seed = int(cfg["seed"] if seed is None else seed)
        self._c = make_config(cfg)
        self._o = SnnOptions(int(n_part), int(inject_fault), int(raster_capacity),
                             float(timeout_s))
        self.n = int(sum(cfg["pop_sizes"]))
        self._u0 = None if u0 is None else np.ascontiguousarray(u0, np.float32)
        if self._u0 is not None and self._u0.size != self.n:
            raise ValueError("u0 must have one value per neuron")
        self.stream = _stream_handle(stream)
        h = C.c_void_p()
        L = lib()
        if rows is None:
            rc = L.snn_create(C.byref(self._c), self.seed, C.byref(self._o),
                              _ptr(self._u0, C.c_float), self.stream, C.byref(h))
        else:
            rp = np.ascontiguousarray(rows["row_ptr"], np.uint64)
            wd = np.ascontiguousarray(rows["words"], np.uint32)
            wt = np.ascontiguousarray(rows["wtab"], np.int32).reshape(-1)
            rc = L.snn_create_from_rows(C.byref(self._c), self.seed, C.byref(self._o),
                                        _ptr(rp, C.c_uint64), _ptr(wd, C.c_uint32),
                                        _ptr(wt, C.c_int32), _ptr(self._u0, C.c_float),
                                        self.stream, C.byref(h))
        _check(rc)
        self._h = h

    # -- stepping ------------------------------------------------------------
    def step(self, n_steps: int):
        _check(lib().snn_step(self._h, int(n_steps)))

    def sync(self):
        _check(lib().snn_sync(self._h))

    def deliver(self, spikes_dev_ptr: int, n_spikes: int, t: int, tiling: int = 0):
        _check(lib().snn_deliver(self._h, C.c_void_p(int(spikes_dev_ptr)), int(n_spikes),
                                 int(t), int(tiling)))

    # -- reads ---------------------------------------------------------------
    def info(self) -> dict:
        i = SnnInfo()
        _check(lib().snn_get_info(self._h, C.byref(i)))
        return {k: (list(getattr(i, k)) if k == "propagators" else getattr(i, k))
                for k, _ in SnnInfo._fields_}

    def read_spikes(self, cap: int | None = None):
        """Drain the device raster; returns (steps, ids) sorted by (step, id)."""
        if cap is None:
            cap = max(1, self.raster_size())
        st = np.zeros(cap, np.uint32)
        ids = np.zeros(cap, np.uint32)
        n = C.c_int64()
        _check(lib().snn_read_spikes(self._h, _ptr(st, C.c_uint32), _ptr(ids, C.c_uint32),
                                     int(cap), C.byref(n)))
        st, ids = st[:n.value], ids[:n.value]
        order = np.lexsort((ids, st))
        return st[order].astype(np.int64), ids[order].astype(np.int64)

    def raster_size(self) -> int:
        n = C.c_int64()
        _check(lib().snn_raster_size(self._h, C.byref(n)))
        return n.value

    def read_spikes_into(self, steps_buf: np.ndarray, ids_buf: np.ndarray) -> int:
        """Drain the raster into caller-provided uint32 host buffers (unsorted)."""
        n = C.c_int64()
        _check(lib().snn_read_spikes(self._h, _ptr(steps_buf, C.c_uint32),
                                     _ptr(ids_buf, C.c_uint32), int(steps_buf.size),
                                     C.byref(n)))
        return n.value

    def state(self):
        u = np.zeros(self.n, np.float32)
        i = np.zeros(self.n, np.float32)
        r = np.zeros(self.n, np.int32)
        _check(lib().snn_read_state(self._h, _ptr(u, C.c_float), _ptr(i, C.c_float),
                                    _ptr(r, C.c_int32)))
        return u, i, r

    def ring(self):
        out = np.zeros(RING_DEPTH * self.n, np.int32)
        _check(lib().snn_read_ring(self._h, _ptr(out, C.c_int32)))
        return out.reshape(RING_DEPTH, self.n)

    def counters(self) -> dict:
        s, a, b = C.c_int64(), C.c_uint64(), C.c_uint64()
        _check(lib().snn_counters(self._h, C.byref(s), C.byref(a), C.byref(b)))
        return {"step": s.value, "spikes": a.value, "events": b.value}

    def record_step_times(self, times_dev_ptr: int | None, cap: int = 0):
        """Device int64 buffer (data_ptr) receiving the clock (ns) at the end
        of each following step; None stops recording."""
        _check(lib().snn_record_step_times(self._h, None if times_dev_ptr is None
                                           else C.c_void_p(int(times_dev_ptr)), int(cap)))

    def record_step_counts(self, counts_dev_ptr: int | None, cap: int = 0):
        """Device uint32 buffer (data_ptr) of 4 * cap words receiving, for each
        following step, [spikes, synaptic events, busiest partition's
        spikes, empty (spike, partition) pairs]; None stops recording."""
        _check(lib().snn_record_step_counts(self._h, None if counts_dev_ptr is None
                                            else C.c_void_p(int(counts_dev_ptr)), int(cap)))

    def set_realtime(self, period_ns: int):
        """Pace the following steps to wall-clock time: one step per period_ns
        (100_000 for the paper's true real time at dt = 0.1 ms); 0 stops."""
        _check(lib().snn_set_realtime(self._h, int(period_ns)))

    def realtime_stats(self) -> dict:
        """Deadlines missed since set_realtime and the largest lateness (ns)."""
        m, late = C.c_int64(), C.c_int64()
        _check(lib().snn_realtime_stats(self._h, C.byref(m), C.byref(late)))
        return {"missed": m.value, "max_late_ns": late.value}

    # -- state, parameters, gradient -------------------------------------------
    def save_state(self) -> np.ndarray:
        """The dynamic state as bytes (uint8 array) for :meth:`load_state`."""
        n = C.c_int64()
        L = lib()
        _check(L.snn_save_state(self._h, None, 0, C.byref(n)))
        buf = np.zeros(n.value, np.uint8)
        _check(L.snn_save_state(self._h, buf.ctypes.data, buf.size, C.byref(n)))
        return buf

    def load_state(self, buf: np.ndarray):
        buf = np.ascontiguousarray(buf, np.uint8)
        _check(lib().snn_load_state(self._h, buf.ctypes.data, buf.size))

    def set_params(self, scales, nu_bg: float):
        """Projection weight scales [8][8] (target, source) and background rate."""
        a = np.ascontiguousarray(np.asarray(scales, np.float64).reshape(MAX_POP * MAX_POP))
        _check(lib().snn_set_params(self._h, _ptr(a, C.c_double), float(nu_bg)))

    def grad_forward(self, n_steps: int, ckpt_every: int = 100) -> np.ndarray:
        """Run with checkpoints; population rates (Hz, one per population)."""
        r = np.zeros(MAX_POP, np.float64)
        _check(lib().snn_grad_forward(self._h, int(n_steps), int(ckpt_every), _ptr(r, C.c_double)))
        return r[:len(self.cfg["pop_sizes"])]

    def set_grad_trace_budget(self, n_bytes: int):
        """Largest whole-forward trajectory kept for the backward (bytes)."""
        _check(lib().snn_grad_set_trace_budget(self._h, int(n_bytes)))

    def grad_backward(self, g_rate):
        """dL/dalpha [8][8] and dL/dnu for g_rate = dL/d(rates)."""
        g = np.zeros(MAX_POP, np.float64)
        gr = np.asarray(g_rate, np.float64).reshape(-1)
        g[:gr.size] = gr
        ga = np.zeros(MAX_POP * MAX_POP, np.float64)
        gn = C.c_double()
        _check(lib().snn_grad_backward(self._h, _ptr(g, C.c_double), _ptr(ga, C.c_double),
                                       C.byref(gn)))
        return ga.reshape(MAX_POP, MAX_POP), gn.value

    def export_network(self, rows_only: bool = False):
        """(row_ptr, words, wtab); words is None with rows_only."""
        inf = self.info()
        rp = np.zeros(self.n + 1, np.uint64)
        wd = None if rows_only else np.zeros(max(int(inf["n_synapses"]), 1), np.uint32)
        wt = np.zeros(MAX_POP * MAX_POP * WCODES, np.int32)
        _check(lib().snn_export_network(self._h, _ptr(rp, C.c_uint64), _ptr(wd, C.c_uint32),
                                        _ptr(wt, C.c_int32)))
        words = None if rows_only else wd[:int(inf["n_synapses"])]
        return rp, words, wt.reshape(MAX_POP, MAX_POP, WCODES)

    def close(self):
        if getattr(self, "_h", None):
            lib().snn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MicrocircuitBatch:
    """Many independent networks (own configuration and seed each) stepped
    together by one persistent kernel replayed from a CUDA graph."""

    def __init__(self, cfgs: list, seeds: list | None = None, raster_capacity: int = 0,
                 timeout_s: float = 0.0, stream=None, inject_fault: int = 0):
        if not cfgs:
            raise ValueError("at least one configuration")
        self.cfgs = list(cfgs)
        self.seeds = [int(c["seed"]) for c in cfgs] if seeds is None else [int(x) for x in seeds]
        if len(self.seeds) != len(self.cfgs):
            raise ValueError("one seed per configuration")
        arr = (SnnConfig * len(cfgs))(*[make_config(c) for c in cfgs])
        sd = np.ascontiguousarray(self.seeds, np.uint64)
        self._o = SnnOptions(0, int(inject_fault), int(raster_capacity), float(timeout_s))
        self.sizes = [int(sum(c["pop_sizes"])) for c in cfgs]
        self._drained = {}                  # spikes read so far, per instance
        self.stream = _stream_handle(stream)
        h = C.c_void_p()
        _check(lib().snn_batch_create(arr, _ptr(sd, C.c_uint64), len(cfgs), C.byref(self._o),
                                      self.stream, C.byref(h)))
        self._h = h

    def __len__(self):
        return len(self.cfgs)

    def step(self, n_steps: int):
        _check(lib().snn_batch_step(self._h, int(n_steps)))

    def sync(self):
        _check(lib().snn_batch_sync(self._h))

    def set_tiling(self, k: int, tiling: int):
        _check(lib().snn_batch_set_tiling(self._h, int(k), int(tiling)))

    def info(self, k: int = 0) -> dict:
        i = SnnBatchInfo()
        _check(lib().snn_batch_get_info(self._h, int(k), C.byref(i)))
        return {f: getattr(i, f) for f, _ in SnnBatchInfo._fields_}

    def read_spikes(self, k: int, cap: int | None = None):
        """Drain instance k's spikes; returns (steps, ids) sorted by (step, id)."""
        if cap is None:                     # spikes not read yet bound the undrained ones
            cap = max(1, self.counters(k)["spikes"] - self._drained.get(k, 0))
        st = np.zeros(cap, np.uint32)
        ids = np.zeros(cap, np.uint32)
        n = self.read_spikes_into(k, st, ids)
        st, ids = st[:n], ids[:n]
        order = np.lexsort((ids, st))
        return st[order].astype(np.int64), ids[order].astype(np.int64)

    def read_spikes_into(self, k: int, steps_buf: np.ndarray, ids_buf: np.ndarray) -> int:
        """Drain instance k's spikes into caller-provided uint32 host buffers
        (ids relative to the instance, in recording order, not sorted)."""
        n = C.c_int64()
        _check(lib().snn_batch_read_spikes(self._h, int(k), _ptr(steps_buf, C.c_uint32),
                                           _ptr(ids_buf, C.c_uint32), int(steps_buf.size),
                                           C.byref(n)))
        self._drained[k] = self._drained.get(k, 0) + n.value
        return n.value

    def state(self, k: int):
        n = self.sizes[k]
        u = np.zeros(n, np.float32)
        i = np.zeros(n, np.float32)
        r = np.zeros(n, np.int32)
        _check(lib().snn_batch_read_state(self._h, int(k), _ptr(u, C.c_float),
                                          _ptr(i, C.c_float), _ptr(r, C.c_int32)))
        return u, i, r

    def counters(self, k: int) -> dict:
        s, a, b = C.c_int64(), C.c_uint64(), C.c_uint64()
        _check(lib().snn_batch_counters(self._h, int(k), C.byref(s), C.byref(a), C.byref(b)))
        return {"step": s.value, "spikes": a.value, "events": b.value}

    def close(self):
        if getattr(self, "_h", None):
            lib().snn_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def step_noalloc(cfg: dict, seed: int, io: SnnNoallocIO, t0: int, n_steps: int, stream=None):
    """``snn_step_noalloc``: step a network held in caller-owned device memory
    (``io`` holds the device pointers); allocates no device memory."""
    c = make_config(cfg)
    _check(lib().snn_step_noalloc(C.byref(c), int(seed), C.byref(io), int(t0), int(n_steps),
                                  _stream_handle(stream)))


def decode_words(words: np.ndarray):
    """Split packed synaptic words into (target, delay, code)."""
    w = np.asarray(words, np.uint32)
    return (w & 0x7FFFF).astype(np.int64), ((w >> 19) & 63).astype(np.int64), (w >> 25).astype(np.int64)


def encode_words(tgt, delay, code) -> np.ndarray:
    """Pack (target, delay, code) into synaptic words."""
    t = np.asarray(tgt, np.uint32)
    d = np.asarray(delay, np.uint32)
    c = np.asarray(code, np.uint32)
    return t | (d << 19) | (c << 25)
