"""CPU oracle for the time-stepped cortical-microcircuit simulation.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  The CUDA product path
(``paper_1909_08665_gb300``) never imports it and shares no code with it.

The simulation core is plain C (``oracle.c``); this module marshals arguments
with ctypes and holds the paper's validation statistics (Sec. 4.2): per-neuron
firing rates, coefficient of variation of inter-spike intervals and
correlation coefficients of binned spike trains (Freedman-Diaconis bins),
with an initial transient discarded (Sec. 2.1).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
MAX_POP = 8
POIS_TABLE = 32
WCODES = 128
DCODES = 256


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` (gcc, no FMA contraction)."""
    src = os.path.join(_HERE, "oracle.c")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-pthread", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrcConfig(C.Structure):
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


def make_config(cfg: dict) -> OrcConfig:
    c = OrcConfig()
    npop = len(cfg["pop_sizes"])
    assert 1 <= npop <= MAX_POP
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


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        P = C.POINTER
        L.orc_philox4x32_10.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
        L.orc_norm_quantile.argtypes = [C.c_double]
        L.orc_norm_quantile.restype = C.c_double
        L.orc_propagators.argtypes = [P(OrcConfig), P(C.c_double), P(C.c_float)]
        L.orc_poisson_thresholds.argtypes = [C.c_double, P(C.c_uint64)]
        L.orc_poisson_count.argtypes = [C.c_uint32, P(C.c_uint64)]
        L.orc_poisson_count.restype = C.c_int
        L.orc_tables.argtypes = [P(OrcConfig), P(C.c_int32), P(C.c_uint8), P(C.c_uint64),
                                 P(C.c_uint64), P(C.c_int32), P(C.c_int32)]
        L.orc_tables.restype = C.c_int
        L.orc_poisson_draws.argtypes = [C.c_uint64, C.c_int64, C.c_int64, C.c_int64,
                                        P(C.c_uint64), P(C.c_int32)]
        L.orc_net_generate.argtypes = [P(OrcConfig), C.c_uint64, C.c_int]
        L.orc_net_generate.restype = C.c_void_p
        L.orc_net_custom.argtypes = [P(OrcConfig), P(C.c_int64), P(C.c_int32), P(C.c_uint8),
                                     P(C.c_uint8), P(C.c_int32)]
        L.orc_net_custom.restype = C.c_void_p
        L.orc_net_neurons.argtypes = [C.c_void_p]
        L.orc_net_neurons.restype = C.c_int64
        L.orc_net_synapses.argtypes = [C.c_void_p]
        L.orc_net_synapses.restype = C.c_int64
        L.orc_net_export.argtypes = [C.c_void_p, P(C.c_int64), P(C.c_int32), P(C.c_uint8),
                                     P(C.c_uint8)]
        L.orc_net_row.argtypes = [P(OrcConfig), C.c_uint64, C.c_int64, P(C.c_int32),
                                  P(C.c_uint8), P(C.c_uint8), C.c_int64]
        L.orc_net_row.restype = C.c_int64
        L.orc_net_free.argtypes = [C.c_void_p]
        L.orc_deliver.argtypes = [C.c_void_p, P(OrcConfig), P(C.c_int32), C.c_int64, C.c_int64,
                                  P(C.c_int64)]
        L.orc_sim_create.argtypes = [C.c_void_p, P(OrcConfig), C.c_uint64, P(C.c_float)]
        L.orc_sim_create.restype = C.c_void_p
        L.orc_sim_run.argtypes = [C.c_void_p, C.c_int64]
        L.orc_sim_run.restype = C.c_int64
        L.orc_sim_raster_count.argtypes = [C.c_void_p]
        L.orc_sim_raster_count.restype = C.c_int64
        L.orc_sim_raster_read.argtypes = [C.c_void_p, P(C.c_int64), P(C.c_int32)]
        L.orc_sim_state.argtypes = [C.c_void_p, P(C.c_float), P(C.c_float), P(C.c_int32),
                                    P(C.c_int64)]
        L.orc_sim_set_state.argtypes = [C.c_void_p, P(C.c_float), P(C.c_float),
                                        P(C.c_int32), P(C.c_int64), C.c_int64]
        L.orc_sim_counters.argtypes = [C.c_void_p, P(C.c_int64), P(C.c_int64), P(C.c_int64),
                                       P(C.c_int32)]
        L.orc_sim_free.argtypes = [C.c_void_p]
        L.orc_sim_run_trace.argtypes = [C.c_void_p, C.c_int64, P(C.c_float), P(C.c_uint8),
                                        P(C.c_int32)]
        L.orc_sim_run_trace.restype = C.c_int64
        L.orc_grad_backward.argtypes = [C.c_void_p, P(OrcConfig), C.c_int, C.c_int64,
                                        P(C.c_double), P(C.c_double), P(C.c_uint8),
                                        P(C.c_double), P(C.c_double), P(C.c_double),
                                        P(C.c_double)]
        L.orc_relaxed_forward.argtypes = [C.c_void_p, P(OrcConfig), C.c_int64, P(C.c_double),
                                          P(C.c_double), P(C.c_double), P(C.c_double),
                                          P(C.c_double)]
        L.orc_surrogate_forward.argtypes = [C.c_void_p, P(OrcConfig), P(C.c_double), C.c_double,
                                            C.c_int64, P(C.c_double), P(C.c_float),
                                            P(C.c_uint8), P(C.c_int32), P(C.c_double)]
        _lib = L
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


# --------------------------------------------------------------------------
# primitives
# --------------------------------------------------------------------------
def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one counter (4 x u32) under one key (2 x u32)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(out, C.c_uint32))
    return out


def norm_quantile(p: float) -> float:
    return lib().orc_norm_quantile(float(p))


def propagators(cfg: dict):
    """(P22, P21, P11, P20) in double and rounded to fp32."""
    c = make_config(cfg)
    d = np.zeros(4, np.float64)
    f = np.zeros(4, np.float32)
    lib().orc_propagators(C.byref(c), _ptr(d, C.c_double), _ptr(f, C.c_float))
    return d, f


def poisson_thresholds(lam: float) -> np.ndarray:
    t = np.zeros(POIS_TABLE, np.uint64)
    lib().orc_poisson_thresholds(float(lam), _ptr(t, C.c_uint64))
    return t


def poisson_count(x: int, thr: np.ndarray) -> int:
    thr = np.ascontiguousarray(thr, np.uint64)
    return lib().orc_poisson_count(int(x), _ptr(thr, C.c_uint64))


def poisson_draws(seed: int, neuron: int, t0: int, n: int, thr: np.ndarray) -> np.ndarray:
    thr = np.ascontiguousarray(thr, np.uint64)
    out = np.zeros(n, np.int32)
    lib().orc_poisson_draws(int(seed), int(neuron), int(t0), int(n), _ptr(thr, C.c_uint64),
                            _ptr(out, C.c_int32))
    return out


def tables(cfg: dict) -> dict:
    c = make_config(cfg)
    wtab = np.zeros(MAX_POP * MAX_POP * WCODES, np.int32)
    dtab = np.zeros(MAX_POP * DCODES, np.uint8)
    pois = np.zeros(MAX_POP * POIS_TABLE, np.uint64)
    conn = np.zeros(MAX_POP * MAX_POP, np.uint64)
    wq = C.c_int32()
    nref = C.c_int32()
    rc = lib().orc_tables(C.byref(c), _ptr(wtab, C.c_int32), _ptr(dtab, C.c_uint8),
                          _ptr(pois, C.c_uint64), _ptr(conn, C.c_uint64), C.byref(wq),
                          C.byref(nref))
    if rc != 0:
        raise ValueError("weight does not fit the fixed-point range")
    return {"wtab": wtab.reshape(MAX_POP, MAX_POP, WCODES), "dtab": dtab.reshape(MAX_POP, DCODES),
            "pois": pois.reshape(MAX_POP, POIS_TABLE), "conn_thr": conn.reshape(MAX_POP, MAX_POP),
            "wext_q": wq.value, "n_ref": nref.value}


# --------------------------------------------------------------------------
# network and simulation
# --------------------------------------------------------------------------
class Network:
    """Oracle network: rows per presynaptic neuron, ascending targets."""

    def __init__(self, cfg: dict, seed: int | None = None, n_threads: int | None = None,
                 custom: dict | None = None):
        self.cfg = cfg
        self._c = make_config(cfg)
        L = lib()
        if custom is None:
            seed = cfg["seed"] if seed is None else seed
            nt = n_threads or max(1, os.cpu_count() or 1)
            self._h = L.orc_net_generate(C.byref(self._c), int(seed), int(nt))
        else:
            rp = np.ascontiguousarray(custom["row_ptr"], np.int64)
            tg = np.ascontiguousarray(custom["tgt"], np.int32)
            dl = np.ascontiguousarray(custom["delay"], np.uint8)
            wc = np.ascontiguousarray(custom["wcode"], np.uint8)
            wt = np.ascontiguousarray(custom["wtab"], np.int32).reshape(-1)
            assert wt.size == MAX_POP * MAX_POP * WCODES
            self._h = L.orc_net_custom(C.byref(self._c), _ptr(rp, C.c_int64),
                                       _ptr(tg, C.c_int32), _ptr(dl, C.c_uint8),
                                       _ptr(wc, C.c_uint8), _ptr(wt, C.c_int32))
        if not self._h:
            raise ValueError("oracle network generation failed")
        self.n = L.orc_net_neurons(self._h)
        self.nnz = L.orc_net_synapses(self._h)

    def export(self):
        rp = np.zeros(self.n + 1, np.int64)
        tg = np.zeros(max(self.nnz, 1), np.int32)
        dl = np.zeros(max(self.nnz, 1), np.uint8)
        wc = np.zeros(max(self.nnz, 1), np.uint8)
        lib().orc_net_export(self._h, _ptr(rp, C.c_int64), _ptr(tg, C.c_int32),
                             _ptr(dl, C.c_uint8), _ptr(wc, C.c_uint8))
        return rp, tg[:self.nnz], dl[:self.nnz], wc[:self.nnz]

    def deliver(self, spikes, t: int, ring: np.ndarray | None = None) -> np.ndarray:
        """Add the rows of ``spikes`` (spikes of step ``t``) into ``ring``
        ([D][n] int64, zeros if omitted) and return it."""
        D = int(self.cfg["ring_depth"])
        if ring is None:
            ring = np.zeros((D, self.n), np.int64)
        ring = np.ascontiguousarray(ring, np.int64)
        sp = np.ascontiguousarray(spikes, np.int32)
        lib().orc_deliver(self._h, C.byref(self._c), _ptr(sp, C.c_int32), int(sp.size), int(t),
                          _ptr(ring, C.c_int64))
        return ring

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_net_free(self._h)
            self._h = None


def network_row(cfg: dict, seed: int, j: int, cap: int | None = None):
    """Row of source ``j`` generated on its own (sampled checks at full size)."""
    c = make_config(cfg)
    cap = cap or int(sum(cfg["pop_sizes"]))
    tg = np.zeros(cap, np.int32)
    dl = np.zeros(cap, np.uint8)
    wc = np.zeros(cap, np.uint8)
    n = lib().orc_net_row(C.byref(c), int(seed), int(j), _ptr(tg, C.c_int32),
                          _ptr(dl, C.c_uint8), _ptr(wc, C.c_uint8), int(cap))
    return tg[:n], dl[:n], wc[:n]


class Simulation:
    """Oracle simulation over a :class:`Network`."""

    def __init__(self, net: Network, cfg: dict | None = None, seed: int | None = None,
                 u0: np.ndarray | None = None):
        cfg = net.cfg if cfg is None else cfg
        self.net = net
        self.cfg = cfg
        self._c = make_config(cfg)
        seed = cfg["seed"] if seed is None else seed
        self._u0 = None if u0 is None else np.ascontiguousarray(u0, np.float32)
        up = None if self._u0 is None else _ptr(self._u0, C.c_float)
        self._h = lib().orc_sim_create(net._h, C.byref(self._c), int(seed), up)
        if not self._h:
            raise ValueError("oracle simulation create failed")
        self.n = net.n
        self.D = int(cfg["ring_depth"])

    def run(self, n_steps: int) -> int:
        return lib().orc_sim_run(self._h, int(n_steps))

    def raster(self):
        """Drain the recorded spikes as (steps int64, ids int32), ordered by
        step then id."""
        L = lib()
        n = L.orc_sim_raster_count(self._h)
        st = np.zeros(max(n, 1), np.int64)
        ids = np.zeros(max(n, 1), np.int32)
        L.orc_sim_raster_read(self._h, _ptr(st, C.c_int64), _ptr(ids, C.c_int32))
        return st[:n], ids[:n]

    def state(self):
        u = np.zeros(self.n, np.float32)
        i = np.zeros(self.n, np.float32)
        r = np.zeros(self.n, np.int32)
        ring = np.zeros(self.D * self.n, np.int64)
        lib().orc_sim_state(self._h, _ptr(u, C.c_float), _ptr(i, C.c_float),
                            _ptr(r, C.c_int32), _ptr(ring, C.c_int64))
        return u, i, r, ring.reshape(self.D, self.n)

    def set_state(self, u, i_syn, refr, ring, step: int):
        u = np.ascontiguousarray(u, np.float32)
        i_syn = np.ascontiguousarray(i_syn, np.float32)
        refr = np.ascontiguousarray(refr, np.int32)
        ring = np.ascontiguousarray(ring, np.int64).reshape(-1)
        lib().orc_sim_set_state(self._h, _ptr(u, C.c_float), _ptr(i_syn, C.c_float),
                                _ptr(refr, C.c_int32), _ptr(ring, C.c_int64), int(step))

    def run_trace(self, n_steps: int):
        """Run ``n_steps`` recording, per step and neuron, u after the
        membrane update (before reset), flags = spike | non-refractory << 1,
        and the Poisson count."""
        u = np.zeros((n_steps, self.n), np.float32)
        f = np.zeros((n_steps, self.n), np.uint8)
        k = np.zeros((n_steps, self.n), np.int32)
        lib().orc_sim_run_trace(self._h, int(n_steps), _ptr(u, C.c_float), _ptr(f, C.c_uint8),
                                _ptr(k, C.c_int32))
        return u, f, k

    def counters(self):
        a, b, c, d = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int32()
        lib().orc_sim_counters(self._h, C.byref(a), C.byref(b), C.byref(c), C.byref(d))
        return {"step": a.value, "spikes": b.value, "events": c.value,
                "saturated": bool(d.value)}

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_sim_free(self._h)
            self._h = None


# --------------------------------------------------------------------------
# gradient of a population-rate loss (surrogate BPTT; the paper has none)
# --------------------------------------------------------------------------
HARD, RELAXED = 0, 1


def with_params(cfg: dict, alpha, nu: float) -> dict:
    """Configuration with projection weight scales ``alpha`` [8][8] (target,
    source) and background rate ``nu`` (Hz)."""
    import copy
    c = copy.deepcopy(cfg)
    a = np.asarray(alpha, np.float64).reshape(MAX_POP, MAX_POP)
    npop = len(c["pop_sizes"])
    c["proj_scale"] = [[float(a[p][q]) for q in range(npop)] for p in range(npop)]
    c["nu_bg"] = float(nu)
    return c


def rate_loss(rates, targets) -> float:
    """Mean squared error of the population rates (Hz^2)."""
    d = np.asarray(rates, np.float64) - np.asarray(targets, np.float64)
    return float(np.mean(d * d))


def rate_loss_grad(rates, targets) -> np.ndarray:
    d = np.asarray(rates, np.float64) - np.asarray(targets, np.float64)
    return 2.0 * d / d.size


def rates_from_flags(cfg: dict, flags: np.ndarray) -> np.ndarray:
    """Population rates (Hz) of a recorded run: spikes / (N_p T)."""
    bounds = np.cumsum([0] + list(cfg["pop_sizes"]))
    spk = (flags & 1).sum(axis=0, dtype=np.int64)
    T = flags.shape[0] * cfg["dt"] * 1e-3
    return np.array([spk[bounds[p]:bounds[p + 1]].sum() / (cfg["pop_sizes"][p] * T)
                     for p in range(len(cfg["pop_sizes"]))], np.float64)


def _g8(g_rate):
    g = np.zeros(MAX_POP, np.float64)
    g[:len(g_rate)] = g_rate
    return g


def grad_backward(net: Network, cfg: dict, mode: int, u_tr, s_tr, m_tr, g_rate, z=None):
    """Adjoint pass of the hard (mode 0) or relaxed (mode 1) model over the
    recorded trajectory; returns (dL/dalpha [8][8], dL/dnu)."""
    c = make_config(cfg)
    u = np.ascontiguousarray(u_tr, np.float64)
    sv = np.ascontiguousarray(s_tr, np.float64)
    m = np.ascontiguousarray(m_tr if m_tr is not None else np.zeros(u.shape, np.uint8), np.uint8)
    zz = np.ascontiguousarray(z if z is not None else np.zeros(u.shape), np.float64)
    g = _g8(g_rate)
    ga = np.zeros(MAX_POP * MAX_POP, np.float64)
    gn = C.c_double()
    lib().orc_grad_backward(net._h, C.byref(c), int(mode), int(u.shape[0]), _ptr(u, C.c_double),
                            _ptr(sv, C.c_double), _ptr(m, C.c_uint8), _ptr(zz, C.c_double),
                            _ptr(g, C.c_double), _ptr(ga, C.c_double), C.byref(gn))
    return ga.reshape(MAX_POP, MAX_POP), gn.value


def relaxed_forward(net: Network, cfg: dict, n_steps: int, u0, z, record: bool = False):
    """Sigmoid-relaxed model in double; returns rates (and the u, s records)."""
    c = make_config(cfg)
    n = net.n
    u0 = np.ascontiguousarray(u0, np.float64)
    zz = np.ascontiguousarray(z, np.float64)
    rates = np.zeros(MAX_POP, np.float64)
    ut = np.zeros((n_steps, n)) if record else None
    st = np.zeros((n_steps, n)) if record else None
    lib().orc_relaxed_forward(net._h, C.byref(c), int(n_steps), _ptr(u0, C.c_double),
                              _ptr(zz, C.c_double),
                              _ptr(ut, C.c_double) if record else None,
                              _ptr(st, C.c_double) if record else None,
                              _ptr(rates, C.c_double))
    npop = len(cfg["pop_sizes"])
    return (rates[:npop], ut, st) if record else rates[:npop]


def surrogate_forward(net0: Network, cfg0: dict, alpha, nu: float, n_steps: int, u0,
                      u_star, f_star, k_star) -> np.ndarray:
    """Smooth model around a recorded hard run (its exact gradient at the
    recording's parameters is the surrogate gradient); returns rates."""
    c = make_config(cfg0)
    a = np.ascontiguousarray(np.asarray(alpha, np.float64).reshape(-1), np.float64)
    u0 = np.ascontiguousarray(u0, np.float64)
    us = np.ascontiguousarray(u_star, np.float32)
    fs = np.ascontiguousarray(f_star, np.uint8)
    ks = np.ascontiguousarray(k_star, np.int32)
    rates = np.zeros(MAX_POP, np.float64)
    lib().orc_surrogate_forward(net0._h, C.byref(c), _ptr(a, C.c_double), float(nu),
                                int(n_steps), _ptr(u0, C.c_double), _ptr(us, C.c_float),
                                _ptr(fs, C.c_uint8), _ptr(ks, C.c_int32), _ptr(rates, C.c_double))
    return rates[:len(cfg0["pop_sizes"])]


def hard_gradient(cfg: dict, alpha, nu: float, n_steps: int, targets, seed: int | None = None,
                  n_threads: int | None = None):
    """Hard-model forward at (alpha, nu) with the recorded trajectory, then the
    surrogate backward of the rate MSE.  Returns a dict with rates, loss,
    g_alpha [8][8], g_nu and the trajectory (u0, u, flags, k, network)."""
    cp = with_params(cfg, alpha, nu)
    net = Network(cp, seed=seed, n_threads=n_threads or os.cpu_count())
    sim = Simulation(net, seed=seed)
    u0 = sim.state()[0].copy()
    u, f, k = sim.run_trace(n_steps)
    rates = rates_from_flags(cp, f)
    g_rate = rate_loss_grad(rates, targets)
    ga, gn = grad_backward(net, cp, HARD, u, (f & 1).astype(np.float64), f, g_rate)
    return {"rates": rates, "loss": rate_loss(rates, targets), "g_alpha": ga, "g_nu": gn,
            "u0": u0, "u": u, "flags": f, "k": k, "net": net, "cfg": cp}


# --------------------------------------------------------------------------
# validation statistics (Sec. 4.2)
# --------------------------------------------------------------------------
def pop_of(cfg: dict, ids: np.ndarray) -> np.ndarray:
    bounds = np.cumsum([0] + list(cfg["pop_sizes"]))
    return np.searchsorted(bounds, ids, side="right") - 1


def population_rates(cfg: dict, steps, ids, t_start: int, t_stop: int) -> np.ndarray:
    """Mean firing rate (Hz) of each population over steps [t_start, t_stop)."""
    steps = np.asarray(steps)
    ids = np.asarray(ids)
    m = (steps >= t_start) & (steps < t_stop)
    pops = pop_of(cfg, ids[m])
    counts = np.bincount(pops, minlength=len(cfg["pop_sizes"]))
    dur_s = (t_stop - t_start) * cfg["dt"] * 1e-3
    return counts / (np.asarray(cfg["pop_sizes"], np.float64) * dur_s)


def neuron_rates(cfg: dict, steps, ids, t_start: int, t_stop: int) -> np.ndarray:
    """Single-neuron firing rates (Hz) over steps [t_start, t_stop)."""
    steps = np.asarray(steps)
    ids = np.asarray(ids)
    m = (steps >= t_start) & (steps < t_stop)
    n = int(sum(cfg["pop_sizes"]))
    counts = np.bincount(ids[m], minlength=n)
    return counts / ((t_stop - t_start) * cfg["dt"] * 1e-3)


def cv_isi(steps, ids, n_neurons: int, t_start: int, t_stop: int, min_spikes: int = 3):
    """Coefficient of variation of the inter-spike intervals of every neuron
    with at least ``min_spikes`` spikes in the window (NaN otherwise)."""
    steps = np.asarray(steps, np.int64)
    ids = np.asarray(ids, np.int64)
    m = (steps >= t_start) & (steps < t_stop)
    steps, ids = steps[m], ids[m]
    order = np.lexsort((steps, ids))
    steps, ids = steps[order], ids[order]
    out = np.full(n_neurons, np.nan)
    if ids.size == 0:
        return out
    starts = np.flatnonzero(np.r_[True, ids[1:] != ids[:-1]])
    ends = np.r_[starts[1:], ids.size]
    for s, e in zip(starts, ends):
        if e - s >= min_spikes:
            isi = np.diff(steps[s:e]).astype(np.float64)
            mu = isi.mean()
            out[ids[s]] = isi.std() / mu if mu > 0 else np.nan
    return out


def freedman_diaconis_width(x: np.ndarray) -> float:
    """Freedman-Diaconis bin width 2 IQR n^(-1/3)."""
    x = np.asarray(x, np.float64)
    if x.size < 2:
        return 1.0
    q75, q25 = np.percentile(x, [75, 25])
    return 2.0 * (q75 - q25) * x.size ** (-1.0 / 3.0)


def binned_correlations(steps, ids, neuron_ids, t_start: int, t_stop: int, bin_steps: int):
    """Pearson correlation coefficients between the binned spike trains of
    ``neuron_ids`` (upper triangle, NaN rows of silent trains dropped)."""
    steps = np.asarray(steps, np.int64)
    ids = np.asarray(ids, np.int64)
    neuron_ids = np.asarray(neuron_ids, np.int64)
    m = (steps >= t_start) & (steps < t_stop) & np.isin(ids, neuron_ids)
    nb = max(1, (t_stop - t_start) // bin_steps)
    index = {int(v): k for k, v in enumerate(neuron_ids)}
    mat = np.zeros((neuron_ids.size, nb))
    for s, i in zip(steps[m], ids[m]):
        b = (s - t_start) // bin_steps
        if b < nb:
            mat[index[int(i)], b] += 1
    keep = mat.std(axis=1) > 0
    mat = mat[keep]
    if mat.shape[0] < 2:
        return np.zeros(0)
    cc = np.corrcoef(mat)
    iu = np.triu_indices(mat.shape[0], 1)
    return cc[iu]


def population_statistics(cfg: dict, steps, ids, t_start: int, t_stop: int,
                          n_corr: int = 200) -> dict:
    """The within-population statistics the paper compares between
    simulators (Sec. 4.2) over steps [t_start, t_stop): per population, the
    mean and standard deviation of single-neuron firing rates (Hz), the mean
    coefficient of variation of inter-spike intervals (neurons with at least 3
    spikes), and the mean correlation coefficient between the binned spike
    trains of its first ``n_corr`` neurons.  Spike trains are binned by the
    Freedman-Diaconis rule applied to the population's pooled spike times in
    the window."""
    steps = np.asarray(steps, np.int64)
    ids = np.asarray(ids, np.int64)
    n = int(sum(cfg["pop_sizes"]))
    bounds = np.cumsum([0] + list(cfg["pop_sizes"]))
    rates = neuron_rates(cfg, steps, ids, t_start, t_stop)
    cv = cv_isi(steps, ids, n, t_start, t_stop)
    win = (steps >= t_start) & (steps < t_stop)
    out = {"rate_mean": [], "rate_sd": [], "cv_mean": [], "corr_mean": [], "corr_bin_steps": []}
    for p in range(len(cfg["pop_sizes"])):
        lo, hi = int(bounds[p]), int(bounds[p + 1])
        out["rate_mean"].append(float(rates[lo:hi].mean()))
        out["rate_sd"].append(float(rates[lo:hi].std()))
        c = cv[lo:hi]
        out["cv_mean"].append(float(np.nanmean(c)) if np.isfinite(c).any() else float("nan"))
        pooled = steps[win & (ids >= lo) & (ids < hi)]
        width = max(1, int(round(freedman_diaconis_width(pooled)))) if pooled.size > 1 else 1
        cc = binned_correlations(steps, ids, np.arange(lo, min(lo + n_corr, hi)), t_start, t_stop,
                                 width)
        out["corr_mean"].append(float(np.mean(cc)) if cc.size else 0.0)
        out["corr_bin_steps"].append(width)
    return out

