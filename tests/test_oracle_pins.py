"""Pins of the CPU oracle against things other than itself.

Each test ties one oracle function to a closed form, an independent library
routine, the paper's printed values or a brute-force evaluation, so that a
plausible mistake (dropped term, wrong sign, index or operand order) fails.
"""
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest
from scipy import linalg, special, stats

import oracle
import workload
from helpers import custom_network, tiny_config

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.json")


def golden():
    with open(GOLDEN) as f:
        return {k: v["value"] for k, v in json.load(f).items() if not k.startswith("_")}


# --------------------------------------------------------------------------
# Philox4x32-10 against triton's independent implementation (CPU interpreter)
# --------------------------------------------------------------------------
_TRITON_SCRIPT = r"""
import json, os, sys
os.environ["TRITON_INTERPRET"] = "1"
import torch, triton, triton.language as tl
cases = json.loads(sys.stdin.read())

@triton.jit
def kern(out_ptr, c_ptr, seed):
    offs = tl.arange(0, 1)
    c0 = tl.load(c_ptr + 0 + offs).to(tl.uint32)
    c1 = tl.load(c_ptr + 1 + offs).to(tl.uint32)
    c2 = tl.load(c_ptr + 2 + offs).to(tl.uint32)
    c3 = tl.load(c_ptr + 3 + offs).to(tl.uint32)
    r0, r1, r2, r3 = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + 0 + offs, r0.to(tl.int64) & 0xffffffff)
    tl.store(out_ptr + 1 + offs, r1.to(tl.int64) & 0xffffffff)
    tl.store(out_ptr + 2 + offs, r2.to(tl.int64) & 0xffffffff)
    tl.store(out_ptr + 3 + offs, r3.to(tl.int64) & 0xffffffff)

res = []
for ctr, seed in cases:
    c = torch.tensor(ctr, dtype=torch.int64)
    o = torch.zeros(4, dtype=torch.int64)
    kern[(1,)](o, c, seed)
    res.append(o.tolist())
print(json.dumps(res))
"""


def test_philox_matches_triton_reference():
    pytest.importorskip("triton")
    rng = np.random.default_rng(3)
    cases = [([0, 0, 0, 0], 0), ([1, 2, 3, 4], 0), ([0xFFFFFFFF] * 4, (1 << 64) - 1)]
    for _ in range(12):
        cases.append((rng.integers(0, 2**32, 4).tolist(), int(rng.integers(0, 2**63))))
    env = dict(os.environ, TRITON_INTERPRET="1")
    out = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(cases),
                         capture_output=True, text=True, env=env, timeout=600)
    if out.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + out.stderr[-300:])
    ref = json.loads(out.stdout.strip().splitlines()[-1])
    for (ctr, seed), r in zip(cases, ref):
        key = [seed & 0xFFFFFFFF, seed >> 32]
        got = oracle.philox(ctr, key)
        assert got.tolist() == r, (ctr, seed)


def test_philox_output_is_uniform():
    # 2^16 outputs of consecutive counters: bytes uniform (chi-square)
    vals = np.concatenate([oracle.philox([i, 7, 3, 0], [12345, 0]) for i in range(4096)])
    by = (vals[:, None] >> np.arange(0, 32, 8)).astype(np.uint8).ravel()
    chi = stats.chisquare(np.bincount(by, minlength=256))
    assert chi.pvalue > 1e-4


# --------------------------------------------------------------------------
# normal quantile, propagators, Poisson thresholds
# --------------------------------------------------------------------------
def test_norm_quantile_matches_scipy():
    for p in np.r_[np.linspace(1e-6, 1 - 1e-6, 97), (np.arange(128) + 0.5) / 128]:
        x = oracle.norm_quantile(p)
        assert abs(x - special.ndtri(p)) <= 1e-12 * max(1.0, abs(x))


def test_propagators_match_matrix_exponential():
    cfg = workload.microcircuit(0.1)
    d, f = oracle.propagators(cfg)
    tm, ts, cm, dt = cfg["tau_m"], cfg["tau_syn"], cfg["c_m"], cfg["dt"]
    # state (u, I, I_dc): u' = -u/tm + (I + I_dc)/cm, I' = -I/ts, I_dc' = 0
    A = np.array([[-1 / tm, 1 / cm, 1 / cm], [0, -1 / ts, 0], [0, 0, 0]])
    E = linalg.expm(A * dt)
    P22, P21, P11, P20 = E[0, 0], E[0, 1], E[1, 1], E[0, 2]
    np.testing.assert_allclose(d, [P22, P21, P11, P20], rtol=1e-12)
    assert f.tolist() == [float(np.float32(v)) for v in d]
    # R = tau_m / C_m = 40 MOhm: P20 = R (1 - P22)
    assert abs(P20 - tm / cm * (1 - P22)) < 1e-15


@pytest.mark.parametrize("lam", [0.0, 0.3, 1.28, 2.0, 2.32, 5.0])
def test_poisson_thresholds_match_scipy_cdf(lam):
    thr = oracle.poisson_thresholds(lam).astype(np.float64)
    cdf = stats.poisson.cdf(np.arange(32), lam)
    # floor(2^32 F) / 2^32 lies within one quantum below F (plus rounding)
    diff = cdf - thr / 2**32
    assert np.all(diff > -1e-14) and np.all(diff < 2.0**-32 + 1e-14)
    assert np.all(np.diff(thr) >= 0)


def test_poisson_count_inverse_transform():
    thr = oracle.poisson_thresholds(2.0)
    assert oracle.poisson_count(0, thr) == 0
    assert oracle.poisson_count(int(thr[0]) - 1, thr) == 0
    assert oracle.poisson_count(int(thr[0]), thr) == 1
    assert oracle.poisson_count(int(thr[3]), thr) == 4
    assert oracle.poisson_count(2**32 - 1, thr) >= 12


@pytest.mark.parametrize("lam", [1.28, 2.32])
def test_poisson_draws_chi_square(lam):
    thr = oracle.poisson_thresholds(lam)
    k = oracle.poisson_draws(777, neuron=5, t0=0, n=200_000, thr=thr)
    assert abs(k.mean() - lam) < 5 * math.sqrt(lam / k.size)
    assert abs(k.var() - lam) < 0.03 * lam
    kmax = 9
    obs = np.bincount(np.minimum(k, kmax), minlength=kmax + 1)
    pmf = stats.poisson.pmf(np.arange(kmax), lam)
    exp = np.r_[pmf, 1 - pmf.sum()] * k.size
    assert stats.chisquare(obs, exp).pvalue > 1e-4


# --------------------------------------------------------------------------
# parameter tables against the paper's printed values
# --------------------------------------------------------------------------
def test_tables_reproduce_paper_parameters():
    g = golden()
    cfg = workload.microcircuit(1.0)
    t = oracle.tables(cfg)
    wt = t["wtab"] / 256.0
    exc = wt[2, 0]            # L2/3e source -> L4e target
    inh = wt[0, 1]            # L2/3i source -> L2/3e target
    l4 = wt[0, 2]             # L4e -> L2/3e
    # equiprobable quantile grid: mean exact up to rounding, sd 0.99x (grid)
    assert abs(exc.mean() - g["w_exc_mean_pA"]) < 1e-2
    assert abs(-inh.mean() - g["w_inh_mean_pA"]) < 1e-2
    assert abs(l4.mean() - g["w_l4e_l23e_mean_pA"]) < 1e-2
    assert 0.98 < exc.std() / g["w_exc_sd_pA"] < 1.0
    assert 0.98 < inh.std() / g["w_inh_sd_pA"] < 1.0
    assert 0.98 < l4.std() / g["w_l4e_l23e_sd_pA"] < 1.0
    assert np.all(wt[:, 0::2] > 0) and np.all(wt[:, 1::2] < 0)      # Dale's law
    # delays: rounded normal, clamped to [1, 63]; compare with scipy's normal
    for q, (mu, sd) in [(0, (g["d_exc_mean_ms"], g["d_exc_sd_ms"])),
                        (1, (g["d_inh_mean_ms"], g["d_inh_sd_ms"]))]:
        d = t["dtab"][q].astype(np.int64)
        assert d.min() >= 1 and d.max() <= 63 and np.all(np.diff(d) >= 0)
        steps = np.arange(1, 64)
        edges = (steps - 0.5) * g["dt_ms"]
        pk = np.diff(np.r_[0.0, stats.norm.cdf(edges[1:], mu, sd), 1.0])
        frac = np.bincount(d, minlength=64)[1:] / d.size
        assert np.all(np.abs(frac - pk) <= 1.0 / 256 + 1e-12)
    # Poisson background 8 Hz x K_ext spans 12.8 .. 23.2 kHz (Sec. 3.1.3)
    rates = np.array(cfg["k_ext"]) * cfg["nu_bg"] / 1000.0
    assert abs(rates.min() - g["poisson_rate_min_kHz"]) < 1e-9
    assert abs(rates.max() - g["poisson_rate_max_kHz"]) < 1e-9
    lam = rates.min() * 1000 * g["dt_ms"] * 1e-3
    np.testing.assert_array_equal(t["pois"][0], oracle.poisson_thresholds(lam))
    assert t["wext_q"] == round(87.8 * 256)
    assert t["n_ref"] == 20


def test_workload_matches_paper_sizes():
    g = golden()
    cfg = workload.microcircuit(1.0)
    n = np.array(cfg["pop_sizes"])
    assert n.sum() == g["n_neurons"]
    p = np.array(cfg["conn_prob"])
    assert abs((n[:, None] * n[None, :] * p).sum() / g["n_synapses_approx"] - 1) < 0.01
    assert sum(workload.population_sizes(0.1)) == 7717
    assert sum(workload.population_sizes(4)) == 4 * g["n_neurons"]


# --------------------------------------------------------------------------
# connectivity statistics (Sec. 2.1: probabilistic, Dale's law)
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def net01():
    cfg = workload.microcircuit(0.1)
    net = oracle.Network(cfg)
    return cfg, net, net.export()


def test_connectivity_matches_probabilities(net01):
    cfg, net, (rp, tgt, dl, wc) = net01
    n = np.array(cfg["pop_sizes"])
    bounds = np.r_[0, np.cumsum(n)]
    src_pop = np.repeat(oracle.pop_of(cfg, np.arange(net.n)), np.diff(rp))
    tgt_pop = oracle.pop_of(cfg, tgt)
    counts = np.zeros((8, 8))
    np.add.at(counts, (tgt_pop, src_pop), 1)
    p = np.array(cfg["conn_prob"])
    pairs = n[:, None] * n[None, :] - np.diag(n)         # no autapses
    expect = pairs * p
    sd = np.sqrt(pairs * p * (1 - p))
    assert np.all(np.abs(counts - expect) <= 5 * sd + 1)
    # no autapses, ascending targets within a row
    src = np.repeat(np.arange(net.n), np.diff(rp))
    assert not np.any(src == tgt)
    for j in range(0, net.n, 97):
        row = tgt[rp[j]:rp[j + 1]]
        assert np.all(np.diff(row) > 0)
    assert bounds[-1] == net.n


def test_weight_codes_and_delays_distribution(net01):
    cfg, net, (rp, tgt, dl, wc) = net01
    assert stats.chisquare(np.bincount(wc, minlength=128)).pvalue > 1e-4
    src_pop = np.repeat(oracle.pop_of(cfg, np.arange(net.n)), np.diff(rp))
    t = oracle.tables(cfg)
    for q in (0, 1):
        d = dl[src_pop == q].astype(np.int64)
        ref = t["dtab"][q].astype(np.float64)
        assert abs(d.mean() - ref.mean()) < 5 * ref.std() / math.sqrt(d.size)


def test_single_row_matches_network(net01):
    cfg, net, (rp, tgt, dl, wc) = net01
    for j in (0, 1, 2067, 4000, net.n - 1):
        t2, d2, w2 = oracle.network_row(cfg, cfg["seed"], j)
        np.testing.assert_array_equal(t2, tgt[rp[j]:rp[j + 1]])
        np.testing.assert_array_equal(d2, dl[rp[j]:rp[j + 1]])
        np.testing.assert_array_equal(w2, wc[rp[j]:rp[j + 1]])


# --------------------------------------------------------------------------
# single-neuron closed forms (Eq. 1)
# --------------------------------------------------------------------------
def _run_tiny(cfg, net_desc, u0, steps):
    net = oracle.Network(cfg, custom=net_desc)
    sim = oracle.Simulation(net, u0=np.asarray(u0, np.float32))
    traces = []
    for _ in range(steps):
        sim.run(1)
        traces.append(sim.state()[0].copy())
    st, ids = sim.raster()
    return np.array(traces), st, ids, sim


def test_free_membrane_decay_closed_form():
    cfg = tiny_config(1)
    desc = custom_network(1, [], [0])
    u0 = 10.0
    tr, st, ids, _ = _run_tiny(cfg, desc, [u0], 300)
    n = np.arange(1, 301)
    exact = u0 * np.exp(-n * cfg["dt"] / cfg["tau_m"])
    # fp32 recurrence: relative error grows at most ~1 ulp per step
    assert np.all(np.abs(tr[:, 0] - exact) <= exact * (n + 2) * 2.0**-23)
    assert st.size == 0


def test_single_psc_response_closed_form():
    cfg = tiny_config(2)
    wq = round(87.8 * 256)
    d = 7
    desc = custom_network(2, [(0, 1, 0, d)], [wq])
    # neuron 0 starts above threshold and spikes in step 0; neuron 1 at rest
    tr, st, ids, _ = _run_tiny(cfg, desc, [16.0, 0.0], 220)
    assert st.tolist()[:1] == [0] and ids.tolist()[:1] == [0]
    w = wq / 256.0
    tm, ts, cm, dt = cfg["tau_m"], cfg["tau_syn"], cfg["c_m"], cfg["dt"]
    k = np.arange(0, 200)              # steps after arrival
    closed = (w / cm) * tm * ts / (tm - ts) * (np.exp(-k * dt / tm) - np.exp(-k * dt / ts))
    u1 = tr[d:d + 200, 1]              # value after step d + k
    np.testing.assert_allclose(u1, closed, rtol=2e-5, atol=1e-9)
    assert np.all(tr[:d, 1] == 0.0)
    # peak at t* = tm ts/(tm - ts) ln(tm/ts) = 1.5767 ms; 0.14999 mV for 87.8 pA
    tstar = tm * ts / (tm - ts) * math.log(tm / ts)
    assert abs(tstar - 1.5767) < 1e-4
    assert int(np.argmax(u1)) in (math.floor(tstar / dt), math.ceil(tstar / dt))
    peak = (87.8 / cm) * tm * ts / (tm - ts) * (math.exp(-tstar / tm) - math.exp(-tstar / ts))
    assert abs(peak - 0.14999) < 1e-5
    assert abs(u1.max() - peak * w / 87.8) < 2e-4


@pytest.mark.parametrize("i_dc", [400.0, 500.0, 800.0, 1500.0])
def test_fi_curve_closed_form(i_dc):
    cfg = tiny_config(1, input_mode=1, i_dc=i_dc)
    desc = custom_network(1, [], [0])
    net = oracle.Network(cfg, custom=desc)
    sim = oracle.Simulation(net, u0=np.zeros(1, np.float32))
    sim.run(3000)
    st, _ = sim.raster()
    tm, cm, dt = cfg["tau_m"], cfg["c_m"], cfg["dt"]
    R = tm / cm
    uinf = R * i_dc
    p22 = math.exp(-dt / tm)
    nstar = math.floor(math.log(1 - cfg["theta"] / uinf) / math.log(p22)) + 1
    # margin: the crossing is far from the fp32 rounding scale
    assert uinf * (1 - p22 ** nstar) - cfg["theta"] > 1e-4
    assert cfg["theta"] - uinf * (1 - p22 ** (nstar - 1)) > 1e-4
    n_ref = round(cfg["t_ref"] / dt)
    assert st[0] == nstar - 1
    isi = np.diff(st)
    assert np.all(isi == n_ref + nstar)
    # continuous-time limit T = t_ref + tau_m ln(u_inf / (u_inf - theta))
    T = cfg["t_ref"] + tm * math.log(uinf / (uinf - cfg["theta"]))
    assert abs(isi[0] * dt - T) <= dt


def test_subthreshold_current_never_fires():
    # rheobase: R I = theta  ->  I = 375 pA
    cfg = tiny_config(1, input_mode=1, i_dc=370.0)
    net = oracle.Network(cfg, custom=custom_network(1, [], [0]))
    sim = oracle.Simulation(net, u0=np.zeros(1, np.float32))
    sim.run(20000)
    st, _ = sim.raster()
    assert st.size == 0
    u = sim.state()[0][0]
    assert abs(u - (cfg["tau_m"] / cfg["c_m"]) * 370.0) < 1e-3


# --------------------------------------------------------------------------
# brute-force tiny networks: closed-form superposition in double precision
# --------------------------------------------------------------------------
def _brute_force(cfg, n, synapses, weights_pa, u0, i_dc, steps):
    """Spike steps by direct superposition of exact solutions (double).

    I_t = sum over arrivals s <= t of w P11^(t-s);  while free,
    u_t = P22^(t-a) u_a + sum_{m=a}^{t-1} P22^(t-1-m) (P21 I_m + P20 I_dc).
    Input arriving in step s enters I_s; a spike in step t is delivered to
    step t + delay; after a spike u is held at 0 for n_ref steps.
    Returns spikes and the smallest |u - theta| seen (the rounding margin).
    """
    tm, ts, cm, dt = cfg["tau_m"], cfg["tau_syn"], cfg["c_m"], cfg["dt"]
    P22, P11 = math.exp(-dt / tm), math.exp(-dt / ts)
    P21 = tm * ts / (cm * (tm - ts)) * (P22 - P11)
    P20 = tm / cm * (1 - P22)
    n_ref = round(cfg["t_ref"] / dt)
    theta = cfg["theta"]
    arrivals = [dict() for _ in range(n)]     # step -> total pA
    anchor = [(-1, float(u0[i])) for i in range(n)]   # (a, u_a)
    hold_until = [-1] * n
    spikes = []
    margin = float("inf")

    def current(i, t):
        return sum(w * P11 ** (t - s) for s, w in arrivals[i].items() if s <= t)

    for t in range(steps):
        fired = []
        for i in range(n):
            if t <= hold_until[i]:
                anchor[i] = (t, 0.0)
                continue
            a, ua = anchor[i]
            u = P22 ** (t - a) * ua
            for m in range(a, t):
                Im = current(i, m) if m >= 0 else 0.0
                u += P22 ** (t - 1 - m) * (P21 * Im + P20 * i_dc[i])
            margin = min(margin, abs(u - theta))
            if u > theta:
                fired.append(i)
                anchor[i] = (t, 0.0)
                hold_until[i] = t + n_ref
        for j in fired:
            spikes.append((t, j))
            for (s, tg, wi, d) in synapses:
                if s == j:
                    arrivals[tg][t + d] = arrivals[tg].get(t + d, 0.0) + weights_pa[wi]
    return spikes, margin


def test_tiny_network_brute_force():
    n = 6
    weights_q = [round(87.8 * 256 * 12), round(-351.2 * 256 * 3), round(87.8 * 256 * 20)]
    weights_pa = [w / 256.0 for w in weights_q]
    synapses = [(0, 1, 0, 3), (0, 2, 2, 15), (1, 3, 2, 1), (2, 3, 1, 5), (3, 4, 0, 40),
                (4, 5, 2, 63), (5, 0, 1, 9), (3, 5, 2, 2), (1, 0, 1, 30)]
    i_dc = [520.0, 480.0, 600.0, 450.0, 500.0, 390.0]
    u0 = [14.9, 5.0, 12.0, 0.0, 10.0, 3.0]
    cfg = tiny_config(n, input_mode=1)
    cfg["i_dc"] = [0.0] * 8
    # per-neuron DC is not a population parameter: give each neuron its own
    # population so that i_dc is set per neuron
    cfg["pop_sizes"] = [1] * n
    cfg["pop_exc"] = [1] * n
    cfg["i_dc"] = i_dc + [0.0] * (8 - n)
    cfg["conn_prob"] = [[0.0] * 8 for _ in range(8)]
    desc = custom_network(n, [(s, t, w, d) for s, t, w, d in synapses], weights_q)
    wt = np.zeros((8, 8, 128), np.int32)
    wt[:, :, :3] = np.asarray(weights_q, np.int32)
    desc["wtab"] = wt
    steps = 700
    net = oracle.Network(cfg, custom=desc)
    sim = oracle.Simulation(net, u0=np.asarray(u0, np.float32))
    sim.run(steps)
    st, ids = sim.raster()
    got = list(zip(st.tolist(), ids.tolist()))
    ref, margin = _brute_force(cfg, n, synapses, weights_pa, u0, i_dc, steps)
    assert margin > 1e-4
    assert len(ref) > 20
    assert got == ref


def test_refractory_clamp_and_saturation_flag():
    # a huge weight saturates int32: the oracle flags it
    cfg = tiny_config(2)
    desc = custom_network(2, [(0, 1, 0, 1)] * 1, [2**30])
    net = oracle.Network(cfg, custom=desc)
    sim = oracle.Simulation(net, u0=np.array([16.0, 0.0], np.float32))
    sim.run(3)
    assert not sim.counters()["saturated"]
    desc = custom_network(2, [(0, 1, 0, 1), (0, 1, 1, 1)], [2**30, 2**30])
    net = oracle.Network(cfg, custom=desc)
    sim = oracle.Simulation(net, u0=np.array([16.0, 0.0], np.float32))
    sim.run(3)
    assert sim.counters()["saturated"]


def test_default_initial_potential_uniform():
    cfg = workload.microcircuit(0.1)
    net = oracle.Network(cfg)
    sim = oracle.Simulation(net)
    u = sim.state()[0]
    assert u.min() >= cfg["u0_lo"] and u.max() < cfg["u0_hi"]
    assert stats.kstest(u, "uniform", args=(cfg["u0_lo"], cfg["u0_hi"] - cfg["u0_lo"])).pvalue > 1e-4


# --------------------------------------------------------------------------
# validation statistics (Sec. 4.2)
# --------------------------------------------------------------------------
def test_statistics_on_known_trains():
    # regular train: CV 0; Poisson train: CV ~ 1; identical trains: r = 1
    steps = np.arange(0, 10000, 50)
    cv = oracle.cv_isi(steps, np.zeros_like(steps), 1, 0, 10000)
    assert cv[0] == 0.0
    rng = np.random.default_rng(0)
    pst = np.flatnonzero(rng.random(200000) < 0.01)
    cvp = oracle.cv_isi(pst, np.zeros_like(pst), 1, 0, 200000)
    assert abs(cvp[0] - 1.0) < 0.05
    st = np.r_[pst, pst]
    ids = np.r_[np.zeros_like(pst), np.ones_like(pst)]
    cc = oracle.binned_correlations(st, ids, [0, 1], 0, 200000, 100)
    assert abs(cc[0] - 1.0) < 1e-12
    x = rng.normal(size=1000)
    edges = np.histogram_bin_edges(x, bins="fd")
    assert abs(oracle.freedman_diaconis_width(x) - (edges[1] - edges[0])) < 0.05 * (edges[1] - edges[0])
    cfg = workload.microcircuit(0.1)
    r = oracle.population_rates(cfg, np.zeros(2068, np.int64), np.arange(2068), 0, 10000)
    assert abs(r[0] - 1.0) < 1e-12 and r[1:].sum() == 0


# --------------------------------------------------------------------------
# stand-alone delivery (step 6 alone) pinned two ways: against the ring
# change of one full oracle step with a forced spike list, and against arrival
# sums written directly from the synapse list of a hand-set network
# --------------------------------------------------------------------------
def test_deliver_equals_ring_change_of_one_step(net01):
    """Neurons set far above threshold spike in the next step and no other
    does (the rest start at rest with no current, so one step of input cannot
    lift them to threshold); that step leaves in the ring exactly the rows of
    the forced spikes, which is what the stand-alone delivery must add."""
    cfg, net, (rp, _, _, _) = net01
    n = net.n
    spikes = workload.random_spike_list(n, 300, seed=17).astype(np.int32)
    t = 1234
    sim = oracle.Simulation(net)
    u = np.zeros(n, np.float32)
    u[spikes] = 25.0
    sim.set_state(u, np.zeros(n, np.float32), np.zeros(n, np.int32),
                  np.zeros((64, n), np.int64), t)
    sim.run(1)
    st, ids = sim.raster()
    assert np.all(st == t)
    np.testing.assert_array_equal(ids, np.sort(spikes))
    ring = sim.state()[3]
    ref = net.deliver(spikes, t)
    np.testing.assert_array_equal(ring, ref)
    assert sim.counters()["events"] == int(np.diff(rp)[spikes].sum())
    # duplicates in a list add twice; the result is linear in the list
    twice = net.deliver(np.r_[spikes, spikes], t)
    np.testing.assert_array_equal(twice, 2 * ref)
    assert cfg["ring_depth"] == 64


def test_deliver_brute_force_tiny_network():
    n = 6
    weights_q = [round(87.8 * 256 * 12), round(-351.2 * 256 * 3), round(87.8 * 256 * 20)]
    synapses = [(0, 1, 0, 3), (0, 2, 2, 15), (1, 3, 2, 1), (2, 3, 1, 5), (3, 4, 0, 40),
                (4, 5, 2, 63), (5, 0, 1, 9), (3, 5, 2, 2), (1, 0, 1, 30), (0, 5, 1, 63)]
    cfg = tiny_config(n)
    desc = custom_network(n, synapses, weights_q)
    net = oracle.Network(cfg, custom=desc)
    spikes = [0, 3, 1, 0, 5, 4, 4]
    for t in (0, 7, 61, 1000003):
        got = net.deliver(np.asarray(spikes, np.int32), t)
        want = np.zeros((64, n), np.int64)
        for j in spikes:                       # every synapse of every listed source
            for (s, tg, wi, d) in synapses:
                if s == j:
                    want[(t + d) % 64, tg] += weights_q[wi]
        np.testing.assert_array_equal(got, want)
