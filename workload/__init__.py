"""Seeded synthetic inputs for the cortical-microcircuit simulation.

This module is shared by the CPU oracle (``oracle/``) and the CUDA library
(``paper_1909_08665_gb300``).  It holds *inputs only*: model parameters,
population sizes, a synthetic connection-probability table, seeds, initial
membrane potentials and spike lists.  It contains none of the simulation
arithmetic (no propagators, no random-number generator of the method, no
quantisation, no network generation) so that the two implementations stay
independent.

Model parameters follow the paper's use-case description (Sec. 2.1): eight
populations (L2/3, L4, L5, L6; excitatory and inhibitory), 77,169 neurons,
about 3e8 synapses, normally distributed weights 87.8 +- 8.78 pA (excitatory
sources), 351.2 +- 35.32 pA (inhibitory sources, sign negative), L4e -> L2/3e
weights 175.6 +- 8.78 pA, delays 1.5 +- 0.75 ms (excitatory) and
0.75 +- 0.375 ms (inhibitory), dt = 0.1 ms, Poisson background at rates
12.8 - 23.2 kHz per neuron (Sec. 3.1.3, Poisson core).  Neuron constants
(tau_m 10 ms, C_m 250 pF, tau_syn 0.5 ms, t_ref 2 ms, threshold 15 mV above
rest) are those of the benchmark configuration.

The population-to-population connection-probability table of the original
model is not printed in the paper (Sec. 2.1 defers to the model's own
publication), so :func:`connection_table` draws a seeded synthetic stand-in of
the same shape: 8x8 probabilities, Dale's law by source population,
inhibition-dominated, rescaled so that the full-size network has 3.0e8
synapses.  A user who has the real table can pass it as ``conn_prob``.
"""
from __future__ import annotations

import copy
import json
import os
from fractions import Fraction

import numpy as np

POP_NAMES = ["L23e", "L23i", "L4e", "L4i", "L5e", "L5i", "L6e", "L6i"]
# Full-scale population sizes of the benchmark microcircuit (77,169 neurons).
POP_SIZES_FULL = [20683, 5834, 21915, 5479, 4850, 1065, 14395, 2948]
POP_EXC = [1, 0, 1, 0, 1, 0, 1, 0]
N_FULL = sum(POP_SIZES_FULL)
SYNAPSES_FULL = 3.0e8          # Sec. 2.1: "approximately 3 x 10^8 synapses"

RING_DEPTH = 64                # delay slots per neuron (max delay 63 steps)

_TABLE_FILE = os.path.join(os.path.dirname(__file__), "microcircuit_table.json")


def _round_half_even(x: Fraction) -> int:
    """Round an exact rational to the nearest integer, ties to even."""
    fl = x.numerator // x.denominator
    rem = x - fl
    if rem > Fraction(1, 2):
        return fl + 1
    if rem < Fraction(1, 2):
        return fl
    return fl if fl % 2 == 0 else fl + 1


def population_sizes(scale) -> list[int]:
    """Population sizes at ``scale`` x the full model, ties to even.

    The rounding is done on exact decimals (``Fraction(str(scale))``) so that
    0.1 x 1065 = 106.5 rounds to 106 and the 10 % model has 7,717 neurons.
    """
    s = Fraction(str(scale))
    return [_round_half_even(s * n) for n in POP_SIZES_FULL]


def generate_connection_table(seed: int = 1909, nu_ref: float = 3.0, mu_ref: float = 12.0,
                              min_ratio: float = 2.0, jitter: float = 0.1,
                              weak_frac: float = 0.15):
    """Draw a synthetic 8x8 connection-probability table ``p[target][source]``.

    Recipe (stand-in for the table the paper does not print):
      * every projection starts from one base probability times a seeded
        factor U(1 - jitter, 1 + jitter); a fraction ``weak_frac`` of the
        between-population projections is made "weak" (x U(0.05, 0.3));
        Sec. 4.1 mentions populations reached by low-probability connections;
      * every target population gets the same total in-degree
        K = 3.0e8 / 77,169 (Sec. 2.1: 0.3 billion synapses);
      * each row is split into excitatory in-degree K_E and inhibitory
        in-degree K_I (Dale's law by source) so that, with all populations at
        ``nu_ref`` Hz plus the population's own Poisson background, the mean
        free membrane potential R tau_syn (sum K w nu) is ``mu_ref`` mV, just
        below the 15 mV threshold; the inhibitory share is raised where needed
        so that inhibitory input (in-degree x |weight|) is at least
        ``min_ratio`` times the excitatory input.  Every row is then
        inhibition-dominated, and the network fires asynchronously at a few Hz.
    """
    rng = np.random.default_rng(seed)
    p = rng.uniform(1.0 - jitter, 1.0 + jitter, (8, 8))
    weak = (rng.random((8, 8)) < weak_frac) & ~np.eye(8, dtype=bool)
    p = np.where(weak, p * rng.uniform(0.05, 0.3, (8, 8)), p)
    n = np.array(POP_SIZES_FULL, dtype=np.float64)
    exc = np.array(POP_EXC, dtype=bool)
    kext = np.array(background_indegrees(), dtype=np.float64)
    k_tot = SYNAPSES_FULL / N_FULL
    # mV per (Hz x synapse) of an 87.8 pA synapse: R tau_syn w = 40 MOhm * 0.5 ms * 87.8 pA
    unit = 40e6 * 0.5e-3 * 87.8e-12 * 1e3
    for r in range(8):
        wrel = np.where(exc, 1.0, 4.0)
        if r == 0:
            wrel = wrel.copy()
            wrel[2] = 2.0                      # L4e -> L2/3e doubled weight
        pe = p[r] * exc * n
        pi = p[r] * ~exc * n
        e_gain = float((pe * wrel).sum() / pe.sum())   # mean |w| / 87.8 of exc inputs
        i_gain = float((pi * wrel).sum() / pi.sum())
        # K_E e_gain - K_I i_gain = (mu_ref/unit - nu_bg K_ext) / nu_ref,  K_E + K_I = K
        rhs = (mu_ref / unit - 8.0 * kext[r]) / nu_ref
        k_i = (k_tot * e_gain - rhs) / (e_gain + i_gain)
        # floor: K_I i_gain >= min_ratio K_E e_gain
        k_i = max(k_i, k_tot * min_ratio * e_gain / (i_gain + min_ratio * e_gain))
        k_e = k_tot - k_i
        p[r, exc] *= k_e / float(pe.sum())
        p[r, ~exc] *= k_i / float(pi.sum())
    return p


def background_indegrees():
    """K_ext per population, spread evenly over 1600..2900 so that
    8 Hz x K_ext spans the 12.8 - 23.2 kHz of Sec. 3.1.3."""
    return [1600.0 + 1300.0 * k / 7.0 for k in range(8)]


def connection_table():
    """The committed synthetic table (``microcircuit_table.json``)."""
    with open(_TABLE_FILE) as f:
        d = json.load(f)
    return d


def base_config() -> dict:
    """Full-scale (77,169 neurons) Poisson-driven microcircuit configuration."""
    tab = connection_table()
    w_mean = [[0.0] * 8 for _ in range(8)]
    w_sd = [[0.0] * 8 for _ in range(8)]
    for p in range(8):
        for q in range(8):
            if POP_EXC[q]:
                w_mean[p][q] = 87.8
                w_sd[p][q] = 8.78
            else:
                w_mean[p][q] = -351.2       # g = -4
                w_sd[p][q] = 35.32          # as printed in Sec. 2.1
    # L4e -> L2/3e: doubled mean, same standard deviation (Sec. 2.1).
    w_mean[0][2] = 175.6
    d_mean = [1.5 if e else 0.75 for e in POP_EXC]
    d_sd = [0.75 if e else 0.375 for e in POP_EXC]
    return {
        "name": "microcircuit",
        "pop_names": list(POP_NAMES),
        "pop_sizes": list(POP_SIZES_FULL),
        "pop_exc": list(POP_EXC),
        "conn_prob": [list(map(float, r)) for r in tab["conn_prob"]],
        "conn_scale": 1.0,
        "w_mean": w_mean,
        "w_sd": w_sd,
        "w_scale": 1.0,
        "proj_scale": [[1.0] * 8 for _ in range(8)],
        "d_mean": d_mean,
        "d_sd": d_sd,
        "k_ext": list(map(float, tab["k_ext"])),
        "nu_bg": 8.0,
        "w_ext": 87.8,
        "input_mode": 0,          # 0 = Poisson background, 1 = DC background
        "i_dc": [0.0] * 8,
        "tau_m": 10.0,            # ms
        "c_m": 250.0,             # pF
        "tau_syn": 0.5,           # ms
        "t_ref": 2.0,             # ms
        "theta": 15.0,            # mV above rest (V_th - E_L = -50 - (-65))
        "dt": 0.1,                # ms
        "u0_lo": float(tab["u0_lo"]),
        "u0_hi": float(tab["u0_hi"]),
        "ring_depth": RING_DEPTH,
        "seed": 12345,
    }


def microcircuit(scale=1.0, seed: int = 12345, input_mode: str = "poisson") -> dict:
    """Microcircuit at ``scale`` x the full size.

    * ``scale <= 1``: population sizes x scale, connection probabilities kept
      (so in-degrees scale by ``scale``), recurrent weights x 1/scale.
    * ``scale > 1``: population sizes x scale, probabilities x 1/scale (same
      in-degrees), weights unchanged.
    The background (K_ext, w_ext) is not scaled.
    """
    cfg = base_config()
    s = Fraction(str(scale))
    cfg["pop_sizes"] = population_sizes(scale)
    if s <= 1:
        cfg["conn_scale"] = 1.0
        cfg["w_scale"] = float(1 / s)
    else:
        cfg["conn_scale"] = float(1 / s)
        cfg["w_scale"] = 1.0
    cfg["seed"] = int(seed)
    cfg["scale"] = float(scale)
    if input_mode == "dc":
        cfg = dc_variant(cfg)
    return cfg


def dc_variant(cfg: dict) -> dict:
    """DC-background version (Sec. 2.1 / Sec. 3.1.3): the Poisson drive is
    replaced by its mean current K_ext * nu_bg * w_ext * tau_syn."""
    c = copy.deepcopy(cfg)
    c["input_mode"] = 1
    c["i_dc"] = [k * c["nu_bg"] * 1e-3 * c["w_ext"] * c["tau_syn"] for k in c["k_ext"]]
    return c


def batched_instances(n: int = 64, seed: int = 7, lo: float = 0.05, hi: float = 0.25):
    """``n`` independent microcircuits at scales ~ U(lo, hi), distinct seeds.

    Scales are rounded to 4 decimals so that population sizes are exact
    decimal roundings.
    """
    rng = np.random.default_rng(seed)
    scales = np.round(rng.uniform(lo, hi, n), 4)
    seeds = rng.integers(1, 2**62, n)
    return [microcircuit(float(s), int(sd)) for s, sd in zip(scales, seeds)]


def target_rates(seed: int = 11):
    """Target population rates ~ U(1, 10) Hz for the rate-fitting loss."""
    rng = np.random.default_rng(seed)
    return rng.uniform(1.0, 10.0, 8)


def n_neurons(cfg: dict) -> int:
    return int(sum(cfg["pop_sizes"]))


def random_membrane(cfg: dict, seed: int, lo: float = 0.0, hi: float | None = None):
    """Seeded fp32 membrane potentials (mV above rest), uniform in [lo, hi)."""
    hi = cfg["theta"] if hi is None else hi
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, n_neurons(cfg)).astype(np.float32)


def transient_membrane(cfg: dict, seed: int, n_above: int, lo_above: float = 16.0,
                       hi_above: float = 30.0):
    """Seeded fp32 membrane potentials of an unrelaxed start: ``n_above``
    distinct neurons drawn uniformly in [lo_above, hi_above) mV, far enough
    above the 15 mV threshold to stay above it after one step of leak, the
    rest uniform in [0, theta).  The paper starts from relaxed values because
    unrelaxed ones fire more than 4000 neurons in the first step (Sec. 2.3);
    this input reproduces that transient on purpose."""
    rng = np.random.default_rng(seed)
    n = n_neurons(cfg)
    u = rng.uniform(0.0, cfg["theta"], n)
    above = rng.choice(n, min(int(n_above), n), replace=False)
    u[above] = rng.uniform(lo_above, hi_above, above.size)
    return u.astype(np.float32)


def random_spike_list(n_neurons_: int, n_spikes: int, seed: int):
    """Distinct random source neuron ids, as a delivery-test spike list."""
    rng = np.random.default_rng(seed)
    n_spikes = min(n_spikes, n_neurons_)
    return np.sort(rng.choice(n_neurons_, n_spikes, replace=False)).astype(np.uint32)


def tiny_network(n_neurons_: int, synapses, weights_pa, delays, theta=15.0):
    """A hand-set network description for brute-force tests.

    ``synapses`` is a list of (source, target, weight_index, delay_steps);
    ``weights_pa`` lists the distinct weights (pA).  Returned as plain lists;
    each implementation builds its own structures from it.
    """
    return {
        "n": int(n_neurons_),
        "synapses": [tuple(int(v) for v in s) for s in synapses],
        "weights_pa": [float(w) for w in weights_pa],
        "theta": float(theta),
    }
