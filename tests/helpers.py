"""Shared test helpers: tiny hand-set networks and config builders.

The helpers only arrange inputs (parameters, synapse lists); they contain no
simulation arithmetic.
"""
import copy

import numpy as np

import workload

MAX_POP = 8
WCODES = 128


def tiny_config(n_neurons, input_mode=0, i_dc=0.0, nu_bg=0.0, u0=(0.0, 15.0)):
    """One population of ``n_neurons`` with no generated connectivity."""
    c = copy.deepcopy(workload.microcircuit(0.1))
    c["name"] = "tiny"
    c["pop_sizes"] = [int(n_neurons)]
    c["pop_exc"] = [1]
    c["conn_prob"] = [[0.0] * 8 for _ in range(8)]
    c["k_ext"] = [2000.0] * 8
    c["nu_bg"] = float(nu_bg)
    c["input_mode"] = int(input_mode)
    c["i_dc"] = [float(i_dc)] * 8
    c["w_scale"] = 1.0
    c["conn_scale"] = 1.0
    c["u0_lo"], c["u0_hi"] = float(u0[0]), float(u0[1])
    return c


def custom_network(n_neurons, synapses, weights_q):
    """CSR rows from (source, target, weight_code, delay) tuples.

    ``weights_q`` lists fixed-point weights (1/256 pA) indexed by code; they
    are placed in the population-0 -> population-0 table.
    """
    syn = sorted(synapses, key=lambda s: (s[0], s[1]))
    row_ptr = np.zeros(n_neurons + 1, np.int64)
    for s in syn:
        row_ptr[s[0] + 1] += 1
    row_ptr = np.cumsum(row_ptr)
    tgt = np.array([s[1] for s in syn], np.int32)
    wcode = np.array([s[2] for s in syn], np.uint8)
    delay = np.array([s[3] for s in syn], np.uint8)
    wtab = np.zeros((MAX_POP, MAX_POP, WCODES), np.int32)
    wtab[0, 0, :len(weights_q)] = np.asarray(weights_q, np.int32)
    return {"row_ptr": row_ptr, "tgt": tgt, "delay": delay, "wcode": wcode, "wtab": wtab}
