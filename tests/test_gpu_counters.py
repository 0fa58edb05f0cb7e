"""Fixed-point saturation status and per-step synapse counts, on the GPU
against the CPU oracle.

Saturation: synaptic input is accumulated as int32 fixed point (1/256 pA).
The oracle accumulates in int64 and flags a step whose input leaves the
int32 range; the GPU must raise SNN_ERR_SATURATED in exactly those runs (and
not when a sum wraps on the way but ends in range), while rasters and state
stay bit-exact (both wrap the input modulo 2^32).  Networks whose input bound
stays below 2^31 -- the benchmark's -- take the unchecked kernel.

Per-step counts (the synapse-core profile of Sec. 4.1, Fig. 7): spikes and
synaptic events per step, the busiest partition's processed spikes and the
spike/partition pairs with no target, recomputed here from the oracle's
raster and rows.
"""
import numpy as np
import pytest

import oracle
import workload
from helpers import custom_network, tiny_config

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1909_08665_gb300 as pkg  # noqa: E402


def _tiny(weights_q, sources, steps=40):
    """Neurons 0..k-1 start above threshold and spike in step 0; each has one
    synapse (delay 3, weight code = its index) onto neuron 5."""
    n = 6
    cfg = tiny_config(n, input_mode=1, i_dc=0.0)
    syn = [(s, 5, s, 3) for s in sources]
    desc = custom_network(n, syn, weights_q)
    u0 = np.zeros(n, np.float32)
    u0[list(sources)] = 20.0
    sim = oracle.Simulation(oracle.Network(cfg, custom=desc), u0=u0)
    sim.run(steps)
    rows = {"row_ptr": desc["row_ptr"].astype(np.uint64),
            "words": pkg.encode_words(desc["tgt"], desc["delay"], desc["wcode"]),
            "wtab": desc["wtab"]}
    net = pkg.Microcircuit(cfg, u0=u0, rows=rows, stream=torch.cuda.current_stream())
    assert net.info()["saturation_check"] == 1
    net.step(steps)
    try:
        net.sync()
        code = pkg.SNN_OK
    except pkg.SnnError as e:
        code = e.code
    g, o = net.read_spikes(), sim.raster()
    np.testing.assert_array_equal(g[0], o[0])
    np.testing.assert_array_equal(g[1], o[1])
    g_u, g_i, g_r = net.state()
    o_u, o_i, o_r, _ = sim.state()
    np.testing.assert_array_equal(g_u.view(np.uint32), o_u.view(np.uint32))
    np.testing.assert_array_equal(g_i.view(np.uint32), o_i.view(np.uint32))
    np.testing.assert_array_equal(g_r, o_r)
    return code, sim.counters()["saturated"]


W = int(0.9 * 2**30)


@pytest.mark.parametrize("weights,sources,saturates", [
    ([W, W, W], [0, 1, 2], True),                       # 2.7 * 2^30: above the range
    ([W, W, W, -W], [0, 1, 2, 3], False),               # may wrap on the way, ends in range
    ([2**30, 2**30 - 1], [0, 1], False),                # 2^31 - 1: the top of the range
    ([2**30, 2**30], [0, 1], True),                     # 2^31: one past it
    ([-2**30, -2**30], [0, 1], False),                  # -2^31: the bottom of the range
    ([-2**30, -2**30 - 1], [0, 1], True),               # -2^31 - 1
])
def test_saturation_flag_matches_oracle(weights, sources, saturates):
    code, o_sat = _tiny(weights, sources)
    assert o_sat == saturates
    assert code == (pkg.SNN_ERR_SATURATED if saturates else pkg.SNN_OK)


def test_checked_kernel_on_a_network_that_can_saturate():
    """The 10 % microcircuit with weights x8: its input bound (1.2 * 2^31)
    passes the int32 range, so it runs the kernel that counts wrap-arounds;
    300 steps bit for bit, and the same saturation verdict as the oracle
    (none: excitation and inhibition cancel far below the bound).  The batch
    refuses it."""
    cfg = workload.microcircuit(0.1)
    cfg["w_scale"] = cfg["w_scale"] * 8.0
    net = pkg.Microcircuit(cfg, stream=torch.cuda.current_stream())
    info = net.info()
    assert info["saturation_check"] == 1 and info["input_bound"] > 2**31
    sim = oracle.Simulation(oracle.Network(cfg))
    net.step(300)
    sim.run(300)
    try:
        net.sync()
        g_sat = False
    except pkg.SnnError as e:
        assert e.code == pkg.SNN_ERR_SATURATED
        g_sat = True
    assert g_sat == sim.counters()["saturated"]
    g, o = net.read_spikes(), sim.raster()
    assert o[0].size > 100
    np.testing.assert_array_equal(g[0], o[0])
    np.testing.assert_array_equal(g[1], o[1])
    g_u, g_i, g_r = net.state()
    o_u, o_i, o_r, o_ring = sim.state()
    np.testing.assert_array_equal(g_u.view(np.uint32), o_u.view(np.uint32))
    np.testing.assert_array_equal(g_i.view(np.uint32), o_i.view(np.uint32))
    np.testing.assert_array_equal(net.ring(), o_ring.astype(np.int32))
    with pytest.raises(pkg.SnnError) as e:
        pkg.MicrocircuitBatch([cfg], stream=torch.cuda.current_stream())
    assert e.value.code == pkg.SNN_ERR_SATURATED


@pytest.mark.parametrize("scale", [0.1, 1.0, 4.0])
def test_benchmark_networks_cannot_saturate(scale):
    net = pkg.Microcircuit(workload.microcircuit(scale), stream=torch.cuda.current_stream())
    info = net.info()
    assert info["saturation_check"] == 0
    assert 0 < info["input_bound"] < 2**31
    net.close()


def _expected_counts(cfg, onet, steps, ids, n_part, t0, n_steps):
    rp, tg, _, _ = onet.export()
    n = int(sum(cfg["pop_sizes"]))
    part_lo = (np.arange(n_part + 1, dtype=np.int64) * n) // n_part
    out = np.zeros((n_steps, 4), np.int64)
    for t, j in zip(steps, ids):
        r = t - t0
        if not 0 <= r < n_steps:
            continue
        row = tg[rp[j]:rp[j + 1]]
        parts = np.unique(np.searchsorted(part_lo, row, side="right") - 1)
        out[r, 0] += 1
        out[r, 1] += row.size
        out[r, 3] += n_part - parts.size
    # busiest partition: per step, spikes with at least one target in it
    for r in range(n_steps):
        sel = ids[steps == t0 + r]
        if sel.size == 0:
            continue
        per_part = np.zeros(n_part, np.int64)
        for j in sel:
            row = tg[rp[j]:rp[j + 1]]
            per_part[np.unique(np.searchsorted(part_lo, row, side="right") - 1)] += 1
        out[r, 2] = per_part.max()
    return out


@pytest.mark.parametrize("transient", [False, True])
def test_step_counts_match_oracle(transient):
    """Recording from step t0 (0 for the transient, whose first step has 1,500
    spikes and takes the chunked path), over two launches and 30 steps past
    the record's end; the record must equal the counts recomputed from the
    oracle's raster and rows, and its totals the library's counters."""
    cfg = workload.microcircuit(0.1)
    u0 = workload.transient_membrane(cfg, seed=41, n_above=1500) if transient else None
    net = pkg.Microcircuit(cfg, u0=u0, stream=torch.cuda.current_stream())
    onet = oracle.Network(cfg)
    sim = oracle.Simulation(onet, u0=u0)
    t0 = 0 if transient else 7
    net.step(t0)
    steps = 400
    buf = torch.zeros(4 * (steps + 50), dtype=torch.int32, device="cuda")
    net.record_step_counts(buf.data_ptr(), steps)
    c0 = net.counters()
    net.step(150)
    net.step(steps - 150 + 30)                    # 30 steps past the record's end
    net.record_step_counts(None)
    net.sync()
    c1 = net.counters()
    sim.run(t0 + steps + 30)
    o_st, o_id = sim.raster()
    got = buf.cpu().numpy().view(np.uint32).astype(np.int64).reshape(-1, 4)
    assert np.all(got[steps:] == 0)
    got = got[:steps]
    n_part = net.info()["n_part"]
    want = _expected_counts(cfg, onet, o_st, o_id, n_part, t0, steps + 30)
    np.testing.assert_array_equal(got, want[:steps])
    # totals: the library's counters over the same steps
    assert c1["spikes"] - c0["spikes"] == want[:, 0].sum()
    assert c1["events"] - c0["events"] == want[:, 1].sum()
    if transient:
        assert got[0, 0] == 1500 and got[0, 2] <= 1500
