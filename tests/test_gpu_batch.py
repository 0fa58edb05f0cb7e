"""Batched instances (many independent microcircuits of uneven size and seed
in one persistent kernel replayed from a CUDA graph) against the oracle, one
instance at a time: rasters, fp32 state and event counts bit for bit, for each
delivery tiling (warp per spike, CTA per row, flat) and for the autotuner's
choice."""
import os

import numpy as np
import pytest

import oracle
import workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1909_08665_gb300 as pkg  # noqa: E402


def _mixed_instances():
    """Uneven sizes, distinct seeds, one DC-driven instance."""
    return [workload.microcircuit(0.03, seed=11),
            workload.microcircuit(0.05, seed=22),
            workload.dc_variant(workload.microcircuit(0.02, seed=33)),
            workload.microcircuit(0.04, seed=44),
            workload.microcircuit(0.013, seed=55)]


def _oracle_run(cfg, steps):
    """Raster, state and counters of the oracle after `steps` steps."""
    sim = oracle.Simulation(oracle.Network(cfg, n_threads=os.cpu_count()))
    sim.run(steps)
    return sim.raster(), sim.state(), sim.counters()


def _assert_instance_equal(batch, k, ref):
    (o_st, o_id), (o_u, o_i, o_r, _), oc = ref
    g = batch.read_spikes(k)
    assert o_st.size > 0
    np.testing.assert_array_equal(g[0], o_st)
    np.testing.assert_array_equal(g[1], o_id)
    g_u, g_i, g_r = batch.state(k)
    np.testing.assert_array_equal(g_u.view(np.uint32), o_u.view(np.uint32))
    np.testing.assert_array_equal(g_i.view(np.uint32), o_i.view(np.uint32))
    np.testing.assert_array_equal(g_r, o_r)
    c = batch.counters(k)
    assert c["spikes"] == oc["spikes"] and c["events"] == oc["events"]


@pytest.fixture(scope="module")
def oracle_runs():
    steps = 1250
    return steps, [_oracle_run(cfg, steps) for cfg in _mixed_instances()]


@pytest.mark.parametrize("tilings", [(0, 1, 2, 0, 1), (2, 0, 1, 2, 2), (2, 2, 2, 2, 2)])
def test_batch_forced_tilings_bit_exact(oracle_runs, tilings):
    steps, sims = oracle_runs
    cfgs = _mixed_instances()
    b = pkg.MicrocircuitBatch(cfgs, stream=torch.cuda.current_stream())
    info = b.info(0)
    assert info["graph"] == 1 and info["graph_steps"] == 1000
    for k, tl in enumerate(tilings):
        b.set_tiling(k, tl)
        assert b.info(k)["tiling"] == tl
    b.step(1000)            # one graph replay
    b.step(steps - 1000)    # plain launch for the remainder
    b.sync()
    for k, sim in enumerate(sims):
        _assert_instance_equal(b, k, sim)
    b.close()


def test_batch_autotuned_split_calls(oracle_runs):
    """The autotuner's tilings, stepped in uneven pieces (launch boundaries
    fall at arbitrary phases of the 4-step background cache and the 2- and
    4-step list parities)."""
    steps, sims = oracle_runs
    b = pkg.MicrocircuitBatch(_mixed_instances(), stream=torch.cuda.current_stream())
    for k in range(len(b)):
        inf = b.info(k)
        times = [inf["tune_us_warp"], inf["tune_us_block"], inf["tune_us_flat"]]
        assert min(times) > 0 and inf["tiling"] in (0, 1, 2)
        assert inf["trial_us_per_step"] > 0
    for n in (1, 2, 5, 1000, 241, 1):
        b.step(n)
    b.sync()
    for k, sim in enumerate(sims):
        _assert_instance_equal(b, k, sim)
    b.close()


def test_batch_zero_and_single_steps():
    cfgs = _mixed_instances()[:2]
    b = pkg.MicrocircuitBatch(cfgs, stream=torch.cuda.current_stream())
    b.step(0)
    b.sync()
    u0, i0, r0 = b.state(1)
    assert np.all(i0 == 0) and np.all(r0 == 0)
    sim = oracle.Simulation(oracle.Network(cfgs[1]))
    np.testing.assert_array_equal(u0.view(np.uint32), sim.state()[0].view(np.uint32))
    for _ in range(3):
        b.step(1)
    b.sync()
    sim.run(3)
    g_u, g_i, g_r = b.state(1)
    np.testing.assert_array_equal(g_u.view(np.uint32), sim.state()[0].view(np.uint32))
    np.testing.assert_array_equal(g_i.view(np.uint32), sim.state()[1].view(np.uint32))
    b.close()


def test_batch_of_64_uneven_instances():
    """The 64-instance workload (scales 0.05..0.25, distinct seeds) in its own
    launch shape; the smallest, the largest and one middle instance checked
    bit for bit against the oracle."""
    cfgs = workload.batched_instances(64)
    sizes = [workload.n_neurons(c) for c in cfgs]
    b = pkg.MicrocircuitBatch(cfgs, stream=torch.cuda.current_stream())
    info = b.info(0)
    assert info["n_neurons_total"] == sum(sizes)
    assert info["graph"] == 1
    steps = 120
    b.step(steps)
    b.sync()
    order = np.argsort(sizes)
    for k in (int(order[0]), int(order[32]), int(order[-1])):
        _assert_instance_equal(b, k, _oracle_run(cfgs[k], steps))
    for k in range(64):
        assert b.counters(k)["spikes"] > 0
    b.close()


def _with_delays(cfg, d_mean, d_sd):
    c = dict(cfg)
    c["d_mean"] = [d_mean] * 8
    c["d_sd"] = [d_sd] * 8
    return c


@pytest.mark.parametrize("long_delays", [False, True])
def test_batch_ring_depth_follows_longest_delay(long_delays):
    """The batch ring has one slot more than the longest delay of any
    instance: with delays of 1..3 steps it wraps every few steps; with one
    instance whose delays reach the 63-step cap beside them, all 64 slots are
    in use.  Every instance bit for bit against the oracle."""
    cfgs = [_with_delays(workload.microcircuit(0.03, seed=61), 0.2, 0.05),
            _with_delays(workload.microcircuit(0.02, seed=62), 0.15, 0.05)]
    if long_delays:
        cfgs.append(_with_delays(workload.microcircuit(0.025, seed=63), 3.0, 1.5))
    steps = 300
    b = pkg.MicrocircuitBatch(cfgs, stream=torch.cuda.current_stream())
    b.step(steps)
    b.sync()
    for k, cfg in enumerate(cfgs):
        _assert_instance_equal(b, k, _oracle_run(cfg, steps))
    b.close()


def test_batch_barrier_timeout_is_reported():
    cfgs = _mixed_instances()[:2]
    b = pkg.MicrocircuitBatch(cfgs, stream=torch.cuda.current_stream(), timeout_s=0.05,
                              inject_fault=1)
    b.step(5)
    with pytest.raises(pkg.SnnError) as ei:
        b.sync()
    assert ei.value.code == pkg.SNN_ERR_TIMEOUT
    b.close()
    # the context is still usable
    b2 = pkg.MicrocircuitBatch(cfgs, stream=torch.cuda.current_stream())
    b2.step(10)
    b2.sync()
    b2.close()


def test_batch_raster_overflow_is_reported():
    cfgs = _mixed_instances()[:2]
    b = pkg.MicrocircuitBatch(cfgs, stream=torch.cuda.current_stream(), raster_capacity=4)
    b.step(200)
    with pytest.raises(pkg.SnnError) as ei:
        b.sync()
    assert ei.value.code == pkg.SNN_ERR_OVERFLOW
    b.close()


def test_batch_rejects_bad_arguments():
    with pytest.raises(ValueError):
        pkg.MicrocircuitBatch([])
    cfg = workload.microcircuit(0.02)
    bad = dict(cfg)
    bad["ring_depth"] = 32
    with pytest.raises(pkg.SnnError) as ei:
        pkg.MicrocircuitBatch([cfg, bad])
    assert ei.value.code == pkg.SNN_ERR_INVALID
    b = pkg.MicrocircuitBatch([cfg])
    with pytest.raises(pkg.SnnError):
        b.set_tiling(0, 3)
    with pytest.raises(pkg.SnnError):          # instance index out of range
        pkg._check(pkg.lib().snn_batch_set_tiling(b._h, 1, 0))
    b.close()
