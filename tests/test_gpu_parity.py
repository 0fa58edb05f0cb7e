"""GPU path versus the CPU oracle, element by element, through the C ABI.

The bar is bit-exact: spike rasters (step, id), fp32 membrane potentials and
synaptic currents (compared as bit patterns), refractory counters, int32 ring
buffers and the synaptic matrix itself.
"""
import time

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


@pytest.fixture(scope="module")
def cfg01():
    return workload.microcircuit(0.1)


@pytest.fixture(scope="module")
def onet01(cfg01):
    return oracle.Network(cfg01)


def gpu_net(cfg, **kw):
    return pkg.Microcircuit(cfg, stream=torch.cuda.current_stream(), **kw)


def oracle_words(onet):
    rp, tg, dl, wc = onet.export()
    return rp.astype(np.uint64), pkg.encode_words(tg, dl, wc)


def assert_state_equal(net, sim):
    g_u, g_i, g_r = net.state()
    o_u, o_i, o_r, o_ring = sim.state()
    np.testing.assert_array_equal(g_u.view(np.uint32), o_u.view(np.uint32))
    np.testing.assert_array_equal(g_i.view(np.uint32), o_i.view(np.uint32))
    np.testing.assert_array_equal(g_r, o_r)
    assert np.all(np.abs(o_ring) < 2**31)
    np.testing.assert_array_equal(net.ring(), o_ring.astype(np.int32))


# ---------------------------------------------------------------------------
# network generation
# ---------------------------------------------------------------------------
def test_network_matches_oracle(cfg01, onet01):
    net = gpu_net(cfg01)
    rp, wd, wt = net.export_network()
    orp, owd = oracle_words(onet01)
    np.testing.assert_array_equal(rp, orp)
    np.testing.assert_array_equal(wd, owd)
    np.testing.assert_array_equal(wt, oracle.tables(cfg01)["wtab"])
    info = net.info()
    d, f = oracle.propagators(cfg01)
    assert info["propagators"] == [float(v) for v in f]
    assert info["n_ref"] == 20 and info["wext_q"] == oracle.tables(cfg01)["wext_q"]


@pytest.mark.parametrize("n_part", [2, 5, 61, 152])
def test_network_independent_of_partitioning(cfg01, onet01, n_part):
    net = gpu_net(cfg01, n_part=n_part)
    assert net.info()["n_part"] == n_part
    _, wd, _ = net.export_network()
    np.testing.assert_array_equal(wd, oracle_words(onet01)[1])


# ---------------------------------------------------------------------------
# time stepping: 10 % microcircuit, 100 ms
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n_part", [0, 2, 7, 64])
def test_raster_and_state_bit_exact(cfg01, onet01, n_part):
    steps = 1000
    net = gpu_net(cfg01, n_part=n_part)
    sim = oracle.Simulation(onet01)
    net.step(steps)
    net.sync()
    sim.run(steps)
    g_st, g_id = net.read_spikes()
    o_st, o_id = sim.raster()
    assert o_st.size > 1000
    np.testing.assert_array_equal(g_st, o_st)
    np.testing.assert_array_equal(g_id, o_id)
    assert_state_equal(net, sim)
    gc, oc = net.counters(), sim.counters()
    assert gc["spikes"] == oc["spikes"] and gc["events"] == oc["events"]
    assert not oc["saturated"]


@pytest.mark.parametrize("n_part", [0, 2])
def test_launch_boundaries_do_not_change_results(cfg01, onet01, n_part):
    """Launches of 0 to 371 steps: results equal one long run, with the ring
    in shared memory (default partitions) and in global memory (two
    partitions of 3,859 neurons)."""
    net = gpu_net(cfg01, n_part=n_part)
    sim = oracle.Simulation(onet01)
    for n in (1, 1, 2, 3, 5, 117, 0, 371):
        net.step(n)
    net.sync()
    sim.run(500)
    g = net.read_spikes()
    o = sim.raster()
    np.testing.assert_array_equal(g[0], o[0])
    np.testing.assert_array_equal(g[1], o[1])
    assert_state_equal(net, sim)


def test_user_initial_state_and_dc_input(cfg01):
    cfg = workload.dc_variant(cfg01)
    u0 = workload.random_membrane(cfg, seed=5)
    net = gpu_net(cfg, u0=u0)
    onet = oracle.Network(cfg)
    sim = oracle.Simulation(onet, u0=u0)
    net.step(600)
    sim.run(600)
    g = net.read_spikes()
    o = sim.raster()
    assert o[0].size > 100
    np.testing.assert_array_equal(g[0], o[0])
    np.testing.assert_array_equal(g[1], o[1])
    assert_state_equal(net, sim)


@pytest.mark.parametrize("n_part", [1, 3])
def test_other_seed_and_scale(n_part):
    # 5 % model (3,858 neurons): n_part 1 puts them all in one CTA
    cfg = workload.microcircuit(0.05, seed=987654321987)
    net = gpu_net(cfg, n_part=n_part)
    onet = oracle.Network(cfg)
    sim = oracle.Simulation(onet)
    net.step(400)
    sim.run(400)
    g = net.read_spikes()
    o = sim.raster()
    np.testing.assert_array_equal(g[0], o[0])
    np.testing.assert_array_equal(g[1], o[1])
    assert_state_equal(net, sim)


# ---------------------------------------------------------------------------
# hand-set networks through snn_create_from_rows
# ---------------------------------------------------------------------------
def test_tiny_network_from_rows():
    n = 6
    weights_q = [round(87.8 * 256 * 12), round(-351.2 * 256 * 3), round(87.8 * 256 * 20)]
    synapses = [(0, 1, 0, 3), (0, 2, 2, 15), (1, 3, 2, 1), (2, 3, 1, 5), (3, 4, 0, 40),
                (4, 5, 2, 63), (5, 0, 1, 9), (3, 5, 2, 2), (1, 0, 1, 30)]
    cfg = tiny_config(n, input_mode=1)
    cfg["pop_sizes"] = [1] * n
    cfg["pop_exc"] = [1] * n
    cfg["i_dc"] = [520.0, 480.0, 600.0, 450.0, 500.0, 390.0, 0.0, 0.0]
    desc = custom_network(n, synapses, weights_q)
    wt = np.zeros((8, 8, 128), np.int32)
    wt[:, :, :3] = np.asarray(weights_q, np.int32)
    desc["wtab"] = wt
    u0 = np.array([14.9, 5.0, 12.0, 0.0, 10.0, 3.0], np.float32)
    onet = oracle.Network(cfg, custom=desc)
    sim = oracle.Simulation(onet, u0=u0)
    rows = {"row_ptr": desc["row_ptr"].astype(np.uint64),
            "words": pkg.encode_words(desc["tgt"], desc["delay"], desc["wcode"]), "wtab": wt}
    net = gpu_net(cfg, u0=u0, rows=rows)
    net.step(700)
    sim.run(700)
    g = net.read_spikes()
    o = sim.raster()
    assert o[0].size > 20
    np.testing.assert_array_equal(g[0], o[0])
    np.testing.assert_array_equal(g[1], o[1])
    assert_state_equal(net, sim)


def test_empty_network_and_zero_steps():
    cfg = tiny_config(100, input_mode=0, nu_bg=8.0)
    cfg["k_ext"] = [2300.0] * 8
    net = gpu_net(cfg)
    assert net.info()["n_synapses"] == 0
    net.step(0)
    net.sync()
    assert net.counters()["step"] == 0
    onet = oracle.Network(cfg)
    sim = oracle.Simulation(onet)
    net.step(300)
    sim.run(300)
    g = net.read_spikes()
    o = sim.raster()
    assert o[0].size > 0
    np.testing.assert_array_equal(g[0], o[0])
    np.testing.assert_array_equal(g[1], o[1])
    assert_state_equal(net, sim)


# ---------------------------------------------------------------------------
# standalone delivery: every tiling against the oracle
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n_spikes", [1, 25, 93, 4000])
@pytest.mark.parametrize("tiling", [0, 1, 2, 3, 4, 5])
def test_deliver_matches_oracle(cfg01, onet01, n_spikes, tiling):
    net = gpu_net(cfg01)
    spikes = workload.random_spike_list(net.n, n_spikes, seed=n_spikes)
    spikes = np.r_[spikes, spikes[:3]].astype(np.uint32)     # duplicates allowed
    d = torch.from_numpy(spikes.astype(np.int32)).cuda()
    t = 12345
    net.deliver(d.data_ptr(), spikes.size, t, tiling)
    net.sync()
    ref = onet01.deliver(spikes.astype(np.int32), t)
    np.testing.assert_array_equal(net.ring(), ref.astype(np.int32))


@pytest.mark.parametrize("tiling", [0, 1, 2, 3, 4, 5])
def test_deliver_adds_to_a_live_ring(cfg01, onet01, tiling):
    """Delivery into a ring that already holds the inputs of 20 steps, twice
    in a row at different steps: the ring changes by exactly the oracle's
    delivery (int32 arithmetic modulo 2^32), and the event counter by the
    rows' lengths."""
    net = gpu_net(cfg01)
    net.step(20)
    net.sync()
    rp, _, _, _ = onet01.export()
    for k, (m, t) in enumerate([(4000, 20), (1500, 23)]):
        before = net.ring().astype(np.int64)
        ev0 = net.counters()["events"]
        spikes = workload.random_spike_list(net.n, m, seed=500 + k).astype(np.int32)
        d = torch.from_numpy(spikes).cuda()
        net.deliver(d.data_ptr(), spikes.size, t, tiling)
        net.sync()
        delta = (net.ring().astype(np.int64) - before) % 2**32
        ref = onet01.deliver(spikes, t).astype(np.int64) % 2**32
        np.testing.assert_array_equal(delta, ref)
        if tiling == 3:
            rl = np.diff(rp.astype(np.int64))
            assert net.counters()["events"] - ev0 == int(rl[spikes].sum())


def test_deliver_partition_tilings_with_global_ring(cfg01, onet01):
    """Two partitions of 3,859 neurons: the ring does not fit in shared memory
    and the partition tiling accumulates into global memory."""
    spikes = workload.random_spike_list(7717, 500, seed=3)
    d = torch.from_numpy(spikes.astype(np.int32)).cuda()
    ref = onet01.deliver(spikes.astype(np.int32), 77).astype(np.int32)
    for tiling in (2, 3):
        net = gpu_net(cfg01, n_part=2)
        assert net.info()["ring_in_shared"] == 0
        net.deliver(d.data_ptr(), spikes.size, 77, tiling)
        net.sync()
        np.testing.assert_array_equal(net.ring(), ref)
        net.close()
    net = gpu_net(cfg01, n_part=2)               # ring slices too large for clusters
    for tiling in (4, 5):                        # and for the streamed stages
        with pytest.raises(pkg.SnnError) as e:
            net.deliver(d.data_ptr(), spikes.size, 77, tiling)
        assert e.value.code == pkg.SNN_ERR_UNSUPPORTED


def test_realtime_pacing_keeps_the_wall_clock_and_the_results(cfg01):
    """Paced at 0.1 ms per step (the paper's true real time, Sec. 4.1): 2,000
    steps take 0.2 s of wall time, step ends are 0.1 ms apart, no deadline is
    missed, and the raster and state are those of an unpaced run."""
    steps, period = 2000, 100_000
    ref = gpu_net(cfg01)
    ref.step(steps)
    ref.sync()
    net = gpu_net(cfg01)
    buf = torch.zeros(steps, dtype=torch.int64, device="cuda")
    net.record_step_times(buf.data_ptr(), steps)
    net.set_realtime(period)
    t0 = time.perf_counter()
    net.step(steps // 2)
    net.step(steps - steps // 2)          # the schedule continues across calls
    net.sync()
    wall = time.perf_counter() - t0
    assert (steps - 1) * period * 1e-9 <= wall < steps * period * 1e-9 + 0.5
    d = np.diff(buf.cpu().numpy())
    assert abs(np.median(d) - period) < 0.02 * period
    assert d.min() > 0.5 * period
    st = net.realtime_stats()
    assert st["missed"] <= steps // 100, st
    g, o = net.read_spikes(), ref.read_spikes()
    np.testing.assert_array_equal(g[0], o[0])
    np.testing.assert_array_equal(g[1], o[1])
    for a, b in zip(net.state(), ref.state()):
        np.testing.assert_array_equal(a, b)
    net.set_realtime(0)                   # pacing off: fast again
    t0 = time.perf_counter()
    net.step(steps)
    net.sync()
    assert time.perf_counter() - t0 < 0.1
    with pytest.raises(pkg.SnnError):
        net.set_realtime(-1)
    net.close()
    ref.close()


def test_step_times_are_recorded(cfg01):
    net = gpu_net(cfg01)
    net.step(5)
    buf = torch.zeros(300, dtype=torch.int64, device="cuda")
    net.record_step_times(buf.data_ptr(), 250)
    net.step(120)
    net.step(200)                    # the recording stops after 250 steps
    net.record_step_times(None)
    net.step(10)
    net.sync()
    t = buf.cpu().numpy()
    assert np.all(t[:250] > 0) and np.all(t[250:] == 0)
    # the device clock never runs backwards (its tick may exceed one step)
    assert np.all(np.diff(t[:250]) >= 0) and t[249] > t[0]
    with pytest.raises(pkg.SnnError):
        net.record_step_times(buf.data_ptr(), 0)


# ---------------------------------------------------------------------------
# failure path: a barrier wait that runs out of time returns an error status
# ---------------------------------------------------------------------------
def test_barrier_timeout_reports_error_and_context_survives(cfg01):
    # partition 0 withholds its arrivals: every other wait runs out (50 ms)
    net = gpu_net(cfg01, n_part=8, timeout_s=0.05, inject_fault=1)
    net.step(50)
    with pytest.raises(pkg.SnnError) as e:
        net.sync()
    assert e.value.code == pkg.SNN_ERR_TIMEOUT
    net.close()
    ok = gpu_net(cfg01)
    ok.step(10)
    ok.sync()


def test_raster_reads_in_parts_and_with_a_short_cap(cfg01):
    """snn_read_spikes packs every partition's entries on the device: a read
    with a short cap returns the first entries in partition order and reports
    the rest as dropped, and reads between steps add up to one read of the
    whole run.  Within one step of one partition the recording order is not
    fixed (warps append concurrently), so the prefix is compared by the steps
    it covers and by membership."""
    a, b = gpu_net(cfg01), gpu_net(cfg01)
    a.step(300)
    b.step(300)
    full_st = np.zeros(1 << 20, np.uint32)
    full_id = np.zeros(1 << 20, np.uint32)
    n = a.read_spikes_into(full_st, full_id)
    assert n > 100
    st = np.zeros(n // 2, np.uint32)
    ids = np.zeros(n // 2, np.uint32)
    with pytest.raises(pkg.SnnError) as e:
        b.read_spikes_into(st, ids)
    assert e.value.code == pkg.SNN_ERR_OVERFLOW
    np.testing.assert_array_equal(np.sort(st), np.sort(full_st[:n // 2]))
    whole_a = set(zip(full_st[:n].tolist(), full_id[:n].tolist()))
    assert set(zip(st.tolist(), ids.tolist())) <= whole_a
    c, d = gpu_net(cfg01), gpu_net(cfg01)
    parts = []
    for _ in range(3):
        c.step(100)
        parts.append(c.read_spikes())
    d.step(300)
    whole = d.read_spikes()
    pst = np.concatenate([q[0] for q in parts])
    pid = np.concatenate([q[1] for q in parts])
    order = np.lexsort((pid, pst))
    np.testing.assert_array_equal(pst[order], whole[0])
    np.testing.assert_array_equal(pid[order], whole[1])
    for x in (a, b, c, d):
        x.close()


def test_raster_overflow_is_reported(cfg01):
    net = gpu_net(cfg01, raster_capacity=1)
    net.step(400)
    with pytest.raises(pkg.SnnError) as e:
        net.sync()
    assert e.value.code == pkg.SNN_ERR_OVERFLOW
