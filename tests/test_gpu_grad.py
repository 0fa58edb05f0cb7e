"""Differentiable microcircuit on the GPU: parameter updates, state
save/load, and the surrogate-gradient backward against the oracle's."""
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
from paper_1909_08665_gb300.autograd import microcircuit_rates  # noqa: E402


def _alpha(seed):
    """Projection scales around 1 (a few well away from it)."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.8, 1.2, (8, 8))
    a[0, 2] = 0.5
    a[7, 6] = 1.6
    return a


def test_set_params_matches_oracle():
    cfg = workload.microcircuit(0.05, seed=21)
    alpha, nu = _alpha(1), 9.5
    net = pkg.Microcircuit(cfg, stream=torch.cuda.current_stream())
    net.set_params(alpha, nu)
    net.step(400)
    net.sync()
    sim = oracle.Simulation(oracle.Network(oracle.with_params(cfg, alpha, nu)))
    sim.run(400)
    g = net.read_spikes()
    o = sim.raster()
    assert o[0].size > 100
    np.testing.assert_array_equal(g[0], o[0])
    np.testing.assert_array_equal(g[1], o[1])
    np.testing.assert_array_equal(net.state()[0].view(np.uint32), sim.state()[0].view(np.uint32))
    with pytest.raises(pkg.SnnError):
        net.set_params(np.full((8, 8), np.nan), nu)
    with pytest.raises(pkg.SnnError):
        net.set_params(alpha, -1.0)


def test_save_load_state_resumes_bit_exact():
    cfg = workload.microcircuit(0.05, seed=22)
    net = pkg.Microcircuit(cfg, stream=torch.cuda.current_stream())
    net.step(150)
    net.read_spikes()
    snap = net.save_state()
    net.step(333)
    a = net.read_spikes()
    sa = net.state()
    net.load_state(snap)
    assert net.counters()["step"] == 150
    net.step(333)
    b = net.read_spikes()
    sb = net.state()
    assert a[0].size > 0
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    for x, y in zip(sa, sb):
        np.testing.assert_array_equal(x.view(np.uint32), y.view(np.uint32))
    # a state of another network is refused
    other = pkg.Microcircuit(workload.microcircuit(0.02), stream=torch.cuda.current_stream())
    with pytest.raises(pkg.SnnError):
        other.load_state(snap)


def _parse_state(buf, n):
    """The layout snn_save_state documents: a 32-byte header (magic, n, step,
    ring depth as uint64), then u[n] f32, I[n] f32, refr[n] i32, ring[64][n] i32."""
    hdr = buf[:32].view(np.uint64)
    u = buf[32:32 + 4 * n].view(np.float32)
    i = buf[32 + 4 * n:32 + 8 * n].view(np.float32)
    r = buf[32 + 8 * n:32 + 12 * n].view(np.int32)
    ring = buf[32 + 12 * n:].view(np.int32).reshape(64, n)
    return hdr, u, i, r, ring


def test_resume_matches_oracle_both_ways():
    """A GPU state saved mid-run and loaded into the oracle, and an oracle
    state loaded into the GPU: each pair continues identically, bit for bit."""
    cfg = workload.microcircuit(0.05, seed=24)
    onet = oracle.Network(cfg)
    net = pkg.Microcircuit(cfg, stream=torch.cuda.current_stream())
    n = net.n
    # GPU -> oracle
    net.step(150)
    net.read_spikes()
    buf = net.save_state()
    hdr, u, i, r, ring = _parse_state(buf, n)
    assert int(hdr[1]) == n and int(hdr[2]) == 150 and int(hdr[3]) == 64
    sim = oracle.Simulation(onet)
    sim.set_state(u, i, r, ring.astype(np.int64), 150)
    net.step(333)
    sim.run(333)
    g, o = net.read_spikes(), sim.raster()
    assert o[0].size > 100 and o[0].min() >= 150
    np.testing.assert_array_equal(g[0], o[0])
    np.testing.assert_array_equal(g[1], o[1])
    g_u, g_i, g_r = net.state()
    o_u, o_i, o_r, o_ring = sim.state()
    np.testing.assert_array_equal(g_u.view(np.uint32), o_u.view(np.uint32))
    np.testing.assert_array_equal(g_i.view(np.uint32), o_i.view(np.uint32))
    np.testing.assert_array_equal(g_r, o_r)
    np.testing.assert_array_equal(net.ring(), o_ring.astype(np.int32))
    # oracle -> GPU: an oracle run of 700 steps from its own initial state
    sim2 = oracle.Simulation(onet)
    sim2.run(700)
    sim2.raster()
    o_u, o_i, o_r, o_ring = sim2.state()
    buf2 = buf.copy()
    hdr2, u2, i2, r2, ring2 = _parse_state(buf2, n)
    hdr2[2] = 700
    u2[:], i2[:], r2[:] = o_u, o_i, o_r
    ring2[:] = o_ring.astype(np.int32)
    other = pkg.Microcircuit(cfg, stream=torch.cuda.current_stream())
    other.load_state(buf2)
    assert other.counters()["step"] == 700
    other.step(250)
    sim2.run(250)
    g, o = other.read_spikes(), sim2.raster()
    assert o[0].size > 100 and o[0].min() >= 700
    np.testing.assert_array_equal(g[0], o[0])
    np.testing.assert_array_equal(g[1], o[1])
    g_u, g_i, g_r = other.state()
    o_u, o_i, o_r, o_ring = sim2.state()
    np.testing.assert_array_equal(g_u.view(np.uint32), o_u.view(np.uint32))
    np.testing.assert_array_equal(g_i.view(np.uint32), o_i.view(np.uint32))
    np.testing.assert_array_equal(g_r, o_r)
    np.testing.assert_array_equal(other.ring(), o_ring.astype(np.int32))


@pytest.fixture(scope="module")
def config3():
    """Differentiable workload: 10 % microcircuit, 2000 steps (200 ms), rate
    MSE against targets drawn uniformly from 1-10 Hz, checkpoints every 100
    steps; oracle forward and surrogate backward in double."""
    cfg = workload.microcircuit(0.1)
    targets = workload.target_rates()
    alpha0, nu0 = np.ones((8, 8)), float(cfg["nu_bg"])
    ref = oracle.hard_gradient(cfg, alpha0, nu0, 2000, targets, n_threads=os.cpu_count())
    return cfg, targets, alpha0, nu0, ref


def test_surrogate_gradient_matches_oracle(config3):
    cfg, targets, alpha0, nu0, ref = config3
    net = pkg.Microcircuit(cfg, stream=torch.cuda.current_stream())
    start = net.save_state()
    scales = torch.tensor(alpha0, dtype=torch.float64, requires_grad=True)
    nu = torch.tensor(nu0, dtype=torch.float64, requires_grad=True)
    rates = microcircuit_rates(scales, nu, net, 2000, 100, start)
    np.testing.assert_allclose(rates.detach().numpy(), ref["rates"], rtol=1e-12)
    loss = ((rates - torch.as_tensor(targets)) ** 2).mean()
    assert abs(loss.item() - ref["loss"]) <= 1e-12 * ref["loss"]
    loss.backward()
    # 2000 steps: the adjoint grows about e^0.039 per step (max|g| ~ 4e31 here),
    # and the fp32 rounding of the GPU adjoint grows with it, to ~1e-5 of its
    # largest component: the per-element floor is taken relative to max|g|
    assert_gradient_close(scales.grad.numpy(), nu.grad.item(), ref, rel=2e-3, floor=1e-5)
    # the backward leaves the network as the forward left it
    assert net.counters()["step"] == 2000


def assert_gradient_close(ga, gn, ref, rel=1e-3, floor=1e-6):
    """Element by element: |dg_pq| <= rel |g_pq| + floor max|g| for each of the
    64 projection scales (projections with no synapse have g = 0 on both
    sides), and 1e-4 relative for the background rate.  The GPU adjoint is
    fp32 with double accumulation, the oracle's double throughout."""
    g = ref["g_alpha"]
    gmax = np.abs(g).max()
    assert gmax > 0
    err = np.abs(ga - g)
    bound = rel * np.abs(g) + floor * gmax
    bad = np.argwhere(err > bound)
    assert bad.size == 0, [(int(p), int(q), float(ga[p, q]), float(g[p, q])) for p, q in bad[:8]]
    assert abs(gn - ref["g_nu"]) <= 1e-4 * abs(ref["g_nu"]), (gn, ref["g_nu"])


@pytest.mark.parametrize("t_ref,steps,n_part", [(2.0, 100, 0), (0.0, 60, 0), (2.0, 100, 1)],
                         ids=["t_ref2ms", "t_ref0", "t_ref2ms_one_partition"])
def test_surrogate_gradient_short_horizon(t_ref, steps, n_part):
    """The cases whose oracle gradient is pinned by central differences of the
    smooth deviation model (2 % network, seed 5): the GPU gradient must match
    it element by element.  With the default partitions the adjoint gathers
    partition by partition in shared memory; with one partition spanning all
    eight populations it takes the global-ring gather."""
    cfg = workload.microcircuit(0.02, seed=5)
    cfg["t_ref"] = t_ref
    targets = workload.target_rates()
    alpha0, nu0 = np.ones((8, 8)), float(cfg["nu_bg"])
    ref = oracle.hard_gradient(cfg, alpha0, nu0, steps, targets, seed=5)
    kw = {"n_part": n_part} if n_part else {}
    net = pkg.Microcircuit(cfg, seed=5, stream=torch.cuda.current_stream(), **kw)
    start = net.save_state()
    scales = torch.tensor(alpha0, dtype=torch.float64, requires_grad=True)
    nu = torch.tensor(nu0, dtype=torch.float64, requires_grad=True)
    rates = microcircuit_rates(scales, nu, net, steps, 100, start)
    np.testing.assert_allclose(rates.detach().numpy(), ref["rates"], rtol=1e-12)
    loss = ((rates - torch.as_tensor(targets)) ** 2).mean()
    loss.backward()
    assert_gradient_close(scales.grad.numpy(), nu.grad.item(), ref)


@pytest.mark.parametrize("variant", ["dc_input", "three_partitions"])
def test_surrogate_gradient_variants(variant):
    """The adjoint against the oracle's on the 2 % network (seed 5, 100 steps)
    with DC input in place of the Poisson drive (no nu gradient), and with
    three partitions of uneven population mix."""
    cfg = workload.microcircuit(0.02, seed=5)
    kw = {}
    if variant == "dc_input":
        cfg = workload.dc_variant(cfg)
    else:
        kw["n_part"] = 3
    steps = 100
    targets = workload.target_rates()
    alpha0, nu0 = _alpha(7), float(cfg["nu_bg"])
    ref = oracle.hard_gradient(cfg, alpha0, nu0, steps, targets, seed=5)
    net = pkg.Microcircuit(cfg, seed=5, stream=torch.cuda.current_stream(), **kw)
    start = net.save_state()
    scales = torch.tensor(alpha0, dtype=torch.float64, requires_grad=True)
    nu = torch.tensor(nu0, dtype=torch.float64, requires_grad=True)
    rates = microcircuit_rates(scales, nu, net, steps, 30, start)
    np.testing.assert_allclose(rates.detach().numpy(), ref["rates"], rtol=1e-12)
    loss = ((rates - torch.as_tensor(targets)) ** 2).mean()
    loss.backward()
    assert_gradient_close(scales.grad.numpy(), nu.grad.item(), ref)
    if variant == "dc_input":
        assert nu.grad.item() == 0.0 and ref["g_nu"] == 0.0


def test_gradient_independent_of_checkpoint_spacing(config3):
    """The same gradient bit for bit for every checkpoint spacing, whether the
    forward keeps the whole trajectory or the backward re-runs each segment
    from its checkpoint (trace budget 0)."""
    cfg, targets, alpha0, nu0, _ = config3
    net = pkg.Microcircuit(cfg, stream=torch.cuda.current_stream())
    start = net.save_state()
    out = []
    for every, budget in ((100, 4 << 30), (37, 4 << 30), (2000, 4 << 30), (100, 0), (37, 0)):
        net.set_grad_trace_budget(budget)
        net.load_state(start)
        net.set_params(alpha0, nu0)
        r = net.grad_forward(2000, every)
        out.append(net.grad_backward(oracle.rate_loss_grad(r, targets)))
    for ga, gn in out[1:]:
        np.testing.assert_array_equal(ga, out[0][0])
        assert gn == out[0][1]
    with pytest.raises(pkg.SnnError) as e:
        net.set_grad_trace_budget(-1)
    assert e.value.code == pkg.SNN_ERR_INVALID


def test_backward_restores_state_counters_and_raster():
    cfg = workload.microcircuit(0.05, seed=23)
    net = pkg.Microcircuit(cfg, stream=torch.cuda.current_stream())
    with pytest.raises(pkg.SnnError):
        net.grad_backward(np.ones(8))              # no forward yet
    r = net.grad_forward(450, 100)
    after = net.state()
    c_after = net.counters()
    n_ras = net.raster_size()
    ga, gn = net.grad_backward(np.ones(8))
    assert np.isfinite(ga).all() and np.isfinite(gn)
    for x, y in zip(after, net.state()):
        np.testing.assert_array_equal(x.view(np.uint32), y.view(np.uint32))
    assert net.counters() == c_after
    assert net.raster_size() == n_ras
    st, ids = net.read_spikes()
    pops = oracle.pop_of(cfg, ids)
    counts = np.bincount(pops, minlength=8)
    T = 450 * cfg["dt"] * 1e-3
    np.testing.assert_allclose(r, counts / (np.asarray(cfg["pop_sizes"]) * T), rtol=1e-12)
    net.step(1)
    with pytest.raises(pkg.SnnError):
        net.grad_backward(np.ones(8))              # stepped since the forward
