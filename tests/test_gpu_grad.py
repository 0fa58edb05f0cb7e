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
    ga = scales.grad.numpy()
    gmax = np.abs(ref["g_alpha"]).max()
    assert gmax > 0
    err = np.abs(ga - ref["g_alpha"]).max()
    assert err <= 1e-4 * gmax, (err, gmax)
    assert abs(nu.grad.item() - ref["g_nu"]) <= 1e-4 * abs(ref["g_nu"]), (nu.grad.item(), ref["g_nu"])
    # the backward leaves the network as the forward left it
    assert net.counters()["step"] == 2000


def test_gradient_independent_of_checkpoint_spacing(config3):
    cfg, targets, alpha0, nu0, _ = config3
    net = pkg.Microcircuit(cfg, stream=torch.cuda.current_stream())
    start = net.save_state()
    out = []
    for every in (100, 37, 2000):
        net.load_state(start)
        net.set_params(alpha0, nu0)
        r = net.grad_forward(2000, every)
        out.append(net.grad_backward(oracle.rate_loss_grad(r, targets)))
    for ga, gn in out[1:]:
        np.testing.assert_array_equal(ga, out[0][0])
        assert gn == out[0][1]


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
