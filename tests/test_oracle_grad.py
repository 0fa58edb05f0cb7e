"""Pins of the oracle's gradient of the population-rate loss (BPTT of the
step recursion of Sec. 2.1 / Eq. 1) with respect to the 64 projection weight
scales and the background rate.

The adjoint routine is shared by the two models it serves, so each model pins
it against central finite differences of an explicit smooth forward:
  - sigmoid-relaxed model (its gradient is exact): FD of the relaxed forward;
  - hard model with the fast-sigmoid surrogate: FD of the model written as
    deviations around the recorded hard run, whose exact derivative at the
    recording's parameters is, by construction, the surrogate gradient.
Horizons are short enough that the linearised dynamics stay in the regime
where central differences converge as h^2 (the relaxed soft reset has a gain
of order u s' ~ 37 per step near threshold, so its horizon is the shorter).
"""
import numpy as np
import pytest

import oracle
import workload

PAIRS = [(0, 0), (2, 0), (0, 2), (1, 3), (3, 2), (5, 4), (7, 6), (4, 7)]


def _fd(fun, x0, h):
    return (fun(x0 + h) - fun(x0 - h)) / (2.0 * h)


@pytest.fixture(scope="module")
def relaxed_case():
    cfg = workload.microcircuit(0.02, seed=5)
    steps = 20
    targets = workload.target_rates()
    alpha0, nu0 = np.ones((8, 8)), cfg["nu_bg"]
    cp = oracle.with_params(cfg, alpha0, nu0)
    net = oracle.Network(cp)
    z = np.random.default_rng(3).standard_normal((steps, net.n))
    u0 = oracle.Simulation(net).state()[0].astype(np.float64)
    rates, ut, st = oracle.relaxed_forward(net, cp, steps, u0, z, record=True)
    ga, gn = oracle.grad_backward(net, cp, oracle.RELAXED, ut, st, None,
                                  oracle.rate_loss_grad(rates, targets), z)

    def loss(alpha, nu):
        c = oracle.with_params(cfg, alpha, nu)
        return oracle.rate_loss(oracle.relaxed_forward(net, c, steps, u0, z), targets)
    return loss, alpha0, nu0, ga, gn


def test_relaxed_gradient_matches_central_differences(relaxed_case):
    loss, alpha0, nu0, ga, gn = relaxed_case
    scale = np.abs(ga).max()
    assert scale > 0
    for p, q in PAIRS:
        e = np.zeros((8, 8))
        e[p, q] = 1.0
        fd = _fd(lambda x: loss(alpha0 + x * e, nu0), 0.0, 1e-6)
        assert abs(fd - ga[p, q]) <= 1e-6 * scale, (p, q, fd, ga[p, q])
    fd = _fd(lambda x: loss(alpha0, nu0 + x), 0.0, 1e-5)
    assert abs(fd - gn) <= 1e-6 * abs(gn), (fd, gn)


@pytest.fixture(scope="module", params=[(2.0, 100), (0.0, 60)], ids=["t_ref2ms", "t_ref0"])
def hard_case(request):
    """t_ref = 0 lets a neuron update right after its spike, so the detached
    reset (not the refractory gate) is what stops the gradient there; without
    refractoriness the network is more active and its horizon shorter."""
    cfg = workload.microcircuit(0.02, seed=5)
    cfg["t_ref"], steps = request.param
    targets = workload.target_rates()
    alpha0, nu0 = np.ones((8, 8)), cfg["nu_bg"]
    res = oracle.hard_gradient(cfg, alpha0, nu0, steps, targets, seed=5)

    def loss(alpha, nu):
        r = oracle.surrogate_forward(res["net"], res["cfg"], alpha, nu, steps, res["u0"],
                                     res["u"], res["flags"], res["k"])
        return oracle.rate_loss(r, targets)
    return loss, alpha0, nu0, res


def test_deviation_model_is_the_hard_run_at_its_parameters(hard_case):
    loss, alpha0, nu0, res = hard_case
    r = oracle.surrogate_forward(res["net"], res["cfg"], alpha0, nu0, res["u"].shape[0],
                                 res["u0"], res["u"], res["flags"], res["k"])
    np.testing.assert_array_equal(r, res["rates"])
    assert (res["flags"] & 1).sum() > 100


def test_surrogate_gradient_matches_central_differences(hard_case):
    loss, alpha0, nu0, res = hard_case
    ga, gn = res["g_alpha"], res["g_nu"]
    scale = np.abs(ga).max()
    assert scale > 0
    for p, q in PAIRS:
        e = np.zeros((8, 8))
        e[p, q] = 1.0
        fd = _fd(lambda x: loss(alpha0 + x * e, nu0), 0.0, 1e-6)
        assert abs(fd - ga[p, q]) <= 1e-5 * scale, (p, q, fd, ga[p, q])
    fd = _fd(lambda x: loss(alpha0, nu0 + x), 0.0, 1e-5)
    assert abs(fd - gn) <= 1e-5 * abs(gn), (fd, gn)


def test_gradient_is_linear_in_the_loss_weights(hard_case):
    _, _, _, res = hard_case
    net, cp = res["net"], res["cfg"]
    s = (res["flags"] & 1).astype(np.float64)
    g1 = np.zeros(8); g1[2] = 1.0
    g2 = np.zeros(8); g2[6] = -0.5
    a1, n1 = oracle.grad_backward(net, cp, oracle.HARD, res["u"], s, res["flags"], g1)
    a2, n2 = oracle.grad_backward(net, cp, oracle.HARD, res["u"], s, res["flags"], g2)
    a3, n3 = oracle.grad_backward(net, cp, oracle.HARD, res["u"], s, res["flags"], g1 + g2)
    np.testing.assert_allclose(a3, a1 + a2, rtol=1e-12, atol=1e-12 * np.abs(a3).max())
    assert abs(n3 - (n1 + n2)) <= 1e-12 * abs(n3)
    a0, n0 = oracle.grad_backward(net, cp, oracle.HARD, res["u"], s, res["flags"], np.zeros(8))
    assert np.all(a0 == 0.0) and n0 == 0.0
