"""snn_step_noalloc against snn_step, through the C ABI, on two calls in a row.

snn_step_noalloc serves callers that may not allocate device memory while
they run (an application stepping the network in a closed real-time loop,
with all of its device memory reserved up front): it steps a network held in
the caller's own buffers and keeps its scratch in a static device array.
The test owns every buffer (torch tensors), runs both entry points on the
same network and initial state, and requires identical spikes, state, ring
buffers and counters after each of two consecutive calls.

This file is collected last, so a run that stops at its first failure has
already run every other test.
"""
import numpy as np
import pytest

import workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1909_08665_gb300 as pkg  # noqa: E402


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a).view(dtype)).cuda()


def test_noalloc_matches_step_on_two_calls():
    cfg = workload.microcircuit(0.1)
    stream = torch.cuda.current_stream()
    ref = pkg.Microcircuit(cfg, stream=stream)
    rp, words, wtab = ref.export_network()
    u0, i0, r0 = ref.state()
    ring0 = ref.ring()

    d_rp = _dev(rp, np.int64)
    d_words = _dev(words, np.int32)
    d_wtab = _dev(wtab.reshape(-1), np.int32)
    d_u = _dev(u0.copy(), np.float32)
    d_i = _dev(i0.copy(), np.float32)
    d_r = _dev(r0.copy(), np.int32)
    d_ring = _dev(ring0.reshape(-1).copy(), np.int32)
    cap = 1 << 20
    d_rs = torch.zeros(cap, dtype=torch.int32, device="cuda")
    d_ri = torch.zeros(cap, dtype=torch.int32, device="cuda")
    d_rn = torch.zeros(1, dtype=torch.int32, device="cuda")
    d_cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
    d_status = torch.zeros(1, dtype=torch.int32, device="cuda")
    io = pkg.SnnNoallocIO(
        row_ptr=d_rp.data_ptr(), words=d_words.data_ptr(), wtab=d_wtab.data_ptr(),
        u=d_u.data_ptr(), i_syn=d_i.data_ptr(), refr=d_r.data_ptr(), ring=d_ring.data_ptr(),
        ras_step=d_rs.data_ptr(), ras_id=d_ri.data_ptr(), ras_n=d_rn.data_ptr(), ras_cap=cap,
        counters=d_cnt.data_ptr(), status=d_status.data_ptr())

    t0 = 0
    for n in (300, 450):
        pkg.step_noalloc(cfg, cfg["seed"], io, t0, n, stream)
        ref.step(n)
        ref.sync()
        torch.cuda.synchronize()
        assert int(d_status.item()) == 0
        g_st, g_id = ref.read_spikes()
        nrec = int(d_rn.item())
        assert 0 < nrec <= cap
        st = d_rs[:nrec].cpu().numpy().astype(np.int64)
        ids = d_ri[:nrec].cpu().numpy().astype(np.int64)
        order = np.lexsort((ids, st))
        np.testing.assert_array_equal(st[order], g_st)
        np.testing.assert_array_equal(ids[order], g_id)
        d_rn.zero_()
        u, i, r = ref.state()
        np.testing.assert_array_equal(d_u.cpu().numpy().view(np.uint32), u.view(np.uint32))
        np.testing.assert_array_equal(d_i.cpu().numpy().view(np.uint32), i.view(np.uint32))
        np.testing.assert_array_equal(d_r.cpu().numpy(), r)
        np.testing.assert_array_equal(d_ring.cpu().numpy().reshape(64, -1), ref.ring())
        c = ref.counters()
        assert int(d_cnt[0].item()) == c["spikes"] and int(d_cnt[1].item()) == c["events"]
        t0 += n


def _noalloc_buffers(cfg, rp, words, wtab, u0, cap):
    """Every device buffer of snn_step_noalloc, owned by the test (torch)."""
    n = int(sum(cfg["pop_sizes"]))
    bufs = {
        "rp": _dev(rp, np.int64), "words": _dev(words, np.int32),
        "wtab": _dev(np.asarray(wtab, np.int32).reshape(-1), np.int32),
        "u": _dev(np.asarray(u0, np.float32).copy(), np.float32),
        "i": torch.zeros(n, dtype=torch.float32, device="cuda"),
        "r": torch.zeros(n, dtype=torch.int32, device="cuda"),
        "ring": torch.zeros(64 * n, dtype=torch.int32, device="cuda"),
        "rs": torch.zeros(cap, dtype=torch.int32, device="cuda"),
        "ri": torch.zeros(cap, dtype=torch.int32, device="cuda"),
        "rn": torch.zeros(1, dtype=torch.int32, device="cuda"),
        "cnt": torch.zeros(2, dtype=torch.int64, device="cuda"),
        "status": torch.zeros(1, dtype=torch.int32, device="cuda"),
    }
    io = pkg.SnnNoallocIO(
        row_ptr=bufs["rp"].data_ptr(), words=bufs["words"].data_ptr(),
        wtab=bufs["wtab"].data_ptr(), u=bufs["u"].data_ptr(), i_syn=bufs["i"].data_ptr(),
        refr=bufs["r"].data_ptr(), ring=bufs["ring"].data_ptr(), ras_step=bufs["rs"].data_ptr(),
        ras_id=bufs["ri"].data_ptr(), ras_n=bufs["rn"].data_ptr(), ras_cap=cap,
        counters=bufs["cnt"].data_ptr(), status=bufs["status"].data_ptr())
    return bufs, io


@pytest.mark.parametrize("scale,mode", [(0.1, "dc"), (1.6, "poisson")])
def test_noalloc_matches_oracle(scale, mode):
    """Against the CPU oracle directly, on two calls in a row: the DC-input
    variant at 10 % scale, and a network of 123,470 neurons, just under the
    entry point's limit, whose spike lists fill most of the static scratch."""
    import os

    import oracle
    cfg = workload.microcircuit(scale, input_mode=mode)
    n = int(sum(cfg["pop_sizes"]))
    assert n <= pkg.NOALLOC_MAX_NEURONS
    onet = oracle.Network(cfg, n_threads=os.cpu_count())
    rp, tg, dl, wc = onet.export()
    words = pkg.encode_words(tg, dl, wc)
    u0 = workload.random_membrane(cfg, seed=77)
    stream = torch.cuda.current_stream()
    bufs, io = _noalloc_buffers(cfg, rp.astype(np.uint64), words, oracle.tables(cfg)["wtab"],
                                u0, 1 << 22)
    sim = oracle.Simulation(onet, u0=u0)
    t0 = 0
    for steps in (120, 180):
        pkg.step_noalloc(cfg, cfg["seed"], io, t0, steps, stream)
        torch.cuda.synchronize()
        sim.run(steps)
        assert int(bufs["status"].item()) == 0
        nrec = int(bufs["rn"].item())
        st = bufs["rs"][:nrec].cpu().numpy().astype(np.int64)
        ids = bufs["ri"][:nrec].cpu().numpy().astype(np.int64)
        order = np.lexsort((ids, st))
        o_st, o_id = sim.raster()
        assert o_st.size > 50
        np.testing.assert_array_equal(st[order], o_st)
        np.testing.assert_array_equal(ids[order], o_id)
        bufs["rn"].zero_()
        o_u, o_i, o_r, o_ring = sim.state()
        np.testing.assert_array_equal(bufs["u"].cpu().numpy().view(np.uint32), o_u.view(np.uint32))
        np.testing.assert_array_equal(bufs["i"].cpu().numpy().view(np.uint32), o_i.view(np.uint32))
        np.testing.assert_array_equal(bufs["r"].cpu().numpy(), o_r)
        np.testing.assert_array_equal(bufs["ring"].cpu().numpy().reshape(64, n),
                                      o_ring.astype(np.int32))
        oc = sim.counters()
        assert int(bufs["cnt"][0].item()) == oc["spikes"]
        assert int(bufs["cnt"][1].item()) == oc["events"]
        t0 += steps


def test_noalloc_rejects_networks_above_its_limit():
    cfg = workload.microcircuit(2.0)           # 154,338 neurons
    assert sum(cfg["pop_sizes"]) > pkg.NOALLOC_MAX_NEURONS
    with pytest.raises(pkg.SnnError) as e:
        pkg.step_noalloc(cfg, 1, pkg.SnnNoallocIO(), 0, 1)
    assert e.value.code == pkg.SNN_ERR_INVALID
    assert "131072" in str(e.value)
