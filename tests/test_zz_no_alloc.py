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


def test_noalloc_rejects_networks_above_its_limit():
    cfg = workload.microcircuit(2.0)           # 154,338 neurons
    assert sum(cfg["pop_sizes"]) > pkg.NOALLOC_MAX_NEURONS
    with pytest.raises(pkg.SnnError) as e:
        pkg.step_noalloc(cfg, 1, pkg.SnnNoallocIO(), 0, 1)
    assert e.value.code == pkg.SNN_ERR_INVALID
    assert "131072" in str(e.value)
