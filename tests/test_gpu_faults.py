"""Failure handling of the stream API and the server, with every failure made on the host
(no fault, trap or hang on the GPU): a simulated device allocation failure during admission
(test hook CYC_TEST_FAIL_ALLOC=k fails the k-th allocation of one cyc_create_* or
cyc_server_open call), chunk descriptors that are corrupt or that the feeder drops, and a
feeder thread that stops while its backlog is still being processed."""
import threading

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

LAGS = np.arange(0, 40, 3)
ALPHAS = -0.5 + np.arange(300) / 300.0


def free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_stream_admission_failure_leaves_nothing_behind(cyc, monkeypatch):
    """Every device allocation of cyc_create_ex in turn fails: the call returns CYC_ENOMEM,
    hands out no handle and frees what it had allocated; repeated failures leak no device
    memory; once no allocation fails, the stream works."""
    failed = 0
    for k in range(1, 64):
        monkeypatch.setenv("CYC_TEST_FAIL_ALLOC", str(k))
        try:
            s = cyc.Stream(LAGS, ALPHAS, cyc.CYC_BOTH, precision="bf16x3")
        except cyc.CycError as e:
            assert e.code == cyc.CYC_ENOMEM, k
            failed += 1
            continue
        monkeypatch.delenv("CYC_TEST_FAIL_ALLOC")
        break
    else:
        pytest.fail("every allocation index failed")
    assert failed >= 10                      # staging, sums, tables, partials, read buffer, status
    x = synth.white(9001, seed=401).astype(np.complex64)
    with s:
        s.push(x)
        R, n = s.read()
    Ro, no = oracle.estimate(x, LAGS, ALPHAS)
    assert n == no and np.max(np.abs(R - Ro)) / oracle.r00(x, int(LAGS.max())) < 1e-4
    # and nothing stayed allocated by the failed attempts
    monkeypatch.setenv("CYC_TEST_FAIL_ALLOC", "3")
    base = free_bytes()
    for _ in range(20):
        with pytest.raises(cyc.CycError):
            cyc.Stream(LAGS, ALPHAS, cyc.CYC_BOTH, precision="bf16x3")
    assert base - free_bytes() < (4 << 20)


def test_server_admission_failure_leaves_the_slot_and_budget(cyc, monkeypatch):
    """A server stream whose admission fails on a device allocation reports CYC_EAGAIN (try
    again later), keeps the memory budget's account and the slot unchanged, and the server
    keeps serving: afterwards every slot can be opened."""
    with cyc.Server(max_streams=4, precision="bf16x3", ring_samples=1 << 16) as srv:
        held0 = srv.stats()[3]
        for k in range(1, 8):
            monkeypatch.setenv("CYC_TEST_FAIL_ALLOC", str(k))
            with pytest.raises(cyc.CycError) as e:
                srv.open(LAGS, ALPHAS, cyc.CYC_BOTH)
            assert e.value.code == cyc.CYC_EAGAIN, k
            assert srv.stats()[3] == held0
        monkeypatch.delenv("CYC_TEST_FAIL_ALLOC")
        sids = [srv.open(LAGS, ALPHAS, cyc.CYC_BOTH) for _ in range(4)]
        assert sorted(sids) == [0, 1, 2, 3]
        x = synth.white(20000, seed=402).astype(np.complex64)
        srv.submit(sids[2], x)
        srv.drain(60)
        R, n = srv.read(sids[2])
        Ro, no = oracle.estimate(x, LAGS, ALPHAS)
        assert n == no and np.max(np.abs(R - Ro)) / oracle.r00(x, int(LAGS.max())) < 1e-4


def test_corrupt_descriptors_are_rejected_and_a_dropped_chunk_only_shortens_its_stream(cyc):
    """Corrupt chunk descriptors (NULL data, negative or oversized lengths, unknown or closed
    stream ids) fail with CYC_EINVAL and queue nothing.  A chunk that the feeder drops leaves
    its stream with the estimate of the chunks it did receive -- N_eff tells the client that
    samples are missing -- and the other streams untouched."""
    M = int(LAGS.max())
    xs = [synth.white(30011, seed=410 + i).astype(np.complex64) for i in range(3)]
    cuts = [0, 7001, 15007, 22013, 30011]
    with cyc.Server(max_streams=4, precision="bf16x3", ring_samples=1 << 16) as srv:
        sids = [srv.open(LAGS, ALPHAS, cyc.CYC_BOTH) for _ in range(3)]
        closed = srv.open(LAGS, ALPHAS, cyc.CYC_BOTH)
        srv.close_stream(closed)
        b0 = srv.stats()
        for args in ((sids[0], 0, 100), (sids[0], xs[0], -1), (sids[0], xs[0][:10], 1 << 20), (999, xs[0], 10),
                     (-1, xs[0], 10), (closed, xs[0], 10)):
            with pytest.raises(cyc.CycError) as e:
                srv.submit(*args)
            assert e.value.code == cyc.CYC_EINVAL
        assert srv.stats()[:2] == b0[:2]
        kept = []
        for j in range(4):
            for i, sid in enumerate(sids):
                if i == 1 and j == 2:
                    continue                                      # the feeder drops this chunk
                srv.submit(sid, np.ascontiguousarray(xs[i][cuts[j]:cuts[j + 1]]))
                if i == 1:
                    kept.append(xs[i][cuts[j]:cuts[j + 1]])
        srv.drain(60)
        for i, sid in enumerate(sids):
            R, n = srv.read(sid)
            x = np.concatenate(kept) if i == 1 else xs[i]
            assert n == x.size - M, i
            Ro, _ = oracle.estimate(x, LAGS, ALPHAS)
            assert np.max(np.abs(R - Ro)) / oracle.r00(x, M) < 1e-4, i


def test_a_feeder_that_stops_leaves_a_drainable_backlog(cyc):
    """A feeder thread queues a backlog and stops.  A drain with a timeout shorter than the
    backlog returns CYC_ETIMEDOUT without disturbing anything; a longer one returns once
    everything submitted is in the sums, and the estimate is that of what was submitted."""
    import torch
    M = int(LAGS.max())
    T, C = 1 << 22, 1 << 18
    xs = [synth.white(T, seed=420 + i).astype(np.complex64) for i in range(4)]
    pinned = [torch.from_numpy(x.view(np.float32)).pin_memory() for x in xs]
    with cyc.Server(max_streams=4, precision="bf16x3", ring_samples=1 << 23) as srv:
        sids = [srv.open(LAGS, ALPHAS, cyc.CYC_BOTH) for _ in range(4)]

        def feeder():
            for c in range(0, T, C):
                for i, sid in enumerate(sids):
                    srv.submit(sid, pinned[i].data_ptr() + 8 * c, C)
            # and then the feeder stops

        th = threading.Thread(target=feeder)
        th.start()
        th.join()
        with pytest.raises(cyc.CycError) as e:
            srv.drain(1e-4)
        assert e.value.code == cyc.CYC_ETIMEDOUT
        srv.drain(120)
        R, n = srv.read(sids[3])
    assert n == T - M
    Ro, _ = oracle.estimate(xs[3], LAGS, ALPHAS[:40])
    assert np.max(np.abs(R[:, :40] - Ro)) / oracle.r00(xs[3], M) < 1e-4
