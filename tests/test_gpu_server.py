"""The continuous-batching server (GPU): every stream's result in the mix equals the same
stream run alone, admission by memory budget, ring back-pressure, completion records.
"""
import threading

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def alone(cyc, x, lags, alphas, forms, n0, precision):
    with cyc.Stream(lags, alphas, forms, precision=precision, n0=n0) as s:
        s.push(np.ascontiguousarray(x))
        return s.read()


def stream_case(i):
    rng = np.random.default_rng(1000 + i)
    L = int(rng.integers(1, 40)) if i != 11 else 100       # stream 11: wide (two-form) columns
    lags = np.sort(rng.choice(np.arange(0, 3 * L + 1), size=L, replace=False))
    A = int(rng.integers(1, 300))
    alphas = rng.uniform(-0.5, 0.5, A)
    forms = int(rng.integers(1, 4))
    n0 = int(rng.integers(0, 1 << 40)) if i % 3 == 0 else 0
    T = int(rng.integers(2000, 60000))
    x = synth.white(T, seed=2000 + i).astype(np.complex64)
    cuts = np.sort(rng.choice(np.arange(1, T), size=int(rng.integers(1, 12)), replace=False))
    chunks = np.diff(np.concatenate([[0], cuts, [T]]))
    return dict(lags=lags, alphas=alphas, forms=forms, n0=n0, x=x, chunks=chunks)


@pytest.mark.parametrize("precision,tol", [("bf16x3", 1e-4), ("fp16", 1e-2)])
def test_mix_equals_alone(cyc, precision, tol):
    """Twelve streams of different lags, cycle frequencies, forms, start indices and chunkings
    in one server: each stream's result equals the same stream run alone through cyc_push,
    and the oracle's."""
    cases = [stream_case(i) for i in range(12)]
    with cyc.Server(max_streams=16, precision=precision, item_samples=4096) as srv:
        sids = [srv.open(c["lags"], c["alphas"], c["forms"], c["n0"]) for c in cases]
        pos = [0] * len(cases)
        k = [0] * len(cases)
        tag = 0
        # interleave the streams' chunks, as uneven arrivals would
        while any(k[i] < len(c["chunks"]) for i, c in enumerate(cases)):
            for i, c in enumerate(cases):
                if k[i] < len(c["chunks"]):
                    n = int(c["chunks"][k[i]])
                    srv.submit(sids[i], c["x"][pos[i]:pos[i] + n], tag=tag)
                    tag += 1
                    pos[i] += n
                    k[i] += 1
        srv.drain(120)
        done = srv.poll(100000)
        for i, c in enumerate(cases):
            R, n = srv.read(sids[i])
            Ra, na = alone(cyc, c["x"], c["lags"], c["alphas"], c["forms"], c["n0"], precision)
            M = int(c["lags"].max())
            assert n == na == c["x"].size - M
            r00 = oracle.r00(c["x"], M)
            assert np.max(np.abs(R - Ra)) / r00 < tol / 5, i
            if i < 3:
                Ro, _ = oracle.estimate(c["x"], c["lags"], c["alphas"], c["forms"], n0=c["n0"])
                assert np.max(np.abs(R - Ro)) / r00 < tol, i
        batches, items, busy, held = srv.stats()
        assert batches >= 1 and items >= 12 and busy > 0 and held > 0
    # every chunk that could finish was reported once, with its tag and times in order
    tags = sorted(d[2] for d in done)
    assert len(tags) == len(set(tags))
    assert all(d[1] == 0 and d[5] >= d[4] for d in done)
    assert len(done) >= tag - 12


def test_admission_by_memory_and_slots(cyc):
    lags, alphas = np.arange(64), -0.5 + np.arange(512) / 512.0
    ring = 1 << 20
    per = ring * 8 + 512 * 128 * 16           # ring + sums, roughly one stream
    with cyc.Server(max_streams=8, precision="bf16x3", ring_samples=ring, mem_budget=int(2.5 * per)) as srv:
        a = srv.open(lags, alphas)
        b = srv.open(lags, alphas)
        with pytest.raises(cyc.CycError) as e:
            srv.open(lags, alphas)
        assert e.value.code == cyc.CYC_EAGAIN
        srv.close_stream(a)
        c = srv.open(lags, alphas)          # the budget freed by the close admits it
        assert c == a
        srv.close_stream(b)
        srv.close_stream(c)
    with cyc.Server(max_streams=2, precision="bf16x3", ring_samples=1 << 16) as srv:
        srv.open([0, 1], [0.1])
        srv.open([0, 1], [0.1])
        with pytest.raises(cyc.CycError) as e:
            srv.open([0, 1], [0.1])
        assert e.value.code == cyc.CYC_EAGAIN


def test_ring_backpressure_and_concurrent_submitters(cyc):
    ring = 1 << 15
    lags, alphas = np.arange(0, 32, 3), np.linspace(-0.5, 0.5, 100, endpoint=False)
    xs = [synth.white(200000 + 777 * i, seed=3000 + i).astype(np.complex64) for i in range(4)]
    with cyc.Server(max_streams=4, precision="bf16x3", ring_samples=ring, item_samples=8192) as srv:
        sids = [srv.open(lags, alphas) for _ in xs]
        eagain = [0] * 4

        def feed(i):
            x, pos, step = xs[i], 0, 5000 + 1000 * i
            while pos < x.size:
                n = min(step, x.size - pos)
                try:
                    srv.submit(sids[i], x[pos:pos + n])
                    pos += n
                except cyc.CycError as e:
                    assert e.code == cyc.CYC_EAGAIN
                    eagain[i] += 1
                    threading.Event().wait(0.0005)

        th = [threading.Thread(target=feed, args=(i,)) for i in range(4)]
        for t in th:
            t.start()
        for t in th:
            t.join(120)
        srv.drain(120)
        for i, x in enumerate(xs):
            R, n = srv.read(sids[i])
            Ra, na = alone(cyc, x, lags, alphas, 3, 0, "bf16x3")
            assert n == na
            assert np.max(np.abs(R - Ra)) / oracle.r00(x, 30) < 2e-5
        with pytest.raises(cyc.CycError) as e:
            srv.submit(sids[0], np.zeros(ring, np.complex64))
        assert e.value.code == cyc.CYC_EINVAL
    assert sum(eagain) > 0          # the small ring really pushed back


@pytest.mark.parametrize("precision,tol", [("bf16x3", 1e-4), ("fp16", 1e-2)])
def test_streams_sharing_a_configuration(cyc, precision, tol):
    """Nine streams with the same symmetric cycle-frequency grid (pairs a, -a and the real
    unit), lags and forms (64 lags x 2 forms: one column tile) and different start indices
    and chunkings: each stream's result equals the same stream run alone, and the oracle's."""
    lags = np.arange(64)
    alphas = -0.5 + np.arange(300) / 300.0
    rng = np.random.default_rng(77)
    cases = []
    for i in range(9):
        T = int(rng.integers(20000, 90000))
        x = synth.white(T, seed=3000 + i).astype(np.complex64)
        cuts = np.sort(rng.choice(np.arange(1, T), size=int(rng.integers(1, 8)), replace=False))
        n0 = int(rng.integers(0, 1 << 40)) if i % 2 else 0
        cases.append(dict(x=x, chunks=np.diff(np.concatenate([[0], cuts, [T]])), n0=n0))
    with cyc.Server(max_streams=16, precision=precision, item_samples=8192) as srv:
        sids = [srv.open(lags, alphas, 3, c["n0"]) for c in cases]
        pos, k = [0] * 9, [0] * 9
        while any(k[i] < len(c["chunks"]) for i, c in enumerate(cases)):
            for i, c in enumerate(cases):
                if k[i] < len(c["chunks"]):
                    n = int(c["chunks"][k[i]])
                    srv.submit(sids[i], c["x"][pos[i]:pos[i] + n])
                    pos[i] += n
                    k[i] += 1
        srv.drain(120)
        for i, c in enumerate(cases):
            R, n = srv.read(sids[i])
            Ra, na = alone(cyc, c["x"], lags, alphas, 3, c["n0"], precision)
            assert n == na
            r00 = oracle.r00(c["x"], 63)
            assert np.max(np.abs(R - Ra)) / r00 < tol / 5, i
            if i < 2:
                Ro, _ = oracle.estimate(c["x"], lags, alphas, 3, n0=c["n0"])
                assert np.max(np.abs(R - Ro)) / r00 < tol, i
