"""GPU tests of the serving loop: each result is the same computed alone and in
a mix of concurrent uneven requests (bit for bit -- the emulated product is
deterministic per problem), admission binds under a small HBM budget without
exceeding it, requests that can never fit or are malformed are rejected, the
bounded wait reports a timeout, and the FP64 baseline mode matches mm_naive."""
import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def srv():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1106_1347_gb300 import build

    build.build()
    import paper_1106_1347_gb300 as mm
    from paper_1106_1347_gb300 import serving

    return mm, serving


def _case(i, n, p, m):
    import torch

    a = torch.from_numpy(S.loguniform(n, p, S.stream_seed(4, 1000 + 2 * i))).pin_memory()
    b = torch.from_numpy(S.loguniform(p, m, S.stream_seed(4, 1001 + 2 * i))).pin_memory()
    c = torch.full((n, m), float("nan"), dtype=torch.float64).pin_memory()
    return a, b, c


SHAPES = [(37, 65, 129), (200, 333, 150), (5, 700, 3), (128, 64, 64), (300, 41, 17), (64, 1000, 96), (1, 1, 1),
          (129, 513, 250), (90, 90, 90), (33, 2049, 40)]
TIERS = [1e-14, 1e-6, 1e-14, 1e-14, 1e-6, 1e-14, 1e-6, 1e-14, 1e-6, 1e-14]


def test_alone_and_in_the_mix_agree(srv):
    import torch

    mm, serving = srv
    cases = [_case(i, *sh) for i, sh in enumerate(SHAPES)]
    alone = []
    with serving.Server(1 << 30, max_batch=1, nstreams=1, use_graphs=False) as s1:
        for i, (a, b, c) in enumerate(cases):
            s1.submit(a, b, c, tier=TIERS[i], tag=i)
            assert s1.wait(120) == 0
            alone.append(c.numpy().copy())
        comps = s1.poll()
        assert all(x["status"] == 0 for x in comps)
    with serving.Server(1 << 30, max_batch=64, nstreams=3, use_graphs=True) as s2:
        for rep in range(3):  # repeated mixes exercise graph replays of cached buckets
            mixed = [_case(i, *sh) for i, sh in enumerate(SHAPES)]
            for i, (a, b, c) in enumerate(mixed):
                s2.submit(a, b, c, tier=TIERS[i], tag=100 * rep + i)
            assert s2.wait(120) == 0
            for i, (a, b, c) in enumerate(mixed):
                assert np.array_equal(c.numpy(), alone[i]), f"request {i}"
        st = s2.stats()
        assert st["completed"] == 30 and st["rejected"] == 0
        assert st["batches"] < 30  # requests were batched together
    # and both equal the library's single-call path with the tier's slice count
    for i, (a, b, c) in enumerate(cases):
        ref = mm.emulated(a.cuda(), b.cuda(), tier=TIERS[i]).cpu().numpy()
        assert np.array_equal(alone[i], ref)


def test_auto_format_uses_fp8_for_low_tiers(srv):
    """Method 2 serves the 1e-6 tier from FP8-E4M3 slices (6 of them cost 21
    pairs at twice the BF16 rate, against 15 BF16 pairs) and 1e-14 from 8 BF16
    slices; each result equals the single call with the reported format."""
    mm, serving = srv
    cases = [_case(200 + i, *sh) for i, sh in enumerate(SHAPES)]
    with serving.Server(1 << 30, max_batch=64, nstreams=2, use_graphs=True,
                        method=serving.METHOD_EMULATED_AUTO) as s:
        for i, (a, b, c) in enumerate(cases):
            s.submit(a, b, c, tier=TIERS[i], tag=i)
        assert s.wait(120) == 0
        comps = {x["tag"]: x for x in s.poll()}
    for i, (a, b, c) in enumerate(cases):
        comp = comps[i]
        assert comp["status"] == 0
        if TIERS[i] == 1e-6:
            assert (comp["kind"], comp["slices"]) == (mm.SLICE_FP8E4M3, 6)
        else:
            assert (comp["kind"], comp["slices"]) == (mm.SLICE_BF16, 8)
        ref = mm.emulated(a.cuda(), b.cuda(), nslices=comp["slices"], kind=comp["kind"]).cpu().numpy()
        assert np.array_equal(c.numpy(), ref), f"request {i}"


def test_budget_binds_and_is_respected(srv):
    mm, serving = srv
    budget = 48 << 20
    cases = [_case(50 + i, 256, 256, 256) for i in range(24)]
    with serving.Server(budget, max_batch=8, nstreams=2) as s:
        for i, (a, b, c) in enumerate(cases):
            s.submit(a, b, c, tier=1e-14, tag=i)
        assert s.wait(120) == 0
        st = s.stats()
        assert st["completed"] == 24
        assert st["peak_arena_bytes"] <= budget
        assert st["batches"] >= 3  # not everything fitted at once
    ref = mm.emulated(cases[0][0].cuda(), cases[0][1].cuda(), tier=1e-14).cpu().numpy()
    assert np.array_equal(cases[0][2].numpy(), ref)


def test_rejections_and_timeout(srv):
    import torch

    mm, serving = srv
    with serving.Server(16 << 20, max_batch=4, nstreams=1) as s:
        a, b, c = _case(90, 1024, 1024, 1024)  # 24 MiB of operands: can never fit
        s.submit(a, b, c, tier=1e-14, tag=1)
        assert s.wait(60) == 0
        comp = s.poll()
        assert comp and comp[0]["status"] == -3  # MM_ERR_NOMEM
        with pytest.raises(ValueError):
            s.submit(a[:, :10], b[:9], c[:, :5], tier=1e-14, tag=2)  # shapes checked in Python
        bad = serving.Request(4, 4, 4, a.data_ptr(), 2, b.data_ptr(), 1024, c.data_ptr(), 1024, 1e-14, 3)
        import ctypes

        assert s._L.mm_server_submit(s._h, ctypes.byref(bad)) == -1  # lda < P
    with serving.Server(1 << 30, max_batch=4, nstreams=1) as s:
        a, b, c = _case(91, 2048, 2048, 2048)
        s.submit(a, b, c, tier=1e-14, tag=7)
        assert s.wait(0) == -5  # MM_ERR_TIMEOUT: still running
        assert s.wait(120) == 0


def test_fp64_baseline_mode(srv):
    mm, serving = srv
    cases = [_case(120 + i, *sh) for i, sh in enumerate(SHAPES[:5])]
    with serving.Server(1 << 30, method=serving.METHOD_FP64) as s:
        for i, (a, b, c) in enumerate(cases):
            s.submit(a, b, c, tier=1e-14, tag=i)
        assert s.wait(120) == 0
    for a, b, c in cases:
        assert np.array_equal(c.numpy(), mm.naive(a.cuda(), b.cuda()).cpu().numpy())


def test_graph_replay_across_batch_sizes(srv):
    """Batches of 3 and then 4 requests of one shape have the same size bucket,
    so the second replays the first one's CUDA graph with a different problem
    count; results must still equal the single-call path."""
    mm, serving = srv
    with serving.Server(1 << 30, max_batch=16, nstreams=1, use_graphs=True) as s:
        for count, base in ((3, 200), (4, 210), (3, 220)):
            cases = [_case(base + i, 64, 64, 64) for i in range(count)]
            for i, (a, b, c) in enumerate(cases):
                s.submit(a, b, c, tier=1e-14, tag=base + i)
            assert s.wait(60) == 0, s.error()
            for a, b, c in cases:
                assert np.array_equal(c.numpy(), mm.emulated(a.cuda(), b.cuda(), tier=1e-14).cpu().numpy())
        assert s.stats()["graph_replays"] >= 1


def test_batches_on_different_streams_overlap_on_the_device(srv):
    """Each batch records a CUDA event before its first copy and after its last;
    the server's device intervals show batches on different streams running
    at the same time (their copies and products overlap), and none with one
    stream."""
    mm, serving = srv
    cases = [_case(200 + i, 1536, 1536, 1536) for i in range(4)]
    for nstreams in (1, 2):
        with serving.Server(2 << 30, max_batch=1, nstreams=nstreams, use_graphs=False) as s:
            for i, (a, b, c) in enumerate(cases):
                s.submit(a, b, c, tier=1e-14, tag=i)
            assert s.wait(120) == 0
            st = s.stats()
        assert st["completed"] == 4 and st["batches"] == 4
        assert st["device_busy_ms"] > 0
        if nstreams == 1:
            assert st["overlap_ms"] == 0.0
        else:
            assert st["overlap_ms"] > 0.2 * st["device_busy_ms"], st


@pytest.mark.parametrize("ratio", ["0.5", "4"])
def test_class_ratio_batches_correctly(srv, monkeypatch, ratio):
    """MM_SERVER_CLASS_RATIO limits a batch to requests within a factor of the
    oldest one's estimated time; a factor below 1 counts as 1, and the oldest
    request is always taken, so every request completes, bit for bit as the
    single-call path."""
    mm, serving = srv
    monkeypatch.setenv("MM_SERVER_CLASS_RATIO", ratio)
    cases = [_case(50 + i, *sh) for i, sh in enumerate(SHAPES)]
    with serving.Server(1 << 30, max_batch=64, nstreams=2, use_graphs=True) as s:
        for i, (a, b, c) in enumerate(cases):
            s.submit(a, b, c, tier=TIERS[i], tag=i)
        assert s.wait(120) == 0
        st = s.stats()
        assert st["completed"] == len(cases) and st["rejected"] == 0
    for i, (a, b, c) in enumerate(cases):
        assert np.array_equal(c.numpy(), mm.emulated(a.cuda(), b.cuda(), tier=TIERS[i]).cpu().numpy()), f"request {i}"
