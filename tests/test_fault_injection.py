"""Host-side fault injection and the serving engine's refusal paths, on the CPU (no GPU is
touched: every failure is made on the host, where the real one would be detected).

Covered: an injected device allocation failure in qmpm_init (QMPM_ERR_OOM, while without the
injection a host with no device reports QMPM_ERR_CUDA), corrupted requests refused at
submission (bad scene, bad scheme, non-finite state), a full request queue
(QMPM_ERR_QUEUE_FULL), an injected host allocation failure of a request, admission of a request
larger than the budget (QMPM_ERR_OOM on the request, found by admission before any device
work), and the bounded wait expiring (QMPM_ERR_TIMEOUT), genuinely and by injection."""
import numpy as np
import pytest
import torch

HAVE_GPU = torch.cuda.is_available()


@pytest.fixture(scope="module")
def q():
    from paper_2207_04658_b300 import build, qmpm
    build.build()
    qmpm.lib()
    qmpm.qmpm_fault_clear()
    yield qmpm
    qmpm.qmpm_fault_clear()


@pytest.fixture
def tiny():
    from paper_2207_04658_b300 import scenes
    sc, s0 = scenes.block2d_scene(n_strata=(8, 4))
    return sc, s0, scenes.block2d_scheme()


def code_of(fn):
    from paper_2207_04658_b300 import qmpm
    with pytest.raises(qmpm.QmpmError) as ei:
        fn()
    return ei.value.code


def test_fault_inject_arguments(q):
    assert code_of(lambda: q.qmpm_fault_inject(99)) == q.ERR_INVALID_ARG
    assert code_of(lambda: q.qmpm_fault_inject(q.FAULT_WAIT, -1, 1)) == q.ERR_INVALID_ARG
    q.qmpm_fault_inject(q.FAULT_WAIT, 0, 0)  # count 0 disarms
    assert q.qmpm_fault_hits(q.FAULT_WAIT) == 0


@pytest.mark.skipif(HAVE_GPU, reason="checks the failure on a host without a GPU")
def test_device_allocation_failure_is_reported_as_oom(q, tiny):
    sc, s0, sch = tiny
    q.qmpm_fault_clear()
    # without a device the first allocation fails with a CUDA error ...
    assert code_of(lambda: q.Scene(sc, sch, s0)) == q.ERR_CUDA
    # ... and an injected allocation failure is reported as what it is
    q.qmpm_fault_inject(q.FAULT_DEVICE_ALLOC, 0, 1)
    assert code_of(lambda: q.Scene(sc, sch, s0)) == q.ERR_OOM
    assert q.qmpm_fault_hits(q.FAULT_DEVICE_ALLOC) == 1
    # the fault was used up: the next call fails as before, for its own reason
    assert code_of(lambda: q.Scene(sc, sch, s0)) == q.ERR_CUDA
    q.qmpm_fault_clear()


def test_corrupted_requests_are_refused_at_submission(q, tiny):
    sc, s0, sch = tiny
    e = q.Engine(budget_bytes=2 ** 30)
    try:
        bad = s0.copy()
        bad[3, 1] = np.nan
        assert code_of(lambda: e.submit(sc, sch, bad, 10)) == q.ERR_INVALID_ARG
        bad[3, 1] = np.inf
        assert code_of(lambda: e.submit(sc, sch, bad, 10)) == q.ERR_INVALID_ARG
        assert code_of(lambda: e.submit(dict(sc, dt=-1e-4), sch, s0, 10)) == q.ERR_INVALID_ARG
        assert code_of(lambda: e.submit(dict(sc, grid_log2=14), sch, s0, 10)) == q.ERR_INVALID_ARG
        assert code_of(lambda: e.submit(sc, sch, s0, -1)) == q.ERR_INVALID_ARG
        wide = {k: dict(v) for k, v in sch.items()}
        wide["v"]["bits"] = 30  # wider than the FP32 compute limit
        assert code_of(lambda: e.submit(sc, wide, s0, 10)) == q.ERR_SCHEME
        assert e.stats()["queued"] == 0
        e.submit(sc, sch, s0, 10)  # a sound request is queued
        assert e.stats()["queued"] == 1
    finally:
        e.close()


def test_queue_overflow_and_host_allocation_failure(q, tiny):
    sc, s0, sch = tiny
    e = q.Engine(budget_bytes=2 ** 30, max_queued=3)
    try:
        for _ in range(3):
            e.submit(sc, sch, s0, 10)
        assert code_of(lambda: e.submit(sc, sch, s0, 10)) == q.ERR_QUEUE_FULL
        assert e.stats()["queued"] == 3
    finally:
        e.close()
    e = q.Engine(budget_bytes=2 ** 30)
    try:
        q.qmpm_fault_inject(q.FAULT_HOST_ALLOC, 1, 1)  # the second request's allocation fails
        e.submit(sc, sch, s0, 10)
        assert code_of(lambda: e.submit(sc, sch, s0, 10)) == q.ERR_OOM
        e.submit(sc, sch, s0, 10)
        assert e.stats()["queued"] == 2
        assert q.qmpm_fault_hits(q.FAULT_HOST_ALLOC) == 1
    finally:
        q.qmpm_fault_clear()
        e.close()


def test_bounded_wait_expires(q, tiny):
    sc, s0, sch = tiny
    e = q.Engine(budget_bytes=2 ** 30)
    try:
        assert e.wait(0.0) is False  # idle engine: returns at once
        q.qmpm_fault_inject(q.FAULT_WAIT, 0, 1)
        assert code_of(lambda: e.wait(10.0)) == q.ERR_TIMEOUT  # injected: expires at once
        e.submit(sc, sch, s0, 10)
        # nothing runs the queue (no loop thread), so the deadline passes with work left
        assert code_of(lambda: e.wait(0.05)) == q.ERR_TIMEOUT
        assert code_of(lambda: e.wait(-1.0)) == q.ERR_INVALID_ARG
    finally:
        q.qmpm_fault_clear()
        e.close()


@pytest.mark.skipif(HAVE_GPU, reason="checks the failure on a host without a GPU")
def test_admission_refuses_a_request_above_the_budget(q, tiny):
    sc, s0, sch = tiny
    e = q.Engine(budget_bytes=4096)  # far below any scene's footprint
    try:
        rid = e.submit(sc, sch, s0, 10)
        # admission runs before the engine's device setup, which then fails on this host
        assert code_of(lambda: e.run(1)) == q.ERR_CUDA
        done = e.poll()
        assert [r["id"] for r in done] == [rid]
        assert done[0]["status"] == 3 and done[0]["error"] == q.ERR_OOM  # QMPM_REQ_FAILED
        assert e.wait(0.0) is False  # nothing left
    finally:
        e.close()
