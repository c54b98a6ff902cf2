"""Serving loop: scheduling logic on the library's fake device (CPU) and, on a GPU, identity
of every result alone and in a concurrent mix."""

import time

import numpy as np
import pytest

from paper_2509_03623_b300 import synth


@pytest.fixture(scope="module")
def serve():
    from paper_2509_03623_b300 import build, serve as sv
    build.build()
    return sv


def small(seed=0, **kw):
    return synth.config_small(seed).replace(**kw)


CUBE = 16 * 64 * 64 * 4  # bytes of a small render's cube


def test_admission_by_memory_fifo(serve):
    with serve.Server(mem_budget_bytes=int(2.5 * CUBE), max_inflight=8, fake=True) as s:
        ts = [s.submit_render(small(i), None, cube=16, fake_us=150_000) for i in range(5)]
        time.sleep(0.05)
        st = s.stats()
        assert st["running"] == 2 and st["queued"] == 3 and st["bytes_in_use"] == 2 * CUBE
        lats = [s.wait(t, 5000)[1] for t in ts]
        assert [s.poll(t)[0] for t in ts] == ["done"] * 5
        # FIFO pairs: (0,1) then (2,3) then 4
        assert lats[0] < 250 and lats[2] > 250 and lats[4] > 400
        assert lats[4] >= lats[2] >= lats[0]
        assert s.stats()["completed"] == 5 and s.stats()["bytes_in_use"] == 0


def test_inflight_limit_serializes(serve):
    with serve.Server(mem_budget_bytes=1 << 30, max_inflight=1, fake=True) as s:
        ts = [s.submit_render(small(i), None, cube=16, fake_us=40_000) for i in range(4)]
        lats = [s.wait(t, 5000)[1] for t in ts]
        assert all(b - a > 30 for a, b in zip(lats, lats[1:]))


def test_malformed_and_over_budget_rejected(serve):
    from paper_2509_03623_b300 import _rt
    with serve.Server(mem_budget_bytes=CUBE // 2, max_inflight=2, fake=True) as s:
        with pytest.raises(_rt.RTError) as e:
            s.submit_render(small(0, n_samples=0), None, cube=16)
        assert e.value.code == _rt.RT_EINVAL
        with pytest.raises(_rt.RTError) as e:
            s.submit_render(small(0), None, cube=None)      # render without output
        assert e.value.code == _rt.RT_EINVAL
        with pytest.raises(_rt.RTError) as e:
            s.submit_render(small(0), None, cube=16)        # needs more than the whole budget
        assert e.value.code == _rt.RT_ENOMEM
        grads = dict(T=16, n_h2=16, vturb=16, h_lo=16, h_hi=16, loss=None)
        with pytest.raises(_rt.RTError) as e:                # both seeds given
            s.submit_adjoint(small(0, nx=4, ny=4), None, grads, dL_dcube=16, target=16)
        assert e.value.code == _rt.RT_EINVAL
        assert s.stats()["queued"] == 0


def test_bounded_wait_and_cancel(serve):
    from paper_2509_03623_b300 import _rt
    with serve.Server(mem_budget_bytes=1 << 30, max_inflight=1, fake=True) as s:
        a = s.submit_render(small(0), None, cube=16, fake_us=300_000)
        b = s.submit_render(small(1), None, cube=16, fake_us=10_000)
        time.sleep(0.02)
        t0 = time.perf_counter()
        with pytest.raises(TimeoutError):
            s.wait(a, 10.0)
        assert time.perf_counter() - t0 < 0.2
        with pytest.raises(_rt.RTError) as e:
            s.cancel(a)                                     # running: cannot cancel
        assert e.value.code == _rt.RT_EBUSY
        s.cancel(b)
        assert s.poll(b)[0] == "cancelled"
        assert s.wait(a, 5000)[0] == "done"
        with pytest.raises(_rt.RTError) as e:
            s.poll(12345)
        assert e.value.code == _rt.RT_ENOTFOUND


def test_queue_full_and_destroy_with_pending(serve):
    from paper_2509_03623_b300 import _rt
    s = serve.Server(mem_budget_bytes=1 << 30, max_inflight=1, max_queue=2, fake=True)
    s.submit_render(small(0), None, cube=16, fake_us=200_000)
    time.sleep(0.02)
    s.submit_render(small(1), None, cube=16, fake_us=1000)
    s.submit_render(small(2), None, cube=16, fake_us=1000)
    with pytest.raises(_rt.RTError) as e:
        s.submit_render(small(3), None, cube=16, fake_us=1000)
    assert e.value.code == _rt.RT_EBUSY
    t0 = time.perf_counter()
    s.close()                                               # cancels 2 queued, waits for 1
    assert time.perf_counter() - t0 < 2.0


@pytest.mark.gpu
def test_results_identical_alone_and_in_mix(serve, orc):
    """Renders of differently sized disks submitted together (overlapping on the device)
    equal the same requests run alone bit for bit; gradients agree to the rounding of the
    adjoint's FP32 per-block partial sums (their order on the device is not fixed): 1e-6 of
    the largest entry."""
    import torch
    from paper_2509_03623_b300 import _rt
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(0)
    reqs = []
    for i in range(10):
        px = int(rng.choice([32, 48, 64]))
        p = synth.config_small(40 + i).replace(nx=px, ny=px, v_kms=np.linspace(-4, 4, int(
            rng.choice([16, 32, 64]))), n_samples=int(rng.choice([64, 128, 200])))
        reqs.append((p, i % 3 == 0))
    alone = []
    for p, adj in reqs:
        dd = _rt.DeviceDisk(p)
        if adj:
            tgt = (_rt.rt_render(p, dd) * 1.1).contiguous()
            cube, g = _rt.rt_render_adjoint(p, dd, target=tgt)
            alone.append((dd, tgt, cube.cpu().numpy(), {k: v.cpu().numpy() for k, v in g.items()}))
        else:
            alone.append((dd, None, _rt.rt_render(p, dd).cpu().numpy(), None))
    torch.cuda.synchronize()
    outs = []
    with serve.Server(mem_budget_bytes=1 << 30, max_inflight=4) as s:
        tickets = []
        for (p, adj), (dd, tgt, _, _) in zip(reqs, alone):
            cube = torch.full((p.nch, p.ny, p.nx), float("nan"), device="cuda")
            if adj:
                g = {k: torch.empty_like(v) for k, v in zip(
                    ("T", "n_h2", "vturb", "h_lo", "h_hi"),
                    [t.double() for t in dd.tensors()])}
                g["loss"] = torch.empty(1, dtype=torch.float64, device="cuda")
                tickets.append(s.submit_adjoint(p, dd, g, target=tgt, cube=cube))
                outs.append((cube, g))
            else:
                tickets.append(s.submit_render(p, dd, cube))
                outs.append((cube, None))
        for t in tickets:
            state, lat = s.wait(t, 60000)
            assert state == "done", s.error(t)
            assert lat > 0
        # every request went through the server (whether any was seen running depends on how
        # fast these small renders finish relative to the sampling, so it is not asserted)
        assert s.stats()["completed"] >= len(tickets)
    for (cube, g), (_, _, ref_cube, ref_g) in zip(outs, alone):
        assert np.array_equal(cube.cpu().numpy(), ref_cube)
        if g is not None:
            for k in ("T", "n_h2", "vturb", "h_lo", "h_hi"):
                a, b = g[k].cpu().numpy(), ref_g[k]
                assert np.abs(a - b).max() <= 1e-6 * np.abs(b).max(), k
            assert float(g["loss"].item()) == pytest.approx(float(ref_g["loss"][0]), rel=1e-12)


@pytest.mark.gpu
def test_requests_overlap_on_device(serve):
    """Eight renders that each occupy a few dozen SMs (32x32 px, 64 channels, 2048 samples),
    submitted together, are in flight on the device at the same time: the intervals between
    the events the server records on each request's stream before and after its kernels
    intersect (at least two at one instant), and every cube equals the same render run alone."""
    import torch
    from paper_2509_03623_b300 import _rt
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    reqs = [synth.config_small(60 + i).replace(nx=32, ny=32, v_kms=np.linspace(-6, 6, 64),
                                               n_samples=2048) for i in range(8)]
    disks = [_rt.DeviceDisk(p) for p in reqs]
    alone = [_rt.rt_render(p, dd).cpu().numpy() for p, dd in zip(reqs, disks)]
    torch.cuda.synchronize()
    with serve.Server(mem_budget_bytes=1 << 30, max_inflight=8) as s:
        cubes = [torch.empty((p.nch, p.ny, p.nx), device="cuda") for p in reqs]
        tickets = [s.submit_render(p, dd, c) for p, dd, c in zip(reqs, disks, cubes)]
        for t in tickets:
            assert s.wait(t, 60000)[0] == "done", s.error(t)
        iv = [s.device_times(t) for t in tickets]
    assert all(b > a for a, b in iv)
    peak = serve.max_overlap(iv)
    print(f"device intervals (ms): {[(round(a, 3), round(b, 3)) for a, b in iv]}; "
          f"max in flight {peak}")
    assert peak >= 2
    for c, ref in zip(cubes, alone):
        assert np.array_equal(c.cpu().numpy(), ref)


def test_max_overlap_counts_intersections():
    from paper_2509_03623_b300.serve import max_overlap
    assert max_overlap([]) == 0
    assert max_overlap([(0, 1), (1, 2)]) == 1          # touching ends do not overlap
    assert max_overlap([(0, 3), (1, 2), (1.5, 4)]) == 3
    assert max_overlap([(0, 1), (2, 3), (2.5, 5), (4, 6)]) == 2
