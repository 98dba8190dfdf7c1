"""lll_simulate_noalloc: the entry point for callers that cannot allocate
device memory while running (pool-managed services, latency-bound callers).

It must give the same payoff sums as lll_simulate / lll_get_sums through the
C ABI, call after call (its static scratch keeps the previous call's
contents), and refuse a launch whose scratch would exceed its static maximum.
This file is collected last so that a failure here stops a -x run only after
every other test has run.
"""
import numpy as np
import pytest

from paper_1006_3340_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1006_3340_gb300 import lll

    lll.load()
    return torch, lll


@pytest.mark.parametrize("maker,scheme,paths,launch", [
    (workloads.large_single, "picard", 1 << 16, None),
    (workloads.large_single, "full", 50000, None),
    (workloads.small_plain, "frozen", 20000, None),
    # the other scratch layouts: two paths per thread, and lane groups of four
    (workloads.large_single, "full", 30001, (128, 0, 0, 2, 1)),
    (workloads.large_single, "picard", 30001, (128, 0, 0, 1, 4))])
def test_noalloc_matches_simulate_on_consecutive_calls(env, maker, scheme, paths, launch):
    torch, lll = env
    wl = maker(paths=paths)
    sim = lll.LevyLibor(wl)
    try:
        n, ns = wl.n, wl.strikes.shape[1]
        if launch is not None:
            sim.set_launch(*launch)
        sim.simulate(scheme)
        s1, s2, cnt = sim.sums()
        ref_price = s1 / cnt
        out = torch.empty((n, ns, 2), dtype=torch.float64, device="cuda")
        for call in range(2):
            out.fill_(float("nan"))
            torch.cuda.synchronize()
            lll.lll_simulate_noalloc(sim.ctx, lll.SCHEMES[scheme], 0, wl.paths, wl.seed, out.data_ptr())
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got)), call
            assert np.allclose(got[..., 0], s1, rtol=1e-12, atol=0), call
            assert np.allclose(got[..., 1], s2, rtol=1e-12, atol=0), call
            assert np.abs(got[..., 0] / cnt - ref_price).max() <= 1e-7, call
    finally:
        sim.close()


def test_noalloc_rejects_launch_beyond_static_scratch(env):
    torch, lll = env
    # 119 rates, 256-thread blocks: one block per SM needs SMs x 2 x 119 x 256
    # x 4 B of Picard state (37 MB on 152 SMs), above the 32 MiB maximum; the
    # premise is checked against this GPU's SM count.
    wl = workloads.long_dated(paths=1 << 20)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    if sms * 2 * wl.n * 256 * 4 <= 32 << 20:
        pytest.skip(f"{sms} SMs: one block per SM fits the static scratch")
    sim = lll.LevyLibor(wl)
    try:
        sim.set_launch(256)
        out = torch.empty((wl.n, wl.strikes.shape[1], 2), dtype=torch.float64, device="cuda")
        with pytest.raises(lll.LLLError) as e:
            lll.lll_simulate_noalloc(sim.ctx, lll.LLL_PICARD, 0, wl.paths, wl.seed, out.data_ptr())
        assert e.value.code == lll.LLL_EUNSUPPORTED
        assert "static maximum" in str(e.value)
    finally:
        sim.close()
