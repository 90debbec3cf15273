"""The persistent batched launch (meta_plan_create_persistent): many registration
problems of uneven sizes, 2-D and 3-D, T and sigma, in ONE kernel launch whose CTAs
take tiles of every problem's recorded launches from one work counter.  Every problem
must get, bit for bit, what its own cost_and_grad gives (the same kernel bodies run on
the same tiles); the gradients must meet the FP64 oracle; a dependency wait that never
ends must be reported as a timeout, without a fault, and the plan must run normally
afterwards."""
import numpy as np
import pytest

import oracle
import phantoms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GRAD_RTOL = 1e-3
COST_RTOL = 1e-5


@pytest.fixture(scope="module")
def meta():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_08817_gb300 import _build
    _build.build()
    import paper_2106_08817_gb300 as m
    return m


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def smooth_p(seed, shape, scale, s=2.0):
    from scipy import ndimage
    r = np.random.default_rng(seed)
    out = np.empty(shape, np.float32)
    for b in range(shape[0]):
        out[b] = ndimage.gaussian_filter(r.normal(size=shape[1:]), s) * scale
    return out


# (dims, batch, T, sigma, ckpt, p0 scale): 2-D and 3-D, ragged extents, sigma from a
# 3-tap kernel to 7 (tap loops of 6 chunks, which the persistent kernel runs as its
# runtime loop), checkpoint strides, feet moving a voxel or more in some steps
MIX = [((40, 56), 2, 4, 2.3, 0, 30.0),
       ((64, 64), 1, 5, 3.0, 0, 40.0),
       ((12, 20, 28), 1, 3, 2.0, 0, 30.0),
       ((21, 45, 70), 2, 4, 2.0, 2, 30.0),
       ((33, 70), 1, 6, 1.0, 3, 20.0),
       ((50, 60), 1, 3, 7.0, 0, 60.0),
       ((9, 11, 13), 1, 2, 0.3, 0, 10.0),
       ((96, 40), 3, 3, 5.5, 0, 30.0),
       ((48, 52), 1, 3, 2.0, 0, 60.0),       # steps of up to 1.2-5 voxels: gather window R > 1
       ((14, 16, 18), 1, 3, 1.5, 0, 160.0)]  # up to 1.3-2.4 voxels


def make_problems(seed=900):
    probs = []
    for k, (dims, B, T, sigma, ckpt, scale) in enumerate(MIX):
        I0, _ = phantoms.random_fields(seed + 3 * k, B, dims)
        J, _ = phantoms.random_fields(seed + 3 * k + 1, B, dims)
        p0 = smooth_p(seed + 3 * k + 2, (B,) + dims, scale)
        mu = [0.1, 0.0, 0.2][:B] if B <= 3 else [0.1] * B
        probs.append(dict(I0=cuda(I0), J=cuda(J), p0=cuda(p0), T=T, sigma=sigma, mu=mu,
                          rho=[1.0, 1.3, 0.8][:B], lam=[1e-3, 1e-2, 1e-3][:B], ckpt=ckpt))
    return probs


def eager(meta, it):
    ws = meta.Workspace(it["dims"], it["B"], it["T"], it["sigma"], "cuda", it["ckpt"])
    return meta.cost_and_grad(it["I0"], it["J"], it["p0"], it["T"], it["sigma"], it["mu"],
                              it["rho"], it["lam"], workspace=ws, ckpt=it["ckpt"])


def test_persistent_plan_equals_the_separate_calls_bitwise(meta):
    plan = meta.GroupPlan(make_problems(), persistent=True)
    for rnd in range(2):  # two launches: the counters start over every launch
        plan.launch()
        torch.cuda.synchronize()
        assert plan.status() == 0
        for k, it in enumerate(plan.items):
            c, g = eager(meta, it)
            torch.cuda.synchronize()
            assert torch.isfinite(it["grad"]).all()
            assert torch.equal(it["cost"], c), (rnd, k)
            assert torch.equal(it["grad"], g), (rnd, k)
            assert it["ws"].status() & 1 == 0
        for it in plan.items:  # a gradient step in place; the next launch picks it up
            it["p0"].sub_(0.3 * it["grad"] / it["grad"].abs().max())


def test_persistent_plan_against_the_oracle(meta):
    plan = meta.GroupPlan(make_problems(seed=950), persistent=True)
    plan.launch()
    torch.cuda.synchronize()
    for k in (0, 2, 3, 5, 8, 9):
        it = plan.items[k]
        cost, grad = it["cost"].cpu().numpy(), it["grad"].cpu().numpy()
        I0, J, p0 = (it[f].cpu().numpy() for f in ("I0", "J", "p0"))
        for b in range(it["B"]):
            c, g = oracle.cost_and_grad(I0[b], J[b], p0[b], it["T"], it["sigma"],
                                        float(it["mu"][b]), float(it["rho"][b]),
                                        float(it["lam"][b]))
            np.testing.assert_allclose(cost[b], c, rtol=COST_RTOL, atol=1e-12)
            e = np.linalg.norm(grad[b] - g) / np.linalg.norm(g)
            assert e <= GRAD_RTOL, (k, b, e)


def test_persistent_wait_timeout_is_reported_and_the_plan_recovers(meta):
    """Failure detection without a fault: problem 1's first phase never reports its
    tiles, so its second phase's bounded wait (50 ms) runs out; the launch is abandoned,
    the plan and that problem's workspace report the timeout, and after clearing both
    the plan runs normally."""
    probs = make_problems(seed=980)[:4]
    plan = meta.GroupPlan(probs, persistent=True)
    plan.selftest_timeout(hold=1, limit_ns=50_000_000)
    assert plan.status() & 1 == 1
    assert plan.items[1]["ws"].status() & 1 == 1
    assert plan.status(clear=True) & 1 == 1
    assert plan.status() == 0
    for it in plan.items:
        it["ws"].status(clear=True)
    plan.launch()
    torch.cuda.synchronize()
    assert plan.status() == 0
    for it in plan.items:
        c, g = eager(meta, it)
        torch.cuda.synchronize()
        assert torch.equal(it["cost"], c) and torch.equal(it["grad"], g)


def test_persistent_plan_refuses_what_it_cannot_replay(meta):
    p = make_problems()[:1]
    p[0]["scheme"] = "euler"
    with pytest.raises(meta.MetaError) as e:
        meta.GroupPlan(p, persistent=True)
    assert e.value.code == 7  # META_ERR_UNSUPPORTED
