"""Auxiliary subsystems on the GPU: stopping and resuming a registration (gradient
descent and L-BFGS) through a host file, bit for bit; gradient descent against the
FP64 oracle; the phase ranges a real call pushes (its NVTX ranges); the autotuner's
cache file, written on a miss and used without timing on a hit."""
import json

import numpy as np
import pytest

import oracle
import phantoms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


# (dims, batch, T, sigma, ckpt): 2-D with two instances, 3-D with checkpoint segments
CASES = [((48, 40), 2, 5, 2.0, 0), ((12, 20, 16), 1, 6, 1.5, 2)]


def problem(dims, B, seed):
    I0, _ = phantoms.random_fields(seed, B, dims)
    J, _ = phantoms.random_fields(seed + 1, B, dims)
    p0 = smooth_p(seed + 2, (B,) + dims, 5.0)
    return I0, J, p0


@pytest.mark.parametrize("optimizer", ["lbfgs", "gd"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_saved_and_resumed_registration_equals_one_run(meta, tmp_path, optimizer, case):
    dims, B, T, sigma, ckpt = CASES[case]
    I0, J, p0 = problem(dims, B, 700 + 10 * case)
    kw = dict(mu=[0.1, 0.05][:B], rho=[1.0, 1.2][:B], lam=[1e-3, 1e-2][:B],
              optimizer=optimizer, m=3, h0=0.3, ckpt=ckpt)
    whole = meta.Registration(cuda(I0), cuda(J), cuda(p0), T, sigma, **kw)
    whole.run(6)
    part = meta.Registration(cuda(I0), cuda(J), cuda(p0), T, sigma, **kw)
    part.run(2)
    part.run(1)  # a resume inside the process, too
    f = tmp_path / "reg.npz"
    part.save(f)
    del part
    torch.cuda.synchronize()
    back = meta.Registration.resume(f, cuda(I0), cuda(J))
    assert back.iterations == 3 and back.optimizer == optimizer
    back.run(3)
    torch.cuda.synchronize()
    assert torch.equal(back.p, whole.p)
    assert np.array_equal(back.costs, whole.costs)
    assert whole.costs[-1].sum() < whole.costs[0].sum()
    with pytest.raises(ValueError):  # other images
        meta.Registration.resume(f, cuda(J), cuda(I0))


def test_lbfgs_resume_refuses_a_workspace_without_a_finished_run(meta):
    dims, B, T, sigma, ckpt = CASES[0]
    I0, J, p0 = problem(dims, B, 760)
    reg = meta.Registration(cuda(I0), cuda(J), cuda(p0), T, sigma, [0.1, 0.1], optimizer="lbfgs")
    reg._started = True  # lws is all zeros: no state header
    with pytest.raises(meta.MetaError) as e:
        reg.run(1)
    assert e.value.code == 8
    assert torch.equal(reg.p, cuda(p0))  # nothing ran


def test_gradient_descent_follows_the_oracle(meta):
    """Three normalised gradient steps on the 64^2 disk pair: each iterate's cost
    against the oracle's, whose steps use its own FP64 gradient."""
    w = phantoms.disk_pair_64(random_p0=False)
    I0, J = w.I0[0], w.J[0]
    p = np.zeros_like(I0, dtype=np.float64)
    mu, rho, lam, h0, iters = 0.1, 1.0, 1e-3, 0.5, 3
    ref = []
    for k in range(iters + 1):
        c, g = oracle.cost_and_grad(I0, J, p, w.T, w.sigma, mu, rho, lam)
        ref.append(float(np.sum(c)))
        if k < iters:
            p = p - h0 * g / np.abs(g).max()
    pg, hist = meta.gd_minimize(cuda(I0[None]), cuda(J[None]), cuda(np.zeros_like(I0)[None]),
                                w.T, w.sigma, mu, rho, lam, iters=iters, h0=h0)
    np.testing.assert_allclose(hist[:, 0], ref, rtol=1e-4)
    e = np.linalg.norm(pg[0].cpu().numpy() - p) / np.linalg.norm(p)
    assert e <= 1e-3, e
    assert ref[-1] < ref[0]


def test_phase_ranges_of_a_checkpointed_call(meta):
    """T = 7 with checkpoint stride 3: segments [0,3), [3,6), [6,7); one set of segment
    slots (two would not be smaller than the whole trajectory), so the adjoint re-runs
    the two segments before the last, newest first."""
    dims, B, T, sigma = (24, 28), 1, 7, 2.0
    I0, J, p0 = problem(dims, B, 780)
    ws = meta.Workspace(dims, B, T, sigma, "cuda", 3)
    with meta.trace() as ev:
        meta.cost_and_grad(cuda(I0), cuda(J), cuda(p0), T, sigma, 0.1, workspace=ws, ckpt=3)
    torch.cuda.synchronize()
    P = lambda n: ("meta." + n, 1)
    Q = lambda n: ("meta." + n, 0)
    assert ev == [P("cost_and_grad"), P("forward"), Q("forward"), P("cost"), Q("cost"),
                  P("adjoint"), P("recompute"), Q("recompute"), P("recompute"), Q("recompute"),
                  Q("adjoint"), Q("cost_and_grad")]
    with meta.trace() as ev:  # every state kept: no recompute
        meta.cost_and_grad(cuda(I0), cuda(J), cuda(p0), T, sigma, 0.1)
    assert [e for e in ev if e[0] == "meta.recompute"] == []
    assert ev[0] == P("cost_and_grad") and ev[-1] == Q("cost_and_grad")


def test_autotuner_cache_file_is_written_then_used_without_timing(meta, tmp_path):
    dims, B, T, sigma = (56, 72), 2, 3, 2.5
    I0, J, p0 = problem(dims, B, 790)
    f = tmp_path / "tiles.json"
    meta.set_tuning(dims, B, sigma, None)
    try:
        assert meta.tuning_cache(f) == 0
        t1 = meta.autotune(cuda(I0), cuda(J), cuda(p0), T, sigma, [0.1, 0.1])
        doc = json.loads(f.read_text())
        e = [x for x in doc["entries"] if x["dims"] == list(dims) and x["batch"] == B]
        assert len(e) == 1 and {k: e[0][k] for k in t1} == t1
        # a new process would read the file: forget the table, name the cache again
        meta.set_tuning(dims, B, sigma, None)
        assert meta.tuning_cache(f) == 1
        import time
        t0 = time.perf_counter()
        t2 = meta.autotune(cuda(I0), cuda(J), cuda(p0), T, sigma, [0.1, 0.1])
        hit_s = time.perf_counter() - t0
        assert t2 == t1 and meta.tuning(dims, B, sigma) == t1
        assert hit_s < 0.5  # a miss times dozens of calls
    finally:
        meta.tuning_cache(None)
        meta.set_tuning(dims, B, sigma, None)
