"""meta_cost_and_grad_noalloc: the entry point for callers that cannot allocate
device memory (graph-capture regions, plug-ins whose host owns the device
memory, real-time loops).  It runs on the library's fixed 64 MiB device array
instead of a caller-provided workspace, so it must give what meta_cost_and_grad
gives, call after call, although the array keeps the previous call's contents.

Collected last on purpose (file name): a failure here leaves every other test
already run.  Works alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest
from scipy import ndimage

import phantoms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GRAD_RTOL = 1e-3   # the gradient tolerance of the parity tests
COST_RTOL = 1e-5   # the cost tolerance of the parity tests


@pytest.fixture(scope="module")
def meta():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_08817_gb300 import _build
    _build.build()
    import paper_2106_08817_gb300 as m
    return m


def _noalloc_via_c_abi(meta, I0, J, p0, T, sigma, mu, rho, lam, ckpt=0, scheme="sl"):
    """Call the C entry point directly (ctypes), outputs preallocated here."""
    lib = meta._load()
    B = I0.shape[0]
    cost = torch.full((B, 3), float("nan"), dtype=torch.float64, device="cuda")
    grad = torch.full_like(I0, float("nan"))
    pr = meta._problem(I0.dim() - 1, tuple(I0.shape[1:]), B, T, sigma, ckpt, 0, scheme)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    rc = lib.meta_cost_and_grad_noalloc(ctypes.byref(pr), p(I0), p(J), p(p0), p(mu), p(rho),
                                        p(lam), p(cost), p(grad),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, meta.STATUS.get(rc, rc)
    return cost, grad


def _check(c_na, g_na, c_ref, g_ref):
    torch.cuda.synchronize()
    np.testing.assert_allclose(c_na.cpu().numpy(), c_ref.cpu().numpy(), rtol=COST_RTOL)
    a, b = g_na.cpu().numpy(), g_ref.cpu().numpy()
    assert np.isfinite(a).all()
    assert np.linalg.norm(a - b) <= GRAD_RTOL * np.linalg.norm(b)


def test_noalloc_matches_workspace_entry_point_on_two_calls_in_a_row(meta):
    dims = (64, 64)
    w = phantoms.disk_pair_64()
    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
    I0, J = t(w.I0), t(w.J)
    mu, rho, lam = t(w.mu), t(w.rho), t(w.lam)
    r = np.random.default_rng(77)
    momenta = [t(w.p0), t(ndimage.gaussian_filter(r.normal(size=dims), 2.0)[None] * 20.0)]
    for p0 in momenta:  # two calls in a row, different inputs
        c_ref, g_ref = meta.cost_and_grad(I0, J, p0, w.T, w.sigma, mu, rho, lam)
        c_na, g_na = _noalloc_via_c_abi(meta, I0, J, p0, w.T, w.sigma, mu, rho, lam)
        _check(c_na, g_na, c_ref, g_ref)
    assert meta.noalloc_status() == 0


# Problems whose workspace layouts differ from each other: the schemes' RAW
# buffer, the checkpoint and segment slots of a stride, and 3-D fields.
LAYOUTS = [((40, 56), 6, "sl", 0), ((40, 56), 6, "euler", 5), ((40, 56), 6, "hybrid", 0),
           ((40, 56), 6, "sl", 5), ((12, 20, 28), 6, "sl", 0), ((12, 20, 28), 6, "hybrid", 4)]


@pytest.mark.parametrize("k", range(len(LAYOUTS)))
def test_noalloc_ignores_what_another_layout_left_in_the_array(meta, k):
    """Before each compared call, a call of a different problem leaves its own data in
    the shared array; the result must still equal meta.cost_and_grad on a fresh
    workspace."""
    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
    dims, T, scheme, ckpt = LAYOUTS[k]
    pdims, pT, pscheme, pckpt = LAYOUTS[(k + 1) % len(LAYOUTS)]
    I, p = phantoms.random_fields(500 + k, 2, pdims, p_std=0.2)
    one = lambda v: t(np.full(2, v))
    _noalloc_via_c_abi(meta, t(I), t(I[::-1].copy()), t(p), pT, 2.0, one(0.1), one(1.0),
                       one(1e-3), pckpt, pscheme)
    I, p = phantoms.random_fields(600 + k, 2, dims, p_std=0.2)
    J = phantoms.random_fields(700 + k, 2, dims)[0]
    mu, rho, lam = t(np.array([0.0, 0.15])), one(1.0), one(1e-3)
    c_ref, g_ref = meta.cost_and_grad(t(I), t(J), t(p), T, 2.5, mu, rho, lam, ckpt=ckpt,
                                      scheme=scheme)
    c_na, g_na = _noalloc_via_c_abi(meta, t(I), t(J), t(p), T, 2.5, mu, rho, lam, ckpt, scheme)
    _check(c_na, g_na, c_ref, g_ref)


def test_noalloc_reports_a_device_timeout_and_clears_it(meta):
    """A bounded device wait that runs out on the no-allocation array is reported by
    meta_noalloc_status (bit 0, META_ERR_TIMEOUT through the C ABI), raised by the
    binding's checked call, and cleared; the next call runs normally."""
    lib = meta._load()
    dev = torch.device("cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    meta.noalloc_selftest_timeout(50_000_000)
    bits = ctypes.c_uint(0)
    assert lib.meta_noalloc_status(0, st, ctypes.byref(bits)) == 5  # META_ERR_TIMEOUT
    assert bits.value & 1
    assert meta.noalloc_status(clear=True) & 1
    assert meta.noalloc_status() == 0
    w = phantoms.disk_pair_64()
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
    c_ref, g_ref = meta.cost_and_grad(t(w.I0), t(w.J), t(w.p0), w.T, w.sigma, t(w.mu),
                                      t(w.rho), t(w.lam))
    c_na, g_na = meta.cost_and_grad_noalloc(t(w.I0), t(w.J), t(w.p0), w.T, w.sigma, t(w.mu),
                                            t(w.rho), t(w.lam), check_status=True)
    _check(c_na, g_na, c_ref, g_ref)
    assert meta.noalloc_status() == 0


def test_noalloc_rejects_problems_beyond_its_fixed_scratch(meta):
    lib = meta._load()
    big = meta._problem(2, (256, 256), 16, 20, 6.0)  # needs ~384 MiB of workspace
    assert meta.workspace_size((256, 256), 16, 20, 6.0) > meta.NOALLOC_MAX_BYTES
    fake = ctypes.c_void_p(0x1000)
    rc = lib.meta_cost_and_grad_noalloc(ctypes.byref(big), fake, fake, fake, fake, fake, fake,
                                        fake, fake, ctypes.c_void_p(0))
    assert rc == 3  # META_ERR_WORKSPACE, before any GPU work
