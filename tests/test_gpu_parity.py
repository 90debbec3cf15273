"""Parity of the sm_103a library (through the C ABI) with the FP64 oracle.

Tolerances: I_T and p_T max-abs <= 1e-4 (scaled by max(1, |p|) for p) for
images in [0, 1]; dL/dp0 relative L2 <= 1e-3; the three cost terms relative
1e-5 (FP64 accumulation of FP32 fields).  Inputs are the seeded phantoms of
the workloads and random smooth fields on ragged shapes that span several
tiles (x tiles are 128 wide, strided tiles 128 long, pointwise tiles 32 x 8).
"""
import ctypes

import numpy as np
import pytest
from scipy import ndimage

import oracle
import phantoms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FWD_ATOL = 1e-4
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


def rel_l2(a, b):
    return float(np.sqrt(((a - b) ** 2).sum()) / max(np.sqrt((b ** 2).sum()), 1e-300))


def smooth_p(seed, shape, scale, s=2.0):
    r = np.random.default_rng(seed)
    out = np.empty(shape, np.float32)
    for b in range(shape[0]):
        out[b] = ndimage.gaussian_filter(r.normal(size=shape[1:]), s) * scale
    return out


def check_forward(meta, I0, p0, T, sigma, mu, rho, p_update=0, scheme="sl"):
    I1, p1, ws = meta.shoot_forward(cuda(I0), cuda(p0), T, sigma, mu, rho, p_update=p_update,
                                    scheme=scheme)
    I1, p1 = I1.cpu().numpy(), p1.cpu().numpy()
    for b in range(I0.shape[0]):
        mb = mu[b] if np.ndim(mu) else mu
        rb = rho[b] if np.ndim(rho) else rho
        It, pt, _ = oracle.shoot(I0[b], p0[b], T, sigma, mb, rb, p_update=p_update,
                                 scheme=scheme)
        assert np.abs(I1[b] - It[-1]).max() <= FWD_ATOL, b
        assert np.abs(p1[b] - pt[-1]).max() <= FWD_ATOL * max(1.0, np.abs(pt[-1]).max()), b
    assert ws.status(clear=True) & 1 == 0


def check_cost_grad(meta, I0, J, p0, T, sigma, mu, rho, lam, grad_rtol=GRAD_RTOL, ckpt=0,
                    p_update=0, scheme="sl"):
    B = I0.shape[0]
    ws = meta.Workspace(I0.shape[1:], B, T, sigma, "cuda", ckpt, scheme)
    cost, grad = meta.cost_and_grad(cuda(I0), cuda(J), cuda(p0), T, sigma, mu, rho, lam,
                                    workspace=ws, ckpt=ckpt, p_update=p_update, scheme=scheme)
    check_cost_grad.status = ws.status()
    assert check_cost_grad.status & 1 == 0
    cost, grad = cost.cpu().numpy(), grad.cpu().numpy()
    worst = 0.0
    for b in range(I0.shape[0]):
        pick = lambda v: v[b] if np.ndim(v) else v
        c, g = oracle.cost_and_grad(I0[b], J[b], p0[b], T, sigma, pick(mu), pick(rho), pick(lam),
                                    p_update=p_update, scheme=scheme)
        np.testing.assert_allclose(cost[b], c, rtol=COST_RTOL, atol=1e-12)
        e = rel_l2(grad[b], g)
        worst = max(worst, e)
        assert e <= grad_rtol, (b, e)
    return worst


# ----------------------------------------------------------------- forward

def test_zero_momentum_leaves_image_unchanged_bitwise(meta):
    w = phantoms.disk_pair_64(random_p0=False)
    I1, p1, _ = meta.shoot_forward(cuda(w.I0), cuda(w.p0), w.T, w.sigma, w.mu, w.rho)
    np.testing.assert_array_equal(I1.cpu().numpy(), w.I0)
    np.testing.assert_array_equal(p1.cpu().numpy(), 0.0)


def test_forward_disk64(meta):
    w = phantoms.disk_pair_64()
    check_forward(meta, w.I0, w.p0, w.T, w.sigma, float(w.mu[0]), float(w.rho[0]))


@pytest.mark.parametrize("dims,B,T,sigma", [((37, 141), 3, 4, 2.3), ((130, 259), 2, 3, 4.0),
                                            ((5, 3), 2, 2, 0.7), ((64, 64), 1, 1, 18.0)])
def test_forward_ragged_2d(meta, dims, B, T, sigma):
    I0, _ = phantoms.random_fields(11, B, dims)
    p0 = smooth_p(12, (B,) + dims, 40.0)
    check_forward(meta, I0, p0, T, sigma, [0.0, 0.3, 0.1][:B], [1.0, 0.7, 1.5][:B])


@pytest.mark.parametrize("dims,B,T,sigma", [((9, 13, 135), 2, 3, 1.5), ((21, 6, 10), 1, 4, 2.0)])
def test_forward_ragged_3d(meta, dims, B, T, sigma):
    I0, _ = phantoms.random_fields(13, B, dims)
    p0 = smooth_p(14, (B,) + dims, 30.0, s=1.5)
    check_forward(meta, I0, p0, T, sigma, [0.2, 0.0][:B], [1.0, 1.3][:B])


# ----------------------------------------------------------------- det momentum update
# p' = p~ det(Id - dt Dv): the same tolerances as the default update.

@pytest.mark.parametrize("dims,B,T,sigma", [((37, 141), 3, 4, 2.3), ((5, 3), 2, 2, 0.7),
                                            ((9, 13, 135), 2, 3, 1.5), ((21, 6, 10), 1, 4, 2.0)])
def test_det_update_forward(meta, dims, B, T, sigma):
    I0, _ = phantoms.random_fields(21, B, dims)
    p0 = smooth_p(22, (B,) + dims, 40.0 if len(dims) == 2 else 30.0, s=1.5)
    mu, rho = [0.0, 0.05, 0.02][:B], [1.0, 0.7, 1.5][:B]
    check_forward(meta, I0, p0, T, sigma, mu, rho, p_update="det")
    # here the two updates differ by more than the tolerance (oracle: 8e-4 to 40)
    a = meta.shoot_forward(cuda(I0), cuda(p0), T, sigma, mu, rho)
    b = meta.shoot_forward(cuda(I0), cuda(p0), T, sigma, mu, rho, p_update="det")
    assert float((a[1] - b[1]).abs().max()) > 5 * FWD_ATOL


@pytest.mark.parametrize("dims,B,T,sigma,scale,k", [((37, 141), 2, 5, 2.3, 40.0, 0),
                                                    ((37, 141), 2, 5, 2.3, 40.0, 2),
                                                    ((9, 13, 135), 2, 3, 1.5, 30.0, 0),
                                                    ((12, 10, 11), 1, 4, 1.0, 30.0, 3)])
def test_det_update_cost_and_grad(meta, dims, B, T, sigma, scale, k):
    """Cost and dL/dp0 against the oracle with the det update, keep-all and with step
    checkpointing (bit-identical to keep-all).  An FP32 torch.autograd run of the same
    scheme is within 3e-5 (relative L2) of the oracle on these inputs."""
    I0, J = phantoms.random_fields(23, B, dims)
    p0 = smooth_p(24, (B,) + dims, scale, s=1.5)
    mu, rho, lam = [0.05, 0.0][:B], [1.0, 1.3][:B], 1e-3
    check_cost_grad(meta, I0, J, p0, T, sigma, mu, rho, lam, ckpt=k, p_update="det")
    if k:
        c0, g0 = meta.cost_and_grad(cuda(I0), cuda(J), cuda(p0), T, sigma, mu, rho, lam,
                                    p_update="det")
        ck, gk = meta.cost_and_grad(cuda(I0), cuda(J), cuda(p0), T, sigma, mu, rho, lam,
                                    ckpt=k, p_update="det")
        torch.cuda.synchronize()
        assert torch.equal(c0, ck) and torch.equal(g0, gk)


def test_det_update_shoot_adjoint(meta):
    dims, T, sigma = (40, 52), 4, 2.0
    I0, _ = phantoms.random_fields(25, 1, dims)
    p0 = smooth_p(26, (1,) + dims, 120.0, s=1.5)
    r = np.random.default_rng(27)
    gI1, gp1 = r.normal(size=(1,) + dims), r.normal(size=(1,) + dims)
    _, _, ws = meta.shoot_forward(cuda(I0), cuda(p0), T, sigma, 0.2, 1.0, p_update="det")
    gI0, gp0 = meta.shoot_adjoint(cuda(gI1), cuda(gp1), ws, T, sigma, 0.2, 1.0, p_update="det")
    eI, ep = oracle.adjoint(I0[0], p0[0], gI1[0], gp1[0], T, sigma, 0.2, 1.0, p_update="det")
    assert rel_l2(gp0.cpu().numpy()[0], ep) <= GRAD_RTOL
    assert rel_l2(gI0.cpu().numpy()[0], eI) <= GRAD_RTOL


# ----------------------------------------------------------------- Eulerian and hybrid
# Forward only (Sec. 2.3): the same tolerances as the semi-Lagrangian forward.

@pytest.mark.parametrize("scheme", ["euler", "hybrid"])
@pytest.mark.parametrize("dims,B,T,sigma,scale", [((37, 141), 2, 4, 2.3, 40.0),
                                                  ((5, 3), 2, 2, 0.7, 10.0),
                                                  ((9, 13, 135), 2, 3, 1.5, 30.0),
                                                  ((21, 6, 10), 1, 4, 2.0, 30.0)])
def test_other_schemes_forward(meta, dims, B, T, sigma, scale, scheme):
    I0, _ = phantoms.random_fields(31, B, dims)
    p0 = smooth_p(32, (B,) + dims, scale, s=1.5)
    check_forward(meta, I0, p0, T, sigma, [0.1, 0.0][:B], [1.0, 1.3][:B], scheme=scheme)
    # with step checkpoints the forward runs the same launches on the same data
    a = meta.shoot_forward(cuda(I0), cuda(p0), T, sigma, [0.1, 0.0][:B], [1.0, 1.3][:B],
                           scheme=scheme)
    b = meta.shoot_forward(cuda(I0), cuda(p0), T, sigma, [0.1, 0.0][:B], [1.0, 1.3][:B],
                           scheme=scheme, ckpt=2)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


@pytest.mark.parametrize("scheme", ["euler", "hybrid"])
def test_other_schemes_zero_momentum_and_deformation(meta, scheme):
    w = phantoms.disk_pair_64(random_p0=False)
    I1, p1, _ = meta.shoot_forward(cuda(w.I0), cuda(w.p0), w.T, w.sigma, w.mu, w.rho,
                                   scheme=scheme)
    np.testing.assert_array_equal(I1.cpu().numpy(), w.I0)
    assert bool((p1 == 0).all())
    # the deformation integrates the scheme's own v_t
    I0, _ = phantoms.random_fields(33, 1, (40, 52))
    p0 = smooth_p(34, (1, 40, 52), 40.0, s=1.5)
    _, _, phi, jac, _ = meta.shoot_deform(cuda(I0), cuda(p0), 4, 2.0, 0.1, 1.0, scheme=scheme)
    wr, Jr = oracle.deformation(I0[0], p0[0], 4, 2.0, 0.1, 1.0, scheme=scheme)
    assert np.abs(phi.cpu().numpy()[0] - wr).max() <= FWD_ATOL * max(1.0, np.abs(wr).max())
    assert np.abs(jac.cpu().numpy()[0] - Jr).max() <= 1e-3


@pytest.mark.parametrize("scheme", ["euler", "hybrid"])
@pytest.mark.parametrize("dims,B,T,sigma,scale,k", [((37, 141), 2, 5, 2.3, 40.0, 0),
                                                    ((37, 141), 2, 5, 2.3, 40.0, 2),
                                                    ((5, 3), 2, 2, 0.7, 10.0, 0),
                                                    ((9, 13, 135), 2, 3, 1.5, 30.0, 0),
                                                    ((12, 10, 11), 1, 4, 1.0, 30.0, 3)])
def test_other_schemes_cost_and_grad(meta, dims, B, T, sigma, scale, k, scheme):
    """Cost and dL/dp0 of the Eulerian and hybrid schemes against the oracle's
    transposes, keep-all and with step checkpointing (bit-identical to keep-all)."""
    I0, J = phantoms.random_fields(37, B, dims)
    p0 = smooth_p(38, (B,) + dims, scale, s=1.5)
    mu, rho, lam = [0.05, 0.0][:B], [1.0, 1.3][:B], 1e-3
    check_cost_grad(meta, I0, J, p0, T, sigma, mu, rho, lam, ckpt=k, scheme=scheme)
    if k:
        c0, g0 = meta.cost_and_grad(cuda(I0), cuda(J), cuda(p0), T, sigma, mu, rho, lam,
                                    scheme=scheme)
        ck, gk = meta.cost_and_grad(cuda(I0), cuda(J), cuda(p0), T, sigma, mu, rho, lam,
                                    ckpt=k, scheme=scheme)
        torch.cuda.synchronize()
        assert torch.equal(c0, ck) and torch.equal(g0, gk)


@pytest.mark.parametrize("scheme", ["euler", "hybrid"])
def test_other_schemes_shoot_adjoint(meta, scheme):
    dims, T, sigma = (40, 52), 4, 2.0
    I0, _ = phantoms.random_fields(39, 1, dims)
    p0 = smooth_p(40, (1,) + dims, 40.0, s=1.5)
    r = np.random.default_rng(41)
    gI1, gp1 = r.normal(size=(1,) + dims), r.normal(size=(1,) + dims)
    _, _, ws = meta.shoot_forward(cuda(I0), cuda(p0), T, sigma, 0.2, 1.0, scheme=scheme)
    gI0, gp0 = meta.shoot_adjoint(cuda(gI1), cuda(gp1), ws, T, sigma, 0.2, 1.0, scheme=scheme)
    eI, ep = oracle.adjoint(I0[0], p0[0], gI1[0], gp1[0], T, sigma, 0.2, 1.0, scheme=scheme)
    assert rel_l2(gp0.cpu().numpy()[0], ep) <= GRAD_RTOL
    assert rel_l2(gI0.cpu().numpy()[0], eI) <= GRAD_RTOL
    # the autograd Function runs the same calls
    Ia, pa = cuda(I0).requires_grad_(True), cuda(p0).requires_grad_(True)
    I1, p1 = meta.shoot(Ia, pa, T, sigma, 0.2, 1.0, scheme=scheme)
    ((I1 * cuda(gI1)).sum() + (p1 * cuda(gp1)).sum()).backward()
    assert torch.equal(pa.grad, gp0) and torch.equal(Ia.grad, gI0)


@pytest.mark.parametrize("scheme", ["euler", "hybrid"])
def test_eulerian_momentum_total_full_size(meta, scheme):
    """16 x 256^2, T = 20, sigma 6: p0 inside a disk of radius 60 around the centre, so p v
    vanishes on the border for all 20 steps and sum p_T = sum p_0 exactly in exact
    arithmetic; FP32 keeps it to 1e-4 of sum |p_0|."""
    w = phantoms.ellipse_pairs()
    Y, X = np.meshgrid(np.arange(256.0), np.arange(256.0), indexing="ij")
    inside = ((Y - 127.5) ** 2 + (X - 127.5) ** 2 <= 60.0 ** 2)
    p0 = (smooth_p(35, w.p0.shape, 1000.0, s=3.0) * inside).astype(np.float32)
    I1, p1, _ = meta.shoot_forward(cuda(w.I0), cuda(p0), w.T, w.sigma, 0.0, 1.0, scheme=scheme)
    p1 = p1.cpu().numpy().astype(np.float64)
    for b in range(p0.shape[0]):
        tot0, tot1 = float(p0[b].astype(np.float64).sum()), float(p1[b].sum())
        assert abs(tot1 - tot0) <= 1e-4 * np.abs(p0[b]).sum(), (b, tot0, tot1)
        assert np.abs(p1[b] - p0[b]).max() > 1.0  # the momentum moved (oracle: by up to 66)


# ----------------------------------------------------------------- L-BFGS

def test_lbfgs_direction_matches_oracle(meta):
    """Two instances, three pairs each; in instance 1 the middle pair has s.y < 0 and is
    skipped.  Vectors are FP32, dot products FP64: relative L2 1e-5."""
    dims, B = (33, 47), 2
    r = np.random.default_rng(41)
    S = [smooth_p(42 + i, (B,) + dims, 1.0) for i in range(3)]
    Y = [(1.5 + 0.5 * i) * S[i] + 0.1 * smooth_p(52 + i, (B,) + dims, 1.0) for i in range(3)]
    Y[1][1] = -Y[1][1]
    g = smooth_p(60, (B,) + dims, 1.0)
    d = meta.lbfgs_direction(cuda(g), [cuda(x) for x in S], [cuda(x) for x in Y], m=4)
    d = d.cpu().numpy()
    for b in range(B):
        ref = oracle.lbfgs_direction(g[b], [x[b] for x in S], [x[b] for x in Y])
        assert rel_l2(d[b], ref) <= 1e-5, b


def test_lbfgs_minimize_follows_the_oracle(meta):
    """Four L-BFGS iterations on two registrations at once (the 64^2 disk pair with
    mu = 0.1 and with mu = 0): the GPU driver's cost history against the oracle's, same
    rules.  Every line-search decision of these iterations clears the Armijo threshold
    by at least 1e-4 of the cost (checked on the oracle's trials), far above the FP32
    cost error, so both take the same steps."""
    w = phantoms.disk_pair_64(random_p0=False)
    I0 = np.concatenate([w.I0, w.I0]); J = np.concatenate([w.J, w.J])
    p0 = np.zeros_like(I0)
    mu, rho, lam = [0.1, 0.0], [1.0, 1.0], [1e-3, 1e-3]
    iters, m, h0 = 4, 5, 0.5
    p, hist, done = meta.lbfgs_minimize(cuda(I0), cuda(J), cuda(p0), w.T, w.sigma, mu, rho, lam,
                                        iters=iters, m=m, h0=h0)
    p = p.cpu().numpy()
    for b in range(2):
        x, h_ref, margins = oracle.lbfgs_minimize(I0[b], J[b], p0[b], w.T, w.sigma, mu[b],
                                                  rho[b], lam[b], iters, m, h0)
        assert min(abs(v) for it in margins for v in it) > 1e-4
        np.testing.assert_allclose(hist[:, b], h_ref, rtol=1e-4)
        assert rel_l2(p[b], x) <= 1e-3
        assert done[b] == iters and h_ref[-1] < (0.25 if mu[b] > 0 else 0.9) * h_ref[0]


# ----------------------------------------------------------------- deformation
# phi_T - Id against the oracle within FWD_ATOL (scaled by max(1, |w|)), the same bar as
# I_T.  det D phi_T differences w over one or two voxels, so each entry of D phi carries
# at most twice that error; a 3 x 3 determinant of entries near 1 sums six products of
# three entries, hence JAC_ATOL = 2 * 3 * FWD_ATOL, rounded up to 1e-3.
JAC_ATOL = 1e-3


def check_deform(meta, I0, p0, T, sigma, mu, rho, ckpt=0):
    I1, p1, phi, jac, ws = meta.shoot_deform(cuda(I0), cuda(p0), T, sigma, mu, rho, ckpt=ckpt)
    F1, q1, _ = meta.shoot_forward(cuda(I0), cuda(p0), T, sigma, mu, rho)
    torch.cuda.synchronize()
    assert torch.equal(I1, F1) and torch.equal(p1, q1)  # the deformation leaves the shot alone
    phi, jac = phi.cpu().numpy(), jac.cpu().numpy()
    moved = 0.0
    for b in range(I0.shape[0]):
        pick = lambda v: v[b] if np.ndim(v) else v
        w, J = oracle.deformation(I0[b], p0[b], T, sigma, pick(mu), pick(rho))
        assert np.abs(phi[b] - w).max() <= FWD_ATOL * max(1.0, np.abs(w).max()), b
        assert np.abs(jac[b] - J).max() <= JAC_ATOL, b
        moved = max(moved, float(np.abs(w).max()))
    assert ws.status(clear=True) & 1 == 0
    return phi, jac, moved


@pytest.mark.parametrize("dims,B,T,sigma", [((37, 141), 2, 5, 2.3), ((5, 3), 2, 2, 0.7),
                                            ((9, 13, 135), 2, 3, 1.5), ((21, 6, 10), 1, 4, 2.0)])
def test_deformation_matches_oracle(meta, dims, B, T, sigma):
    I0, _ = phantoms.random_fields(15, B, dims)
    p0 = smooth_p(16, (B,) + dims, 40.0 if len(dims) == 2 else 30.0, s=1.5)
    mu, rho = [0.2, 0.0][:B], [1.0, 1.4][:B]
    phi, jac, moved = check_deform(meta, I0, p0, T, sigma, mu, rho)
    assert moved > 0.25  # the grid moves by a good part of a voxel (up to 2.6 voxels)
    # with step checkpointing the same launches run on the same data
    _, _, phi3, jac3, _ = meta.shoot_deform(cuda(I0), cuda(p0), T, sigma, mu, rho, ckpt=2)
    assert np.array_equal(phi3.cpu().numpy(), phi) and np.array_equal(jac3.cpu().numpy(), jac)


def test_deformation_at_zero_momentum_is_identity_bitwise(meta):
    w = phantoms.disk_pair_64(random_p0=False)
    _, _, phi, jac, _ = meta.shoot_deform(cuda(w.I0), cuda(w.p0), w.T, w.sigma, w.mu, w.rho)
    assert bool((phi == 0).all()) and bool((jac == 1).all())
    _, _, phi1, jac1, _ = meta.shoot_deform(cuda(w.I0), cuda(w.p0), w.T, w.sigma, w.mu, w.rho,
                                            want_jac=False)
    assert jac1 is None and torch.equal(phi1, phi)


@pytest.mark.parametrize("which", ["ellipses16x256", "mri160"])
def test_lddmm_deformation_carries_an_affine_image_full_size(meta, which):
    """At the workloads' full sizes (16 x 256^2 sigma 6; 160 x 192 x 160 sigma 6), T = 20,
    mu = 0: I_T = I_0 o phi_T for an affine I_0, since image and grid are interpolated at
    the same feet with the same weights.  FP32 bound for |I| <= 1: a step rounds at
    most 3 times in each of its 3 lerp levels (6e-8 each, not amplified by the convex
    weights), 5.4e-7 per step and 1.1e-5 over 20 steps."""
    if which == "ellipses16x256":
        dims, B, a = (256, 256), 16, (0.5 / 256, -0.4 / 256)
    else:
        dims, B, a = (160, 192, 160), 1, (0.3 / 160, -0.25 / 192, 0.35 / 160)
    X = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in dims], indexing="ij")
    ramp = 0.45 + sum(ae * Xe for ae, Xe in zip(a, X))
    I0 = np.broadcast_to(ramp, (B,) + dims).astype(np.float32)
    p0 = smooth_p(17, (B,) + dims, 20000.0, s=4.0)
    I1, _, phi, _, _ = meta.shoot_deform(cuda(I0), cuda(p0), 20, 6.0, 0.0, 1.0, want_jac=False)
    I1, phi = I1.cpu().numpy().astype(np.float64), phi.cpu().numpy().astype(np.float64)
    carried = 0.45 + sum(ae * (Xe[None] + phi[:, e]) for e, (ae, Xe) in enumerate(zip(a, X)))
    assert np.abs(I1 - carried).max() <= 2e-5
    assert np.abs(phi).max() > 0.5  # the grid moves by a voxel or more (2-D: about 5)


# ----------------------------------------------------------------- cost + gradient

def test_cost_and_grad_disk64(meta):
    w = phantoms.disk_pair_64()
    check_cost_grad(meta, w.I0, w.J, w.p0, w.T, w.sigma, w.mu, w.rho, w.lam)


def test_cost_and_grad_disk64_zero_momentum(meta):
    w = phantoms.disk_pair_64(random_p0=False)
    check_cost_grad(meta, w.I0, w.J, w.p0, w.T, w.sigma, w.mu, w.rho, w.lam)


FD_EPS, FD_RTOL = 3e-2, 5e-3


@pytest.mark.parametrize("p_update,scheme", [(0, "sl"), (1, "sl"), (0, "euler"), (0, "hybrid")])
@pytest.mark.parametrize("dims,T,sigma", [((40, 37), 6, 2.0), ((12, 14, 13), 5, 1.5)])
def test_gradient_matches_central_differences_of_the_gpu_cost(meta, dims, T, sigma, p_update,
                                                              scheme):
    """The library's dL/dp0 against central differences of its own cost, with no oracle
    involved: L(p0 + eps d) - L(p0 - eps d) = <dL/dp0, 2 eps d> up to O(eps^3), along the
    gradient and along a smooth direction (|d| <= 1, eps = 0.03, feet moving up to 0.3
    voxel a step).  The FP32 torch re-implementation of the scheme meets this within
    7e-4 on the same inputs; the bound is 5e-3."""
    shape = (1,) + dims
    I0 = phantoms.random_fields(20, 1, dims)[0]
    J = np.clip(I0 + 0.2 * smooth_p(21, shape, 1.0, s=1.5), 0.0, 1.0).astype(np.float32)
    p0 = smooth_p(22, shape, 25.0, s=1.5)
    args = (T, sigma, 0.1, 1.0, 1e-3)
    kw = dict(p_update=p_update, scheme=scheme)

    def L(q):
        c, _ = meta.cost_and_grad(cuda(I0), cuda(J), cuda(q), *args, want_grad=False, **kw)
        return float(c.cpu().numpy().sum())

    _, g = meta.cost_and_grad(cuda(I0), cuda(J), cuda(p0), *args, **kw)
    g = g.cpu().numpy().astype(np.float64)
    for d in (g, smooth_p(99, shape, 1.0).astype(np.float64)):
        d = d / np.abs(d).max()
        qp = (p0 + FD_EPS * d).astype(np.float32)
        qm = (p0 - FD_EPS * d).astype(np.float32)
        fd = L(qp) - L(qm)
        an = float((g * (qp.astype(np.float64) - qm)).sum())  # the steps actually taken
        assert abs(fd - an) <= FD_RTOL * abs(an), (fd, an)


@pytest.mark.parametrize("p_update,scheme", [(0, "sl"), (1, "sl"), (0, "euler"), (0, "hybrid")])
@pytest.mark.parametrize("dims,T,sigma", [((40, 37), 6, 2.0), ((12, 14, 13), 5, 1.5)])
def test_shooting_adjoint_against_central_differences_of_the_gpu_shot(meta, dims, T, sigma,
                                                                      p_update, scheme):
    """meta_shoot_adjoint against central differences of the library's own forward
    shooting, with no oracle involved: for F = <gI1, I_T> + <gp1, p_T> and a tangent
    (dI, dp), F(+eps) - F(-eps) = <dL/dI0, 2 eps dI> + <dL/dp0, 2 eps dp> up to O(eps^3)
    (eps = 0.01, |dI|, |dp| <= 1).  The FP32 torch re-implementation meets this within
    3e-4 against the oracle's adjoint; the bound is 5e-3."""
    shape = (1,) + dims
    I0 = phantoms.random_fields(20, 1, dims)[0]
    p0 = smooth_p(22, shape, 25.0, s=1.5)
    gI1, gp1 = smooth_p(30, shape, 1.0), smooth_p(31, shape, 0.05)
    dI, dp = smooth_p(32, shape, 1.0), smooth_p(33, shape, 1.0)
    dI, dp = dI / np.abs(dI).max(), dp / np.abs(dp).max()
    args = (T, sigma, 0.1, 1.0)
    kw = dict(p_update=p_update, scheme=scheme)
    _, _, ws = meta.shoot_forward(cuda(I0), cuda(p0), *args, **kw)
    gI0, gp0 = meta.shoot_adjoint(cuda(gI1), cuda(gp1), ws, *args, **kw)
    gI0 = gI0.cpu().numpy().astype(np.float64)
    gp0 = gp0.cpu().numpy().astype(np.float64)

    def F(I, p):
        IT, pT, _ = meta.shoot_forward(cuda(I), cuda(p), *args, **kw)
        return float((IT.cpu().numpy().astype(np.float64) * gI1).sum()
                     + (pT.cpu().numpy().astype(np.float64) * gp1).sum())

    eps = 1e-2
    Ip, Im = (I0 + eps * dI).astype(np.float32), (I0 - eps * dI).astype(np.float32)
    pp, pm = (p0 + eps * dp).astype(np.float32), (p0 - eps * dp).astype(np.float32)
    fd = F(Ip, pp) - F(Im, pm)
    an = float((gI0 * (Ip.astype(np.float64) - Im)).sum() + (gp0 * (pp.astype(np.float64) - pm)).sum())
    assert abs(fd - an) <= 5e-3 * abs(an), (fd, an)


@pytest.mark.parametrize("dims,B,T,sigma,scale", [((37, 141), 3, 4, 2.3, 40.0),
                                                  ((70, 33), 2, 5, 3.0, 100.0)])
def test_cost_and_grad_ragged_2d(meta, dims, B, T, sigma, scale):
    I0, _ = phantoms.random_fields(21, B, dims)
    J, _ = phantoms.random_fields(22, B, dims)
    p0 = smooth_p(23, (B,) + dims, scale)
    check_cost_grad(meta, I0, J, p0, T, sigma, np.array([0.0, 0.2, 0.05][:B]),
                    np.array([1.0, 0.8, 1.2][:B]), np.array([1e-3, 1e-2, 0.1][:B]))


@pytest.mark.parametrize("dims,B,T,sigma", [((9, 13, 135), 2, 3, 1.5), ((12, 10, 11), 1, 4, 1.0)])
def test_cost_and_grad_ragged_3d(meta, dims, B, T, sigma):
    I0, _ = phantoms.random_fields(31, B, dims)
    J, _ = phantoms.random_fields(32, B, dims)
    p0 = smooth_p(33, (B,) + dims, 30.0, s=1.5)
    check_cost_grad(meta, I0, J, p0, T, sigma, np.array([0.1, 0.0][:B]),
                    np.array([1.0, 1.1][:B]), np.array([1e-3, 1e-2][:B]))


@pytest.mark.parametrize("dims,T,sigma", [((2, 4099), 3, 1.5), ((3000, 3), 2, 2.0),
                                          ((2, 3, 700), 2, 1.0), ((500, 2, 3), 2, 1.0),
                                          ((3, 129, 2), 3, 1.2)])
def test_extreme_aspect_ratios(meta, dims, T, sigma):
    """Images 2-3 voxels wide along some axis and thousands long along another: the
    shortest blur tiles, marching kernels with fewer than 32 columns or 2 rows,
    pitch padding on narrow rows; forward and cost / gradient against the oracle."""
    B = 2
    I0, _ = phantoms.random_fields(141, B, dims)
    J, _ = phantoms.random_fields(142, B, dims)
    p0 = smooth_p(143, (B,) + dims, 20.0, s=1.0)
    check_forward(meta, I0, p0, T, sigma, [0.1, 0.0], [1.0, 1.3])
    check_cost_grad(meta, I0, J, p0, T, sigma, np.array([0.1, 0.0]), np.array([1.0, 1.3]),
                    np.array([1e-3, 1e-2]))


@pytest.mark.parametrize("dims,sigma", [
    ((6, 128), 7.0), ((5, 129), 8.5), ((7, 127), 7.0), ((3, 257), 8.5),   # x: 1 and 2-3 tiles
    ((129, 5), 7.0), ((128, 6), 8.5), ((257, 4), 7.0),                    # y: strided tiles
    ((5, 33, 129), 8.5), ((129, 6, 7), 7.0), ((33, 17, 20), 8.0),         # 3-D, z tiles
])
def test_tile_multiples_and_the_widest_compiled_tap_loops(meta, dims, sigma):
    """Extents at, one below and one above the 128-wide tiles of the blur passes, with
    sigma 7 to 8.5 (r = 21 to 26): the tap loops compiled for 6 and 7 chunks of 8 taps,
    whose halos are wider than most of these images.  Momenta move the feet 0.15 to 2.3
    voxels a step (in 3-D past the deterministic gather window, into the scatter
    fallback).  Forward and cost / gradient against the oracle (the FP32 torch
    re-implementation meets them within 3.4e-5 of the gradient bound's 1e-3)."""
    B = 2
    I0, _ = phantoms.random_fields(161, B, dims)
    J, _ = phantoms.random_fields(162, B, dims)
    p0 = smooth_p(163, (B,) + dims, 300.0 if len(dims) == 2 else 3000.0, s=1.2)
    check_forward(meta, I0, p0, 3, sigma, [0.002, 0.0], [1.0, 1.3])
    # lambda small enough that dL/dp0 is the adjoint's, not the regulariser's 2 lambda rho p0
    check_cost_grad(meta, I0, J, p0, 3, sigma, np.array([0.002, 0.0]), np.array([1.0, 1.3]),
                    np.array([1e-7, 1e-6]))


@pytest.mark.parametrize("dims,B,T,sigma,p_update", [
    ((21, 19), 3, 1, 1.5, "div"),       # a single step
    ((11, 12, 13), 2, 1, 1.0, "det"),   # a single 3-D step, det update
    ((17, 19), 40, 3, 1.2, "div"),      # many small instances in one launch (blockIdx.z)
    ((9, 10, 11), 24, 2, 0.3, "div"),   # the narrowest kernel: sigma 0.3, r = 1
    ((24, 30), 2, 64, 2.0, "det"),      # a long trajectory
])
def test_edge_cases_of_T_batch_and_sigma(meta, dims, B, T, sigma, p_update):
    I0, J = phantoms.random_fields(151, B, dims)
    p0 = smooth_p(152, (B,) + dims, 20.0 if len(dims) == 2 else 15.0, s=1.2)
    mu = np.linspace(0.0, 0.2, B).astype(np.float32)
    rho = np.linspace(0.8, 1.4, B).astype(np.float32)
    lam = np.full(B, 1e-3, np.float32)
    check_forward(meta, I0, p0, T, sigma, mu, rho, p_update=p_update)
    check_cost_grad(meta, I0, J, p0, T, sigma, mu, rho, lam, p_update=p_update)


def test_deformation_with_the_det_update(meta):
    I0, _ = phantoms.random_fields(153, 2, (30, 41))
    p0 = smooth_p(154, (2, 30, 41), 40.0, s=1.5)
    I1, p1, phi, jac, _ = meta.shoot_deform(cuda(I0), cuda(p0), 4, 2.0, [0.1, 0.0], 1.0,
                                            p_update="det")
    F1, q1, _ = meta.shoot_forward(cuda(I0), cuda(p0), 4, 2.0, [0.1, 0.0], 1.0, p_update="det")
    torch.cuda.synchronize()
    assert torch.equal(I1, F1) and torch.equal(p1, q1)
    for b, mu in enumerate((0.1, 0.0)):
        # the deformation integrates the v_t of the det-update shot: the oracle's shot
        # with the same update gives the same v_t
        It, pt, u = oracle.shoot(I0[b], p0[b], 4, 2.0, mu, 1.0, want_u=True, p_update="det")
        X = np.stack(np.meshgrid(np.arange(30.0), np.arange(41.0), indexing="ij"))
        ph = X.copy()
        for t in range(4):
            ph = np.stack([oracle.interp(ph[a], u[t] / 4.0) for a in range(2)])
        assert np.abs(phi.cpu().numpy()[b] - (ph - X)).max() <= FWD_ATOL * max(1.0, np.abs(ph - X).max())
        np.testing.assert_allclose(jac.cpu().numpy()[b], oracle.jacobian_det(ph), atol=JAC_ATOL)


@pytest.mark.parametrize("p_update,scheme", [("div", "sl"), ("det", "sl"), ("div", "hybrid")])
@pytest.mark.parametrize("dims,seed,scale,T,sigma,mu,rho,lam", [
    ((70, 33), 21, 200.0, 5, 3.0, 0.2, 0.8, 1e-2),     # per-step |d|: .2 1.6 4.3 8.1 17
    ((14, 16, 18), 31, 300.0, 4, 1.5, 0.1, 1.0, 1e-3),  # per-step |d|: .3 1.8 4.8 17
])
def test_large_displacements(meta, dims, seed, scale, T, sigma, mu, rho, lam, p_update, scheme):
    """Per-step displacements of 0.2 to 17 voxels: the gather window grows with
    them (R = 1 + floor(max|d|)) and, from 8 voxels in 2-D or 4 in 3-D on, the
    adjoint switches to the atomic scatter.  These inputs stay well conditioned
    in FP32 (an FP32 torch implementation of the same scheme is within 3e-5)."""
    I0, _ = phantoms.random_fields(seed, 1, dims)
    J, _ = phantoms.random_fields(seed + 1, 1, dims)
    p0 = smooth_p(seed + 2, (1,) + dims, scale)
    _, _, u = oracle.shoot(I0[0], p0[0], T, sigma, mu, rho, want_u=True, p_update=p_update,
                           scheme=scheme)
    per_step = [np.abs(u[k]).max() * rho / T for k in range(T)]
    assert max(per_step) > 9 and min(per_step) < 1
    check_cost_grad(meta, I0, J, p0, T, sigma, mu, rho, lam, p_update=p_update, scheme=scheme)
    assert check_cost_grad.status & 2  # the scatter fallback ran


@pytest.mark.parametrize("p_update,scheme", [("div", "sl"), ("det", "sl"), ("div", "hybrid")])
def test_3d_gather_window_up_to_four_voxels_is_deterministic(meta, p_update, scheme):
    """3-D per-step displacements 0.18, 0.67, 1.15, 1.88, 3.76 voxels (windows R = 1,
    1, 2, 2, 4): every step transposes the interpolation by the fixed-order gather (no
    scatter bit), the gradient meets the oracle, and two calls agree bit for bit."""
    dims, T, sigma, mu, rho, lam = (14, 16, 18), 5, 1.5, 0.1, 1.0, 1e-3
    I0, _ = phantoms.random_fields(31, 1, dims)
    J, _ = phantoms.random_fields(32, 1, dims)
    p0 = smooth_p(33, (1,) + dims, 220.0)
    _, _, u = oracle.shoot(I0[0], p0[0], T, sigma, mu, rho, want_u=True, p_update=p_update,
                           scheme=scheme)
    per_step = [np.abs(u[k]).max() * rho / T for k in range(T)]
    assert 3.0 < max(per_step) < 4.0 and min(per_step) < 1.0
    check_cost_grad(meta, I0, J, p0, T, sigma, mu, rho, lam, p_update=p_update, scheme=scheme)
    assert check_cost_grad.status & 2 == 0  # no step fell back to the scatter
    runs = [meta.cost_and_grad(cuda(I0), cuda(J), cuda(p0), T, sigma, mu, rho, lam,
                               p_update=p_update, scheme=scheme) for _ in range(2)]
    torch.cuda.synchronize()
    assert torch.equal(runs[0][0], runs[1][0]) and torch.equal(runs[0][1], runs[1][1])


def test_shoot_adjoint_and_autograd_function(meta):
    dims = (40, 45)
    B, T, sigma = 2, 4, 2.0
    mu, rho = [0.2, 0.0], [1.0, 1.4]
    I0, _ = phantoms.random_fields(51, B, dims)
    p0 = smooth_p(52, (B,) + dims, 50.0)
    r = np.random.default_rng(53)
    gI1 = r.normal(size=(B,) + dims).astype(np.float32)
    gp1 = r.normal(size=(B,) + dims).astype(np.float32)
    tI, tp = cuda(I0).requires_grad_(True), cuda(p0).requires_grad_(True)
    I1, p1 = meta.shoot(tI, tp, T, sigma, mu, rho)
    (I1 * cuda(gI1)).sum().add_((p1 * cuda(gp1)).sum()).backward()
    for b in range(B):
        gI0, gp0 = oracle.adjoint(I0[b], p0[b], gI1[b], gp1[b], T, sigma, mu[b], rho[b])
        assert rel_l2(tp.grad[b].cpu().numpy(), gp0) <= GRAD_RTOL
        assert rel_l2(tI.grad[b].cpu().numpy(), gI0) <= GRAD_RTOL


def test_plan_replays_the_recorded_call(meta):
    """meta_plan: a recorded cost_and_grad gives bit-identical results to the eager
    call, and picks up in-place updates of its inputs on every launch."""
    w = phantoms.disk_pair_64()
    plan = meta.CostAndGradPlan(cuda(w.I0), cuda(w.J), cuda(w.p0), w.T, w.sigma, w.mu, w.rho,
                                w.lam)
    for k in range(3):
        c1, g1 = plan.launch()
        c2, g2 = meta.cost_and_grad(plan.I0, plan.J, plan.p0, w.T, w.sigma, w.mu, w.rho, w.lam)
        torch.cuda.synchronize()
        assert torch.equal(c1, c2) and torch.equal(g1, g2)
        plan.p0.sub_(0.5 * g1 / g1.abs().max())  # a gradient-descent step in place
    assert plan.ws.status() == 0


@pytest.mark.parametrize("scheme", ["sl", "hybrid"])
@pytest.mark.parametrize("dims,B,T,sigma", [((45, 70), 5, 4, 2.5), ((10, 12, 14), 3, 3, 1.5)])
def test_batched_instances_equal_their_single_calls_bitwise(meta, dims, B, T, sigma, scheme):
    """Instances share every launch of a batch (one grid z index each) but nothing else:
    each one's I_T, p_T, cost and dL/dp0 are, bit for bit, what a call on it alone
    gives, with its own mu, rho, lambda and its own displacement window."""
    I0, _ = phantoms.random_fields(171, B, dims)
    J, _ = phantoms.random_fields(172, B, dims)
    p0 = smooth_p(173, (B,) + dims, 20.0 if len(dims) == 2 else 15.0, s=1.5)
    p0 *= np.linspace(0.2, 1.0, B, dtype=np.float32).reshape((B,) + (1,) * len(dims))
    mu = np.linspace(0.0, 0.2, B).astype(np.float32)
    rho = np.linspace(0.8, 1.3, B).astype(np.float32)
    lam = np.geomspace(1e-3, 1e-1, B).astype(np.float32)
    I1, p1, _ = meta.shoot_forward(cuda(I0), cuda(p0), T, sigma, mu, rho, scheme=scheme)
    c, g = meta.cost_and_grad(cuda(I0), cuda(J), cuda(p0), T, sigma, mu, rho, lam, scheme=scheme)
    for b in range(B):
        one = slice(b, b + 1)
        I1b, p1b, _ = meta.shoot_forward(cuda(I0[one]), cuda(p0[one]), T, sigma, mu[one], rho[one],
                                         scheme=scheme)
        cb, gb = meta.cost_and_grad(cuda(I0[one]), cuda(J[one]), cuda(p0[one]), T, sigma, mu[one],
                                    rho[one], lam[one], scheme=scheme)
        assert torch.equal(I1b[0], I1[b]) and torch.equal(p1b[0], p1[b]), b
        assert torch.equal(cb[0], c[b]) and torch.equal(gb[0], g[b]), b


def test_group_plan_runs_mixed_shapes_in_one_graph(meta):
    """Problems of different size, dimension, T and sigma recorded as parallel
    graph branches give what their separate calls give, bit for bit; one small
    member is also checked against the oracle."""
    specs = [((48, 52), 2, 5, 2.5, 0.1), ((33, 40), 1, 3, 4.0, 0.0), ((12, 14, 11), 1, 4, 1.5, 0.2),
             ((64, 64), 3, 6, 3.0, 0.05), ((9, 10, 12), 2, 2, 2.2, 0.1)]
    problems = []
    for k, (dims, B, T, sigma, mu) in enumerate(specs):
        I0, _ = phantoms.random_fields(70 + k, B, dims)
        J, _ = phantoms.random_fields(80 + k, B, dims)
        p0 = smooth_p(90 + k, (B,) + dims, 20.0, s=1.5)
        problems.append(dict(I0=cuda(I0), J=cuda(J), p0=cuda(p0), T=T, sigma=sigma, mu=mu,
                             rho=1.0, lam=1e-2))
    plan = meta.GroupPlan(problems, streams=3)
    plan.launch()
    torch.cuda.synchronize()
    for pb, it in zip(problems, plan.items):
        c, g = meta.cost_and_grad(pb["I0"], pb["J"], pb["p0"], pb["T"], pb["sigma"], pb["mu"],
                                  pb["rho"], pb["lam"])
        torch.cuda.synchronize()
        assert torch.equal(c, it["cost"]) and torch.equal(g, it["grad"])
    pb, it = problems[2], plan.items[2]
    c_ref, g_ref = oracle.cost_and_grad(pb["I0"][0].cpu().numpy(), pb["J"][0].cpu().numpy(),
                                        pb["p0"][0].cpu().numpy(), pb["T"], pb["sigma"],
                                        pb["mu"], 1.0, 1e-2)
    np.testing.assert_allclose(it["cost"][0].cpu().numpy(), c_ref, rtol=COST_RTOL)
    assert rel_l2(it["grad"][0].cpu().numpy(), g_ref) <= GRAD_RTOL


def test_variants_through_plans_and_lbfgs(meta):
    """The momentum update and the scheme reach every entry point: a group plan whose
    members use the det update, the Eulerian and the hybrid scheme gives what their
    separate calls give, bit for bit; a recorded plan of a hybrid call likewise; and
    two L-BFGS iterations with the Eulerian scheme follow the oracle's driver."""
    specs = [((40, 44), 2, 4, 2.0, "div", "sl"), ((36, 30), 1, 3, 1.5, "det", "sl"),
             ((10, 12, 11), 1, 3, 1.2, "div", "euler"), ((30, 34), 2, 4, 2.0, "div", "hybrid")]
    problems = []
    for k, (dims, B, T, sigma, pu, sch) in enumerate(specs):
        I0, J = phantoms.random_fields(160 + k, B, dims)
        p0 = smooth_p(170 + k, (B,) + dims, 25.0, s=1.5)
        problems.append(dict(I0=cuda(I0), J=cuda(J), p0=cuda(p0), T=T, sigma=sigma, mu=0.05,
                             rho=1.0, lam=1e-2, p_update=pu, scheme=sch))
    plan = meta.GroupPlan(problems, streams=2)
    plan.launch()
    torch.cuda.synchronize()
    for pb, it in zip(problems, plan.items):
        c, g = meta.cost_and_grad(pb["I0"], pb["J"], pb["p0"], pb["T"], pb["sigma"], pb["mu"],
                                  pb["rho"], pb["lam"], p_update=pb["p_update"],
                                  scheme=pb["scheme"])
        torch.cuda.synchronize()
        assert torch.equal(c, it["cost"]) and torch.equal(g, it["grad"])
    pb = problems[3]
    single = meta.CostAndGradPlan(pb["I0"], pb["J"], pb["p0"], pb["T"], pb["sigma"], pb["mu"],
                                  pb["rho"], pb["lam"], scheme="hybrid")
    single.launch()
    torch.cuda.synchronize()
    assert torch.equal(single.cost, plan.items[3]["cost"])
    assert torch.equal(single.grad, plan.items[3]["grad"])
    # L-BFGS with the Eulerian scheme on one 2-D pair
    I0, J = phantoms.random_fields(180, 1, (32, 36))
    p, hist, done = meta.lbfgs_minimize(cuda(I0), cuda(J), cuda(np.zeros_like(I0)), 4, 2.0, 0.05,
                                        1.0, 1e-3, iters=2, m=3, h0=0.5, scheme="euler")
    x, h_ref, margins = oracle.lbfgs_minimize(I0[0], J[0], np.zeros((32, 36)), 4, 2.0, 0.05, 1.0,
                                              1e-3, 2, 3, 0.5, scheme="euler")
    assert min(abs(v) for it in margins for v in it) > 1e-4
    np.testing.assert_allclose(hist[:, 0], h_ref, rtol=1e-4)
    assert rel_l2(p.cpu().numpy()[0], x) <= 1e-3


@pytest.mark.parametrize("dims,B,T,sigma,k", [((37, 141), 2, 7, 2.3, 2), ((37, 141), 2, 7, 2.3, 3),
                                              ((64, 64), 1, 10, 3.0, 5), ((12, 10, 11), 2, 6, 1.5, 4),
                                              ((70, 33), 1, 5, 3.0, 2)])
def test_step_checkpointing_gives_identical_results(meta, dims, B, T, sigma, k):
    """Keeping every k-th state and recomputing segments in the adjoint runs the same
    kernels on the same values: cost, gradient and shooting adjoint bit for bit."""
    I0, _ = phantoms.random_fields(101, B, dims)
    J, _ = phantoms.random_fields(102, B, dims)
    scale = 100.0 if dims == (70, 33) else 30.0  # the last case has 1-2 voxel steps (R = 2)
    p0 = smooth_p(103, (B,) + dims, scale)
    args = (T, sigma, [0.1, 0.0][:B], [1.0, 1.2][:B], [1e-2, 1e-3][:B])
    c1, g1 = meta.cost_and_grad(cuda(I0), cuda(J), cuda(p0), *args)
    c2, g2 = meta.cost_and_grad(cuda(I0), cuda(J), cuda(p0), *args, ckpt=k)
    torch.cuda.synchronize()
    assert torch.equal(c1, c2) and torch.equal(g1, g2)
    # the shooting map and its adjoint with checkpoints
    r = np.random.default_rng(104)
    gI1 = cuda(r.normal(size=(B,) + dims))
    I1a, p1a, wa = meta.shoot_forward(cuda(I0), cuda(p0), T, sigma, args[2], args[3])
    I1b, p1b, wb = meta.shoot_forward(cuda(I0), cuda(p0), T, sigma, args[2], args[3], ckpt=k)
    assert torch.equal(I1a, I1b) and torch.equal(p1a, p1b)
    ga = meta.shoot_adjoint(gI1, None, wa, T, sigma, args[2], args[3])
    gb = meta.shoot_adjoint(gI1, None, wb, T, sigma, args[2], args[3])
    assert torch.equal(ga[0], gb[0]) and torch.equal(ga[1], gb[1])
    gc = meta.shoot_adjoint(gI1, None, wb, T, sigma, args[2], args[3])  # again, same trajectory
    assert torch.equal(ga[0], gc[0]) and torch.equal(ga[1], gc[1])
    assert wb.nbytes < wa.nbytes


@pytest.mark.parametrize("dims,B,T,sigma,k,scale", [((37, 141), 2, 5, 2.3, 0, 30.0),
                                                    ((70, 33), 1, 5, 3.0, 2, 100.0),
                                                    ((12, 10, 11), 2, 4, 1.5, 0, 30.0),
                                                    ((13, 9, 22), 1, 6, 1.5, 3, 30.0)])
def test_workspace_contents_do_not_matter(meta, dims, B, T, sigma, k, scale):
    """Only the first 16 bytes of a workspace need zeroing: one whose other bytes
    are all 0xFF (NaN as floats) gives the same results bit for bit, so nothing
    reads memory (pitch padding included) before the library wrote it."""
    I0, _ = phantoms.random_fields(111, B, dims)
    J, _ = phantoms.random_fields(112, B, dims)
    p0 = smooth_p(113, (B,) + dims, scale)
    args = (T, sigma, [0.1, 0.0][:B], [1.0, 1.2][:B], [1e-2, 1e-3][:B])
    w0 = meta.Workspace(dims, B, T, sigma, "cuda", k)
    wn = meta.Workspace(dims, B, T, sigma, "cuda", k)
    wn.buf.fill_(255)
    wn.buf[:16].zero_()
    c0, g0 = meta.cost_and_grad(cuda(I0), cuda(J), cuda(p0), *args, workspace=w0, ckpt=k)
    cn, gn = meta.cost_and_grad(cuda(I0), cuda(J), cuda(p0), *args, workspace=wn, ckpt=k)
    torch.cuda.synchronize()
    assert torch.isfinite(g0).all()
    assert torch.equal(c0, cn) and torch.equal(g0, gn)


@pytest.mark.parametrize("dims,B,T,sigma", [((37, 141), 2, 5, 2.3), ((21, 45, 70), 2, 4, 2.0)])
def test_tile_shapes_and_autotuner_do_not_change_results(meta, dims, B, T, sigma):
    """Every output is summed in the same order whatever the tiles: explicit odd
    tile shapes and the autotuner's choice give the built-in results bit for bit."""
    I0, _ = phantoms.random_fields(121, B, dims)
    J, _ = phantoms.random_fields(122, B, dims)
    p0 = smooth_p(123, (B,) + dims, 30.0)
    args = (T, sigma, [0.1, 0.0][:B], [1.0, 1.2][:B], [1e-2, 1e-3][:B])
    meta.set_tuning(dims, B, sigma, None)
    c0, g0 = meta.cost_and_grad(cuda(I0), cuda(J), cuda(p0), *args)
    odd = dict(ly=16, txw=8) if len(dims) == 2 else dict(zc_transport=1, zc_advect=3, ly=16,
                                                         lz=16, txw=24)
    meta.set_tuning(dims, B, sigma, odd)
    c1, g1 = meta.cost_and_grad(cuda(I0), cuda(J), cuda(p0), *args)
    # one x tile over the whole row (144 or 72 wide: 18 or 9 threads per row, padded to
    # 20 or 12, the staged row up to the 256-float TMA box)
    meta.set_tuning(dims, B, sigma, dict(txw=144) if len(dims) == 2 else dict(txw=72))
    c3, g3 = meta.cost_and_grad(cuda(I0), cuda(J), cuda(p0), *args)
    # strided tiles longer than the extent (192 and 160 outputs, most of their groups
    # past the volume) and short ones (32)
    meta.set_tuning(dims, B, sigma, dict(ly=192) if len(dims) == 2 else dict(ly=192, lz=160))
    c4, g4 = meta.cost_and_grad(cuda(I0), cuda(J), cuda(p0), *args)
    meta.set_tuning(dims, B, sigma, dict(ly=32) if len(dims) == 2 else dict(ly=32, lz=32))
    c5, g5 = meta.cost_and_grad(cuda(I0), cuda(J), cuda(p0), *args)
    chosen = meta.autotune(cuda(I0), cuda(J), cuda(p0), *args)
    assert meta.tuning(dims, B, sigma) == chosen
    c2, g2 = meta.cost_and_grad(cuda(I0), cuda(J), cuda(p0), *args)
    # a plan that records the batch as two sub-batches on parallel graph branches
    meta.set_tuning(dims, B, sigma, dict(odd, split=2))
    plan = meta.CostAndGradPlan(cuda(I0), cuda(J), cuda(p0), *args)
    plan.launch()
    meta.set_tuning(dims, B, sigma, None)
    torch.cuda.synchronize()
    assert torch.equal(c0, c1) and torch.equal(g0, g1)
    assert torch.equal(c0, c2) and torch.equal(g0, g2)
    assert torch.equal(c0, c3) and torch.equal(g0, g3)
    assert torch.equal(c0, c4) and torch.equal(g0, g4)
    assert torch.equal(c0, c5) and torch.equal(g0, g5)
    assert torch.equal(c0, plan.cost) and torch.equal(g0, plan.grad)
    assert plan.ws.status() & 1 == 0


def test_device_wait_timeout_is_reported_and_cleared(meta):
    """Failure detection without a fault: a bounded device wait that nothing
    satisfies runs out (50 ms), latches the timeout bit, the status call reports
    it, and after clearing it the same workspace runs a call normally."""
    dims, B, T, sigma = (37, 45), 1, 3, 2.0
    ws = meta.Workspace(dims, B, T, sigma)
    assert ws.status(clear=True) == 0
    ws.selftest_timeout(50_000_000)
    assert ws.status() & 1 == 1
    lib = meta._load()
    bits = ctypes.c_uint(0)
    rc = lib.meta_workspace_status(ctypes.c_void_p(ws.ptr()), ws.nbytes, 1,
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                   ctypes.byref(bits))
    assert rc == 5 and bits.value & 1  # META_ERR_TIMEOUT, then cleared
    assert ws.status() == 0
    I0, _ = phantoms.random_fields(131, B, dims)
    J, _ = phantoms.random_fields(132, B, dims)
    c, g = meta.cost_and_grad(cuda(I0), cuda(J), cuda(np.zeros((B,) + dims)), T, sigma, 0.1, 1.0,
                              1e-3, workspace=ws)
    torch.cuda.synchronize()
    assert ws.status() == 0 and torch.isfinite(g).all()
    with pytest.raises(meta.MetaError):
        ws.selftest_timeout(10)  # below the 1 ms floor


def test_results_are_deterministic(meta):
    w = phantoms.disk_pair_64()
    a = meta.cost_and_grad(cuda(w.I0), cuda(w.J), cuda(w.p0), w.T, w.sigma, w.mu, w.rho, w.lam)
    b = meta.cost_and_grad(cuda(w.I0), cuda(w.J), cuda(w.p0), w.T, w.sigma, w.mu, w.rho, w.lam)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


# ----------------------------------------------------------------- workload sizes

def test_ellipse_batch_16x256_full_size(meta):
    """The 16 x 256^2, T=20, sigma=6 batch (mu in {0, 0.05, 0.2}) at two momenta."""
    w = phantoms.ellipse_pairs()
    oracle.set_threads(oracle.max_threads())
    check_cost_grad(meta, w.I0, w.J, w.p0, w.T, w.sigma, w.mu, w.rho, w.lam)
    p0 = smooth_p(61, w.p0.shape, 2.0, s=4.0)
    check_cost_grad(meta, w.I0, w.J, p0, w.T, w.sigma, w.mu, w.rho, w.lam)


def test_det_update_and_deformation_at_the_batch_size(meta):
    """The 16 x 256^2 batch (T = 20, sigma 6, mu = 0) at a momentum that moves feet by up
    to 0.7 voxel a step, with the det momentum update: cost and dL/dp0 of instances 0 and
    3 against the oracle (the GPU runs the whole batch; there the two updates differ by
    0.4 and 5.5 in p_T, and an FP32 torch run of the scheme is within 5e-8 of the oracle),
    and the deformation of instance 2 against the oracle's."""
    w = phantoms.ellipse_pairs()
    p0 = smooth_p(65, w.p0.shape, 1500.0, s=4.0)
    cost, grad = meta.cost_and_grad(cuda(w.I0), cuda(w.J), cuda(p0), w.T, w.sigma, 0.0, w.rho,
                                    w.lam, p_update="det")
    cost, grad = cost.cpu().numpy(), grad.cpu().numpy()
    for b in (0, 3):
        c, g = oracle.cost_and_grad(w.I0[b], w.J[b], p0[b], w.T, w.sigma, 0.0,
                                    float(w.rho[b]), float(w.lam[b]), p_update="det")
        np.testing.assert_allclose(cost[b], c, rtol=COST_RTOL, atol=1e-12)
        assert rel_l2(grad[b], g) <= GRAD_RTOL, b
    _, _, phi, jac, _ = meta.shoot_deform(cuda(w.I0), cuda(p0), w.T, w.sigma, 0.0, w.rho)
    wr, Jr = oracle.deformation(w.I0[2], p0[2], w.T, w.sigma, 0.0, float(w.rho[2]))
    assert np.abs(phi.cpu().numpy()[2] - wr).max() <= FWD_ATOL * max(1.0, np.abs(wr).max())
    assert np.abs(jac.cpu().numpy()[2] - Jr).max() <= JAC_ATOL * max(1.0, np.abs(wr).max())
    assert np.abs(wr).max() > 1.0


def test_head_128_full_size(meta):
    """128^3, T=20, sigma=5 head phantom: cost and gradient at a smooth momentum,
    with a checkpoint every 5 steps (the workload's configuration) and without."""
    w = phantoms.head_pair_3d()
    oracle.set_threads(oracle.max_threads())
    p0 = smooth_p(62, w.p0.shape, 3.0, s=3.0)
    check_cost_grad(meta, w.I0, w.J, p0, w.T, w.sigma, w.mu, w.rho, w.lam, ckpt=5)
    c5, g5 = meta.cost_and_grad(cuda(w.I0), cuda(w.J), cuda(p0), w.T, w.sigma, w.mu, w.rho,
                                w.lam, ckpt=5)
    c0, g0 = meta.cost_and_grad(cuda(w.I0), cuda(w.J), cuda(p0), w.T, w.sigma, w.mu, w.rho,
                                w.lam)
    torch.cuda.synchronize()
    assert torch.equal(c5, c0) and torch.equal(g5, g0)


def test_mri_160_full_size_against_the_oracle(meta):
    """160 x 192 x 160, T = 20, sigma 6, mu 0.05, lambda 1e-4 with a checkpoint every 5
    steps (the benchmark's configuration): the whole cost and dL/dp0 against the FP64
    oracle at full size (about a minute of the host's cores), at a momentum that moves
    feet by about 0.2 voxel a step (an FP32 torch run of the scheme on the central
    80 x 96 x 80 block is within 2e-5 of the oracle there)."""
    w = phantoms.mri_pair_3d()
    oracle.set_threads(oracle.max_threads())
    p0 = smooth_p(66, w.I0.shape, 1000.0, s=3.0)
    check_cost_grad(meta, w.I0, w.J, p0, w.T, w.sigma, w.mu, w.rho, w.lam, ckpt=5)


def test_gradient_descent_follows_torch_autograd(meta):
    """Gradient descent on p0 driven by the hand-written adjoint and by torch.autograd
    through the same scheme in PyTorch ops (FP32, same GPU) follows the same path:
    40 normalised steps on four 64^2 pairs, costs and iterates compared along the way.
    The descent starts from a smooth p0 whose per-step displacements (about 0.01 to 0.1
    voxel) are far above FP32 rounding of a coordinate: near p0 = 0 the feet sit within
    rounding of the grid lines, where torch (absolute coordinates, rounded onto the
    node) and the kernels (relative feet, which keep the side of the node the foot is
    on, as the FP64 oracle does) take different one-sided derivatives.  The kernels'
    gradient at the final iterate is checked against the FP64 oracle."""
    ts = pytest.importorskip("baseline.torch_scheme")
    w = phantoms.ellipse_pairs(batch=4, size=(64, 64), T=10, sigma=3.0, seed=2024)
    I0, J = cuda(w.I0), cuda(w.J)
    mu, rho, lam = cuda(w.mu), cuda(w.rho), cuda(w.lam)
    start = cuda(smooth_p(125, w.I0.shape, 20.0, s=3.0))
    pa, pb = start.clone(), start.clone()
    for it in range(40):
        ca, ga = meta.cost_and_grad(I0, J, pa, w.T, w.sigma, mu, rho, lam)
        cb, gb = ts.cost_and_grad(I0, J, pb, w.T, w.sigma, mu, rho, lam)
        if it % 10 == 0 or it == 39:
            np.testing.assert_allclose(ca.sum(1).cpu().numpy(), cb.sum(1).double().cpu().numpy(),
                                       rtol=1e-4)
            assert rel_l2(pa.cpu().numpy(), pb.cpu().numpy()) <= 1e-3, it
        for p, g in ((pa, ga), (pb, gb)):
            gmax = g.abs().amax(dim=(1, 2), keepdim=True).clamp_min(1e-30)
            p.sub_(0.05 * g / gmax)
    c_start = meta.cost_and_grad(I0, J, start, w.T, w.sigma, mu, rho, lam)[0].sum(1)
    assert (ca.sum(1) < c_start).all()
    check_cost_grad(meta, w.I0, w.J, pa.cpu().numpy(), w.T, w.sigma, w.mu, w.rho, w.lam)


def test_mri_registration_parity_along_gradient_descent(meta):
    """The 160x192x160 pipeline on its 2x block-averaged copy (80x96x80, sigma 3,
    checkpoint stride 5): 100 gradient-descent iterations of a recorded plan on the
    GPU; cost and dL/dp0 against the oracle at iterations 0, 10 and 100, on the
    GPU's own p0 iterates; the data term decreases."""
    w = phantoms.mri_pair_3d()
    I0s, Js = phantoms.block_average(w.I0), phantoms.block_average(w.J)
    sigma = w.sigma / 2
    mu, rho, lam = float(w.mu[0]), float(w.rho[0]), float(w.lam[0])
    plan = meta.CostAndGradPlan(cuda(I0s), cuda(Js), cuda(np.zeros_like(I0s)), w.T, sigma, mu,
                                rho, lam, ckpt=5)
    oracle.set_threads(oracle.max_threads())
    data = []
    for it in range(101):
        plan.launch()
        if it in (0, 10, 100):
            torch.cuda.synchronize()
            p_it = plan.p0.cpu().numpy()[0].astype(np.float64)
            c, g = oracle.cost_and_grad(I0s[0], Js[0], p_it, w.T, sigma, mu, rho, lam)
            np.testing.assert_allclose(plan.cost.cpu().numpy()[0], c, rtol=COST_RTOL, atol=1e-12)
            e = rel_l2(plan.grad.cpu().numpy()[0], g)
            assert e <= GRAD_RTOL, (it, e)
            data.append(float(c[0]))
        # normalised gradient step (the bench's update)
        gmax = plan.grad.abs().max().clamp_min(1e-30)
        plan.p0.sub_(0.02 * plan.grad / gmax)
    assert plan.ws.status() & 1 == 0
    assert data[1] < data[0] and data[2] < data[0], data


def test_mri_volume_downsampled_and_full_size_properties(meta):
    """160x192x160 (sigma 6): parity on the 2x block-averaged copy (sigma 3) and,
    at full size, the p0 = 0 invariance and the rho-rescaling identity."""
    w = phantoms.mri_pair_3d()
    I0s, Js = phantoms.block_average(w.I0), phantoms.block_average(w.J)
    p0s = smooth_p(63, I0s.shape, 3.0, s=2.0)
    oracle.set_threads(oracle.max_threads())
    check_cost_grad(meta, I0s, Js, p0s, w.T, w.sigma / 2, w.mu, w.rho, w.lam)
    # full size: p0 = 0 leaves the image unchanged bit for bit
    I1, p1, _ = meta.shoot_forward(cuda(w.I0), cuda(w.p0), w.T, w.sigma, w.mu, w.rho)
    assert torch.equal(I1.cpu(), torch.from_numpy(w.I0)) and bool((p1 == 0).all())
    # full size: (rho, mu, p0) and (1, mu/rho, rho p0) shoot to the same image
    p0 = smooth_p(64, w.I0.shape, 3.0, s=3.0)
    A = meta.shoot_forward(cuda(w.I0), cuda(p0), w.T, w.sigma, 0.1, 2.0)[0]
    B = meta.shoot_forward(cuda(w.I0), cuda(2.0 * p0), w.T, w.sigma, 0.05, 1.0)[0]
    assert float((A - B).abs().max()) <= FWD_ATOL
