"""The same semi-Lagrangian Metamorphosis scheme written with stock PyTorch ops.

This is the comparator the GPU library is measured against ("torch.autograd
through the same scheme"), and, run in FP64 on the CPU, an independent
re-implementation that cross-checks the oracle's conventions: it uses
``F.grid_sample`` (bilinear/trilinear, border padding, align_corners=True) for
the backtracking interpolation, grouped ``conv`` with zero padding for the
Gaussian RKHS kernel, slicing of a replicate-padded tensor for central
differences, and torch.autograd for dL/dp0.  It shares no code with the
oracle or with the CUDA library.

Scheme (Eq. 3 in the semi-Lagrangian form of Sec. 2.3; cost Eq. 4):
    v = -rho K*(p grad I);  y = x - dt v;  I~ = I(y), p~ = p(y);
    p' = p~ (1 - dt div v);  I' = I~ + dt mu p~;
    L = 1/2 |I_T - J|^2 + lambda [ <m0, K m0> + rho |p0|^2 ],  m0 = p0 grad I_0.
With p_update = "det" the momentum update is p' = p~ det(Id - dt Dv), Dv_ae = D_e v_a,
the determinant taken by torch.linalg.det.  scheme = "euler" integrates Eq. 5 and the
conservative Eq. 7 by explicit Euler steps, I' = I - dt <grad I, v> + dt mu p and
p' = p - dt div(p v); scheme = "hybrid" keeps the semi-Lagrangian I' and takes that p'.
"""
from __future__ import annotations

import math
from typing import Sequence, Tuple

import torch
import torch.nn.functional as F


def gaussian_taps(sigma: float, dtype=torch.float32, device="cpu") -> torch.Tensor:
    r = int(math.ceil(3.0 * sigma))
    k = torch.arange(-r, r + 1, dtype=torch.float64)
    w = torch.exp(-(k * k) / (2.0 * sigma * sigma))
    return (w / w.sum()).to(dtype=dtype, device=device)


def _conv_axis(f: torch.Tensor, w: torch.Tensor, axis: int, nd: int) -> torch.Tensor:
    """1-D zero-padded correlation of every channel of f [B, C, *dims] along spatial axis."""
    C = f.shape[1]
    K = w.numel()
    shape = [1] * nd
    shape[axis] = K
    weight = w.reshape(1, 1, *shape).expand(C, 1, *shape).contiguous()
    pad = [0] * nd
    pad[axis] = K // 2
    conv = F.conv2d if nd == 2 else F.conv3d
    return conv(f, weight, padding=tuple(pad), groups=C)


def blur(f: torch.Tensor, w: torch.Tensor) -> torch.Tensor:
    nd = f.dim() - 2
    for axis in reversed(range(nd)):
        f = _conv_axis(f, w, axis, nd)
    return f


def central_diff(f: torch.Tensor) -> torch.Tensor:
    """[B, *dims] -> [B, nd, *dims]; (f[x+1]-f[x-1])/2 with replicated edges."""
    nd = f.dim() - 1
    fp = F.pad(f.unsqueeze(1), [1, 1] * nd, mode="replicate").squeeze(1)
    out = []
    for a in range(nd):
        hi = [slice(None)] + [slice(1, -1)] * nd
        lo = [slice(None)] + [slice(1, -1)] * nd
        hi[1 + a] = slice(2, None)
        lo[1 + a] = slice(0, -2)
        out.append(0.5 * (fp[tuple(hi)] - fp[tuple(lo)]))
    return torch.stack(out, 1)


def divergence(v: torch.Tensor) -> torch.Tensor:
    """[B, nd, *dims] -> [B, *dims]."""
    nd = v.shape[1]
    return sum(central_diff(v[:, a])[:, a] for a in range(nd))


def _identity_grid(dims: Sequence[int], dtype, device) -> torch.Tensor:
    axes = [torch.arange(n, dtype=dtype, device=device) for n in dims]
    return torch.stack(torch.meshgrid(*axes, indexing="ij"), 0)  # [nd, *dims]


def sample(fields: torch.Tensor, feet: torch.Tensor) -> torch.Tensor:
    """fields [B, C, *dims]; feet [B, nd, *dims] in voxel units (axis 0 first)."""
    dims = fields.shape[2:]
    nd = len(dims)
    norm = [2.0 * feet[:, a] / (dims[a] - 1) - 1.0 for a in range(nd)]
    grid = torch.stack(norm[::-1], -1)  # grid_sample wants (x, y[, z]) = last axis first
    return F.grid_sample(fields, grid, mode="bilinear", padding_mode="border",
                         align_corners=True)


def jacobian_factor(v: torch.Tensor, dt: float) -> torch.Tensor:
    """det(Id - dt Dv) for v [B, nd, *dims], Dv_ae = D_e v_a: [B, *dims]."""
    nd = v.shape[1]
    Dv = torch.stack([central_diff(v[:, a]) for a in range(nd)], 1)  # [B, a, e, *dims]
    eye = torch.eye(nd, dtype=v.dtype, device=v.device).reshape(1, nd, nd, *([1] * nd))
    M = (eye - dt * Dv).movedim(1, -1).movedim(1, -1)  # [B, *dims, a, e]
    return torch.linalg.det(M)


def shoot(I0: torch.Tensor, p0: torch.Tensor, T: int, sigma: float, mu: torch.Tensor,
          rho: torch.Tensor, keep: bool = False, p_update="div", scheme: str = "sl"):
    """I0, p0 [B, *dims]; mu, rho [B].  Returns (I_T, p_T, v_0[, trajectory])."""
    B, dims = I0.shape[0], I0.shape[1:]
    nd = len(dims)
    bshape = (B,) + (1,) * nd
    w = gaussian_taps(sigma, I0.dtype, I0.device)
    dt = 1.0 / T
    x = _identity_grid(dims, I0.dtype, I0.device).unsqueeze(0)
    I, p = I0, p0
    traj = [(I, p)]
    v0 = None
    mu_b, rho_b = mu.reshape(bshape), rho.reshape(bshape)
    for _ in range(T):
        g = central_diff(I)                                  # [B, nd, *dims]
        u = blur(p.unsqueeze(1) * g, w)                      # K (p grad I)
        v = -rho_b.unsqueeze(1) * u
        if v0 is None:
            v0 = u
        if scheme == "euler":
            I, p = I - dt * (g * v).sum(1) + dt * mu_b * p, p - dt * divergence(p.unsqueeze(1) * v)
        else:
            Ip = sample(torch.stack([I, p], 1), x - dt * v)
            It, pt = Ip[:, 0], Ip[:, 1]
            if scheme == "hybrid":
                p = p - dt * divergence(p.unsqueeze(1) * v)
            elif p_update in ("det", 1):
                p = pt * jacobian_factor(v, dt)
            else:
                p = pt * (1.0 - dt * divergence(v))
            I = It + dt * mu_b * pt
        if keep:
            traj.append((I, p))
    return (I, p, v0, traj) if keep else (I, p, v0)


def cost(I0, J, p0, T, sigma, mu, rho, lam, p_update="div", scheme="sl") -> torch.Tensor:
    """[B, 3]: data, lambda*kinetic, lambda*rho*residual (Eq. 4)."""
    B, nd = I0.shape[0], I0.dim() - 1
    IT, _, u0 = shoot(I0, p0, T, sigma, mu, rho, p_update=p_update, scheme=scheme)
    m0 = p0.unsqueeze(1) * central_diff(I0)
    red = tuple(range(1, nd + 1))
    data = 0.5 * ((IT - J) ** 2).sum(red)
    kin = (m0 * u0).sum(tuple(range(1, nd + 2)))
    res = (p0 ** 2).sum(red)
    return torch.stack([data, lam * kin, lam * rho * res], 1)


def cost_and_grad(I0, J, p0, T, sigma, mu, rho, lam, p_update="div",
                  scheme="sl") -> Tuple[torch.Tensor, torch.Tensor]:
    """Cost [B, 3] and dL/dp0 [B, *dims] by torch.autograd."""
    p = p0.detach().clone().requires_grad_(True)
    c = cost(I0, J, p, T, sigma, mu, rho, lam, p_update, scheme)
    (g,) = torch.autograd.grad(c.sum(), p)
    return c.detach(), g
