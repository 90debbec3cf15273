"""Python binding of the sm_103a semi-Lagrangian Metamorphosis / LDDMM library.

Thin argument marshalling over the C ABI of ``include/meta.h`` (ctypes): every
step of the shooting, the cost and the adjoint runs in the library's CUDA
kernels.  PyTorch supplies device memory (tensors, the workspace) and the
current stream only.  There is no CPU fallback: if ``libmeta.so`` is missing
or no CUDA device is present, every call raises.

Method: François, Gori, Glaunès, "Metamorphic image registration using a
semi-Lagrangian scheme", arXiv:2106.08817 (Eq. 3 shooting in the
semi-Lagrangian form of Sec. 2.3; Eq. 4 cost; its gradient w.r.t. p0).

Arrays are float32 [B, (D,) H, W] (a single instance may omit B); mu, rho and
lam are scalars or per-instance sequences / tensors.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence, Tuple, Union

import numpy as np
import torch

__all__ = ["workspace_size", "Workspace", "shoot_forward", "shoot_deform", "shoot_adjoint",
           "cost_and_grad", "Shoot", "shoot", "library_path", "STATUS", "timer_start",
           "timer_stop", "KERNEL_CLASSES", "CostAndGradPlan", "GroupPlan", "SCHEMES",
           "lbfgs_workspace_size", "lbfgs_direction", "lbfgs_minimize", "clear_workspaces",
           "cost_and_grad_noalloc", "noalloc_status", "noalloc_selftest_timeout",
           "tuning", "set_tuning", "autotune", "tuning_save", "tuning_load", "tuning_cache",
           "trace", "gd_minimize", "Registration"]

KERNEL_CLASSES = ("pack", "xpass_m", "strided_fwd", "advect", "cost", "adj_init", "adj_pre",
                  "adj_gather", "xpass_adj", "strided_adj", "adj_gradp", "unpack", "deform",
                  "deform_out", "adj_jac", "euler")
# kernels launched per timed scope of each class (the cost scope launches three)
_LAUNCHES_PER_SCOPE = {"cost": 3}

_HERE = os.path.dirname(os.path.abspath(__file__))
# META_LIB=check loads the bounds-checked debug build (_build.build(check=True))
_LIB_PATH = os.path.join(_HERE, "libmeta_check.so" if os.environ.get("META_LIB") == "check"
                         else "libmeta.so")
_lib = None

STATUS = {0: "ok", 1: "invalid argument", 2: "unsupported shape", 3: "workspace",
          4: "CUDA error", 5: "device-side wait timed out", 6: "non-finite",
          7: "unsupported device or driver", 8: "malformed or mismatched saved state",
          9: "file I/O error"}
_TRACE_FN = ctypes.CFUNCTYPE(None, ctypes.c_char_p, ctypes.c_int, ctypes.c_void_p)


class MetaError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__("%s failed: %s (status %d)" % (what, STATUS.get(code, "?"), code))
        self.code = code


class _Problem(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("dims", ctypes.c_int * 3), ("batch", ctypes.c_int),
                ("T", ctypes.c_int), ("sigma", ctypes.c_float), ("ckpt_stride", ctypes.c_int),
                ("p_update", ctypes.c_int), ("scheme", ctypes.c_int)]


class _Tuning(ctypes.Structure):
    _fields_ = [("zc_transport", ctypes.c_int), ("zc_advect", ctypes.c_int), ("ly", ctypes.c_int),
                ("lz", ctypes.c_int), ("txw", ctypes.c_int), ("split", ctypes.c_int)]


def library_path() -> str:
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError("libmeta.so is not built (run __graft_entry__.build() or "
                               "python paper_2106_08817_gb300/_build.py)")
        lib = ctypes.CDLL(_LIB_PATH)
        P, V, F, D = ctypes.POINTER(_Problem), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p
        S = ctypes.c_size_t
        lib.meta_workspace_size.argtypes = [P, ctypes.POINTER(S)]
        lib.meta_shoot_forward.argtypes = [P, F, F, F, F, F, F, V, S, V]
        lib.meta_shoot_deform.argtypes = [P, F, F, F, F, F, F, F, F, V, S, V]
        lib.meta_shoot_adjoint.argtypes = [P, F, F, F, F, F, F, V, S, V]
        lib.meta_cost_and_grad.argtypes = [P, F, F, F, F, F, F, D, F, V, S, V]
        lib.meta_plan_create.argtypes = [P, F, F, F, F, F, F, D, F, V, S,
                                         ctypes.POINTER(ctypes.c_void_p)]
        PP = ctypes.POINTER(ctypes.c_void_p)
        lib.meta_plan_create_group.argtypes = [ctypes.c_int, P, PP, PP, PP, PP, PP, PP, PP, PP,
                                               PP, ctypes.POINTER(S), ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_void_p)]
        lib.meta_plan_create_group.restype = ctypes.c_int
        lib.meta_plan_create_persistent.argtypes = [ctypes.c_int, P, PP, PP, PP, PP, PP, PP, PP,
                                                    PP, PP, ctypes.POINTER(S),
                                                    ctypes.POINTER(ctypes.c_void_p)]
        lib.meta_plan_create_persistent.restype = ctypes.c_int
        lib.meta_plan_status.argtypes = [V, ctypes.c_int, V, ctypes.POINTER(ctypes.c_uint)]
        lib.meta_plan_status.restype = ctypes.c_int
        lib.meta_plan_selftest_timeout.argtypes = [V, ctypes.c_int, ctypes.c_ulonglong, V]
        lib.meta_plan_selftest_timeout.restype = ctypes.c_int
        lib.meta_plan_launch.argtypes = [V, V]
        lib.meta_plan_destroy.argtypes = [V]
        for f in ("meta_plan_create", "meta_plan_launch", "meta_plan_destroy"):
            getattr(lib, f).restype = ctypes.c_int
        lib.meta_cost_and_grad_noalloc.argtypes = [P, F, F, F, F, F, F, D, F, V]
        lib.meta_cost_and_grad_noalloc.restype = ctypes.c_int
        lib.meta_noalloc_status.argtypes = [ctypes.c_int, V, ctypes.POINTER(ctypes.c_uint)]
        lib.meta_noalloc_status.restype = ctypes.c_int
        lib.meta_noalloc_selftest_timeout.argtypes = [ctypes.c_ulonglong, V]
        lib.meta_noalloc_selftest_timeout.restype = ctypes.c_int
        lib.meta_workspace_status.argtypes = [V, S, ctypes.c_int, V,
                                              ctypes.POINTER(ctypes.c_uint)]
        lib.meta_status_string.argtypes = [ctypes.c_int]
        lib.meta_status_string.restype = ctypes.c_char_p
        lib.meta_timer_start.argtypes = [ctypes.c_int]
        lib.meta_timer_stop.argtypes = [ctypes.POINTER(ctypes.c_float),
                                        ctypes.POINTER(ctypes.c_int)]
        lib.meta_selftest_timeout.argtypes = [V, S, ctypes.c_ulonglong, V]
        lib.meta_selftest_timeout.restype = ctypes.c_int
        T = ctypes.POINTER(_Tuning)
        lib.meta_autotune.argtypes = [P, F, F, F, F, F, F, D, F, V, S, V, T]
        lib.meta_tuning_get.argtypes = [P, T]
        lib.meta_tuning_set.argtypes = [P, T]
        for f in ("meta_autotune", "meta_tuning_get", "meta_tuning_set"):
            getattr(lib, f).restype = ctypes.c_int
        lib.meta_lbfgs_workspace_size.argtypes = [P, ctypes.c_int, ctypes.POINTER(S)]
        lib.meta_lbfgs_direction.argtypes = [P, ctypes.c_int, ctypes.c_int, PP, PP, F, F, V, S, V]
        lib.meta_lbfgs_minimize.argtypes = [P, F, F, F, F, F, F, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_float, V, S, V, S,
                                            ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_int), V]
        lib.meta_lbfgs_resume.argtypes = lib.meta_lbfgs_minimize.argtypes
        lib.meta_lbfgs_state_size.argtypes = [P, ctypes.c_int, ctypes.POINTER(S)]
        lib.meta_lbfgs_state_check.argtypes = [P, ctypes.c_int, V, S]
        lib.meta_lbfgs_state_save.argtypes = [P, ctypes.c_int, V, S, V, S, V]
        lib.meta_lbfgs_state_load.argtypes = [P, ctypes.c_int, V, S, V, S, V]
        lib.meta_gd_minimize.argtypes = [P, F, F, F, F, F, F, ctypes.c_int, ctypes.c_float, V, S,
                                         V, S, ctypes.POINTER(ctypes.c_double), V]
        for f in ("meta_lbfgs_workspace_size", "meta_lbfgs_direction", "meta_lbfgs_minimize",
                  "meta_lbfgs_resume", "meta_lbfgs_state_size", "meta_lbfgs_state_check",
                  "meta_lbfgs_state_save", "meta_lbfgs_state_load", "meta_gd_minimize"):
            getattr(lib, f).restype = ctypes.c_int
        CP = ctypes.c_char_p
        lib.meta_tuning_save.argtypes = [CP]
        lib.meta_tuning_load.argtypes = [CP, ctypes.POINTER(ctypes.c_int)]
        lib.meta_tuning_cache.argtypes = [CP, ctypes.POINTER(ctypes.c_int)]
        lib.meta_trace_set.argtypes = [_TRACE_FN, V]
        lib.meta_trace_selftest.argtypes = []
        for f in ("meta_tuning_save", "meta_tuning_load", "meta_tuning_cache", "meta_trace_set",
                  "meta_trace_selftest"):
            getattr(lib, f).restype = ctypes.c_int
        lib.meta_kernel_name.argtypes = [ctypes.c_int]
        lib.meta_kernel_name.restype = ctypes.c_char_p
        for f in ("meta_workspace_size", "meta_shoot_forward", "meta_shoot_deform",
                  "meta_shoot_adjoint",
                  "meta_cost_and_grad", "meta_workspace_status", "meta_timer_start",
                  "meta_timer_stop"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


P_UPDATES = {0: 0, 1: 1, "div": 0, "det": 1}


def _pupd(p_update) -> int:
    """Momentum update: 0 / "div" = p~ (1 - dt div v); 1 / "det" = p~ det(Id - dt Dv)."""
    if p_update not in P_UPDATES:
        raise ValueError("p_update must be 0, 1, 'div' or 'det' (got %r)" % (p_update,))
    return P_UPDATES[p_update]


SCHEMES = {"sl": 0, "euler": 1, "hybrid": 2}


def _scheme(scheme) -> int:
    """Integration scheme (Sec. 2.3): "sl" (the method), "euler" or "hybrid"; every call
    takes every scheme, and the adjoint is the exact transpose of the chosen one."""
    if scheme not in SCHEMES:
        raise ValueError("scheme must be 'sl', 'euler' or 'hybrid' (got %r)" % (scheme,))
    return SCHEMES[scheme]


def _problem(ndim: int, dims: Sequence[int], batch: int, T: int, sigma: float,
             ckpt: int = 0, p_update=0, scheme="sl") -> _Problem:
    d3 = list(dims) + [0] * (3 - len(dims))
    return _Problem(int(ndim), (ctypes.c_int * 3)(*d3), int(batch), int(T), float(sigma),
                    int(ckpt), _pupd(p_update), _scheme(scheme))


def workspace_size(dims: Sequence[int], batch: int, T: int, sigma: float, ckpt: int = 0,
                   scheme: str = "sl") -> int:
    """Workspace bytes; ckpt > 1 keeps every ckpt-th state and recomputes the rest."""
    n = ctypes.c_size_t(0)
    rc = _load().meta_workspace_size(
        ctypes.byref(_problem(len(dims), dims, batch, T, sigma, ckpt, 0, scheme)),
        ctypes.byref(n))
    if rc:
        raise MetaError(rc, "meta_workspace_size")
    return int(n.value)


class Workspace:
    """Device workspace (a zero-initialised uint8 tensor) of one problem shape.

    It keeps the trajectory of the last forward shooting; calls that share it
    must run on one stream.
    """

    def __init__(self, dims: Sequence[int], batch: int, T: int, sigma: float,
                 device: Union[torch.device, str, int] = "cuda", ckpt: int = 0,
                 scheme: str = "sl"):
        _scheme(scheme)
        self.key = (tuple(int(x) for x in dims), int(batch), int(T), float(sigma), int(ckpt),
                    scheme)
        self.ckpt = int(ckpt)
        self.scheme = scheme
        self.nbytes = workspace_size(dims, batch, T, sigma, ckpt, scheme)
        self.buf = torch.zeros(self.nbytes, dtype=torch.uint8, device=device)

    def matches(self, dims, batch, T, sigma, ckpt: int = 0, scheme: str = "sl") -> bool:
        return self.key == (tuple(int(x) for x in dims), int(batch), int(T), float(sigma),
                            int(ckpt), scheme)

    def ptr(self) -> int:
        return self.buf.data_ptr()

    def selftest_timeout(self, limit_ns: int = 50_000_000) -> None:
        """Enqueues a bounded device wait that runs out (meta_selftest_timeout): the
        timeout bit then shows in status()."""
        rc = _load().meta_selftest_timeout(ctypes.c_void_p(self.ptr()), self.nbytes,
                                           int(limit_ns), _stream(self.buf.device))
        if rc:
            raise MetaError(rc, "meta_selftest_timeout")

    def status(self, clear: bool = False) -> int:
        """Device fault bits latched since the last clear (synchronises the stream)."""
        bits = ctypes.c_uint(0)
        _load().meta_workspace_status(ctypes.c_void_p(self.ptr()), self.nbytes, int(clear),
                                      _stream(self.buf.device), ctypes.byref(bits))
        return int(bits.value)


def _stream(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _as_batch(x: torch.Tensor, name: str) -> Tuple[torch.Tensor, bool]:
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if x.dtype != torch.float32:
        raise TypeError("%s must be float32" % name)
    squeeze = False
    return x.contiguous(), squeeze


def _shape(I0: torch.Tensor, ndim: Optional[int]) -> Tuple[torch.Tensor, int, Tuple[int, ...], bool]:
    """Arrays are [B, *dims] (ndim = I0.dim() - 1 by default); with ndim = I0.dim()
    a single instance [*dims] is accepted and results drop the batch axis."""
    if ndim is None:
        ndim = I0.dim() - 1
    if ndim not in (2, 3):
        raise ValueError("ndim must be 2 or 3 (got array of rank %d)" % I0.dim())
    if I0.dim() == ndim:
        return I0.unsqueeze(0), ndim, tuple(I0.shape), True
    if I0.dim() == ndim + 1:
        return I0, ndim, tuple(I0.shape[1:]), False
    raise ValueError("expected [B, *dims] or [*dims] with ndim = %d" % ndim)


def _like(x: torch.Tensor, ref: torch.Tensor, name: str) -> torch.Tensor:
    """x with the shape of ref, [B, *dims], on ref's device: x must have that shape or,
    for B = 1, the shape [*dims].  Any other shape raises, even one with as many
    elements (transposed axes would otherwise be read silently in the wrong order)."""
    if x.device != ref.device:
        raise ValueError("%s is on %s, the images on %s" % (name, x.device, ref.device))
    shp, want = tuple(x.shape), tuple(ref.shape)
    if shp == want:
        return x
    if want[0] == 1 and shp == want[1:]:
        return x.reshape(want)
    raise ValueError("%s has shape %s where %s is expected" % (name, shp, want))


def _outputs(out, ref: torch.Tensor):
    """The caller's (cost, grad) for a batch shaped like ref: cost a contiguous float64
    [B, 3], grad None or a contiguous float32 array of ref's shape, both on ref's device
    (the kernels write them whole)."""
    cost, grad = out
    B = ref.shape[0]
    if not (isinstance(cost, torch.Tensor) and cost.dtype == torch.float64
            and tuple(cost.shape) == (B, 3) and cost.is_contiguous()
            and cost.device == ref.device):
        raise ValueError("out cost must be a contiguous float64 [%d, 3] tensor on %s"
                         % (B, ref.device))
    if grad is not None:
        if not (isinstance(grad, torch.Tensor) and grad.dtype == torch.float32
                and grad.is_contiguous()):
            raise ValueError("out grad must be a contiguous float32 tensor")
        _like(grad, ref, "out grad")
    return cost, grad


def _coef(v, B: int, device) -> torch.Tensor:
    t = torch.as_tensor(v, dtype=torch.float32, device=device).reshape(-1)
    if t.numel() == 1:
        t = t.expand(B)
    if t.numel() != B:
        raise ValueError("per-instance coefficient has %d values for batch %d" % (t.numel(), B))
    return t.contiguous()


def _p(t: Optional[torch.Tensor]) -> ctypes.c_void_p:
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


# Workspaces of the calls made without `workspace=`: one per (problem shape, device,
# stream), kept for reuse (each holds a whole trajectory) until clear_workspaces().
_ws_cache = {}


def clear_workspaces() -> None:
    """Drops the cached workspaces of calls made without `workspace=` (their device
    memory returns to torch's allocator once no plan or tensor refers to it)."""
    _ws_cache.clear()


def _workspace(dims, B, T, sigma, device, ws: Optional[Workspace], ckpt: int = 0,
               scheme: str = "sl") -> Workspace:
    if ws is not None:
        if not ws.matches(dims, B, T, sigma, ckpt, scheme):
            raise ValueError("workspace was made for another problem")
        if ws.buf.device != torch.device(device):
            raise ValueError("workspace is on %s, the images on %s" % (ws.buf.device, device))
        return ws
    key = (tuple(dims), B, T, float(sigma), int(ckpt), scheme, str(device),
           torch.cuda.current_stream(device).cuda_stream)
    w = _ws_cache.get(key)
    if w is None:
        w = Workspace(dims, B, T, sigma, device, ckpt, scheme)
        _ws_cache[key] = w
    return w


def shoot_forward(I0: torch.Tensor, p0: torch.Tensor, T: int, sigma: float, mu, rho=1.0,
                  workspace: Optional[Workspace] = None, ndim: Optional[int] = None,
                  ckpt: int = 0, p_update=0, scheme: str = "sl"
                  ) -> Tuple[torch.Tensor, torch.Tensor, Workspace]:
    """Geodesic shooting (Eq. 3, Sec. 2.3): returns (I_T, p_T, workspace with the trajectory).
    scheme "euler" / "hybrid": the other integration schemes of Sec. 2.3."""
    I0b, nd, dims, sq = _shape(_as_batch(I0, "I0")[0], ndim)
    p0b = _like(_as_batch(p0, "p0")[0], I0b, "p0")
    B, dev = I0b.shape[0], I0b.device
    ws = _workspace(dims, B, T, sigma, dev, workspace, ckpt, scheme)
    mu_t, rho_t = _coef(mu, B, dev), _coef(rho, B, dev)
    I1 = torch.empty_like(I0b)
    p1 = torch.empty_like(I0b)
    pr = _problem(nd, dims, B, T, sigma, ws.ckpt, p_update, scheme)
    rc = _load().meta_shoot_forward(ctypes.byref(pr), _p(I0b), _p(p0b), _p(mu_t), _p(rho_t),
                                    _p(I1), _p(p1), ctypes.c_void_p(ws.ptr()), ws.nbytes,
                                    _stream(dev))
    if rc:
        raise MetaError(rc, "meta_shoot_forward")
    if sq:
        I1, p1 = I1[0], p1[0]
    return I1, p1, ws


def shoot_deform(I0: torch.Tensor, p0: torch.Tensor, T: int, sigma: float, mu, rho=1.0,
                 workspace: Optional[Workspace] = None, ndim: Optional[int] = None,
                 ckpt: int = 0, want_phi: bool = True, want_jac: bool = True, p_update=0,
                 scheme: str = "sl") -> Tuple[torch.Tensor, torch.Tensor, Optional[torch.Tensor],
                            Optional[torch.Tensor], Workspace]:
    """Shooting with the deformation of the grid, phi_0 = Id, phi_{t+1} = phi_t o (Id - dt v_t):
    returns (I_T, p_T, phi_T - Id as [B, ndim, *dims] or None, det D phi_T or None,
    workspace with the trajectory)."""
    if not (want_phi or want_jac):
        raise ValueError("ask for phi, jac or both")
    I0b, nd, dims, sq = _shape(_as_batch(I0, "I0")[0], ndim)
    p0b = _like(_as_batch(p0, "p0")[0], I0b, "p0")
    B, dev = I0b.shape[0], I0b.device
    ws = _workspace(dims, B, T, sigma, dev, workspace, ckpt, scheme)
    mu_t, rho_t = _coef(mu, B, dev), _coef(rho, B, dev)
    I1 = torch.empty_like(I0b)
    p1 = torch.empty_like(I0b)
    phi = torch.empty((B, nd) + tuple(dims), dtype=torch.float32, device=dev) if want_phi else None
    jac = torch.empty_like(I0b) if want_jac else None
    pr = _problem(nd, dims, B, T, sigma, ws.ckpt, p_update, scheme)
    rc = _load().meta_shoot_deform(ctypes.byref(pr), _p(I0b), _p(p0b), _p(mu_t), _p(rho_t),
                                   _p(I1), _p(p1), _p(phi), _p(jac), ctypes.c_void_p(ws.ptr()),
                                   ws.nbytes, _stream(dev))
    if rc:
        raise MetaError(rc, "meta_shoot_deform")
    if sq:
        I1, p1 = I1[0], p1[0]
        phi = None if phi is None else phi[0]
        jac = None if jac is None else jac[0]
    return I1, p1, phi, jac, ws


def shoot_adjoint(gI1: torch.Tensor, gp1: Optional[torch.Tensor], workspace: Workspace, T: int,
                  sigma: float, mu, rho=1.0, want_gI0: bool = True, ndim: Optional[int] = None,
                  p_update=0, scheme: str = "sl") -> Tuple[Optional[torch.Tensor], torch.Tensor]:
    """Adjoint of the shooting map on the trajectory kept in `workspace` (shot with the
    same p_update and scheme): returns (dL/dI0 or None, dL/dp0) for dL/dI_T = gI1,
    dL/dp_T = gp1."""
    g1, nd, dims, sq = _shape(_as_batch(gI1, "gI1")[0], ndim)
    B, dev = g1.shape[0], g1.device
    if not workspace.matches(dims, B, T, sigma, workspace.ckpt, scheme):
        raise ValueError("workspace was made for another problem")
    if workspace.buf.device != dev:
        raise ValueError("workspace is on %s, the arrays on %s" % (workspace.buf.device, dev))
    gp1b = None if gp1 is None else _like(_as_batch(gp1, "gp1")[0], g1, "gp1")
    mu_t, rho_t = _coef(mu, B, dev), _coef(rho, B, dev)
    gp0 = torch.empty_like(g1)
    gI0 = torch.empty_like(g1) if want_gI0 else None
    pr = _problem(nd, dims, B, T, sigma, workspace.ckpt, p_update, scheme)
    rc = _load().meta_shoot_adjoint(ctypes.byref(pr), _p(mu_t), _p(rho_t), _p(g1), _p(gp1b),
                                    _p(gI0), _p(gp0), ctypes.c_void_p(workspace.ptr()),
                                    workspace.nbytes, _stream(dev))
    if rc:
        raise MetaError(rc, "meta_shoot_adjoint")
    if sq:
        gp0 = gp0[0]
        gI0 = None if gI0 is None else gI0[0]
    return gI0, gp0


def cost_and_grad(I0: torch.Tensor, J: torch.Tensor, p0: torch.Tensor, T: int, sigma: float,
                  mu, rho=1.0, lam=1e-3, want_grad: bool = True,
                  workspace: Optional[Workspace] = None, ndim: Optional[int] = None,
                  out: Optional[Tuple[torch.Tensor, torch.Tensor]] = None, ckpt: int = 0,
                  p_update=0, scheme: str = "sl") -> Tuple[torch.Tensor, Optional[torch.Tensor]]:
    """Eq. 4 cost per instance ([B, 3] float64: data, lambda*kinetic, lambda*rho*residual)
    and dL/dp0 ([B, *dims] float32) by the hand-written discrete adjoint.  p_update "det"
    shoots with p' = p~ det(Id - dt Dv) instead of p~ (1 - dt div v)."""
    I0b, nd, dims, sq = _shape(_as_batch(I0, "I0")[0], ndim)
    Jb = _like(_as_batch(J, "J")[0], I0b, "J")
    p0b = _like(_as_batch(p0, "p0")[0], I0b, "p0")
    B, dev = I0b.shape[0], I0b.device
    ws = _workspace(dims, B, T, sigma, dev, workspace, ckpt, scheme)
    mu_t, rho_t, lam_t = _coef(mu, B, dev), _coef(rho, B, dev), _coef(lam, B, dev)
    if out is not None:
        cost, grad = _outputs(out, I0b)
    else:
        cost = torch.empty((B, 3), dtype=torch.float64, device=dev)
        grad = torch.empty_like(I0b) if want_grad else None
    pr = _problem(nd, dims, B, T, sigma, ws.ckpt, p_update, scheme)
    rc = _load().meta_cost_and_grad(ctypes.byref(pr), _p(I0b), _p(Jb), _p(p0b), _p(mu_t),
                                    _p(rho_t), _p(lam_t), _p(cost), _p(grad),
                                    ctypes.c_void_p(ws.ptr()), ws.nbytes, _stream(dev))
    if rc:
        raise MetaError(rc, "meta_cost_and_grad")
    if sq and grad is not None and out is None:
        grad = grad[0]
    return cost, grad


TUNING_FIELDS = ("zc_transport", "zc_advect", "ly", "lz", "txw", "split")


def tuning(dims: Sequence[int], batch: int, sigma: float) -> dict:
    """Tile shapes that calls with this problem shape use (tuned, set or built-in)."""
    t = _Tuning()
    rc = _load().meta_tuning_get(ctypes.byref(_problem(len(dims), dims, batch, 1, sigma)),
                                 ctypes.byref(t))
    if rc:
        raise MetaError(rc, "meta_tuning_get")
    return {f: getattr(t, f) for f in TUNING_FIELDS}


def set_tuning(dims: Sequence[int], batch: int, sigma: float, tun: Optional[dict]) -> None:
    """Records tile shapes for the problem shape (None: back to the built-in choice)."""
    pr = _problem(len(dims), dims, batch, 1, sigma)
    if tun is None:
        rc = _load().meta_tuning_set(ctypes.byref(pr), None)
    else:
        t = _Tuning(*[int(tun.get(f, 0)) for f in TUNING_FIELDS])
        rc = _load().meta_tuning_set(ctypes.byref(pr), ctypes.byref(t))
    if rc:
        raise MetaError(rc, "meta_tuning_set")


def autotune(I0: torch.Tensor, J: torch.Tensor, p0: torch.Tensor, T: int, sigma: float, mu,
             rho=1.0, lam=1e-3, ndim: Optional[int] = None, ckpt: int = 0, p_update=0,
             scheme: str = "sl") -> dict:
    """Times cost_and_grad on these inputs for candidate tile shapes (meta_autotune),
    records the fastest for the problem shape and returns it.  Blocking."""
    I0b, nd, dims, _ = _shape(_as_batch(I0, "I0")[0], ndim)
    Jb = _like(_as_batch(J, "J")[0], I0b, "J")
    p0b = _like(_as_batch(p0, "p0")[0], I0b, "p0")
    B, dev = I0b.shape[0], I0b.device
    ws = _workspace(dims, B, T, sigma, dev, None, ckpt, scheme)
    mu_t, rho_t, lam_t = _coef(mu, B, dev), _coef(rho, B, dev), _coef(lam, B, dev)
    cost = torch.empty((B, 3), dtype=torch.float64, device=dev)
    grad = torch.empty_like(I0b)
    t = _Tuning()
    rc = _load().meta_autotune(ctypes.byref(_problem(nd, dims, B, T, sigma, ws.ckpt, p_update,
                                                     scheme)),
                               _p(I0b),
                               _p(Jb), _p(p0b), _p(mu_t), _p(rho_t), _p(lam_t), _p(cost),
                               _p(grad), ctypes.c_void_p(ws.ptr()), ws.nbytes, _stream(dev),
                               ctypes.byref(t))
    if rc:
        raise MetaError(rc, "meta_autotune")
    return {f: getattr(t, f) for f in TUNING_FIELDS}


def _path(path) -> bytes:
    return os.fsencode(os.fspath(path))


def tuning_save(path) -> None:
    """Writes every recorded tile shape of this process to a JSON file
    (meta_tuning_save)."""
    rc = _load().meta_tuning_save(_path(path))
    if rc:
        raise MetaError(rc, "meta_tuning_save")


def tuning_load(path) -> int:
    """Records the tile shapes of a JSON file written by tuning_save or by the
    autotuner's cache (meta_tuning_load); a malformed file is refused whole.
    Returns the number of entries."""
    n = ctypes.c_int(0)
    rc = _load().meta_tuning_load(_path(path), ctypes.byref(n))
    if rc:
        raise MetaError(rc, "meta_tuning_load")
    return int(n.value)


def tuning_cache(path) -> int:
    """Names the autotuner's cache file (None: none; meta_tuning_cache): shapes it
    holds are recorded now and not re-timed by autotune, new results are merged
    into it.  Returns the number of entries it held."""
    n = ctypes.c_int(0)
    rc = _load().meta_tuning_cache(None if path is None else _path(path), ctypes.byref(n))
    if rc:
        raise MetaError(rc, "meta_tuning_cache")
    return int(n.value)


class trace:
    """Context manager that collects the phase ranges the library pushes and pops
    (the same as its NVTX ranges; meta_trace_set) as (name, push) pairs::

        with meta.trace() as events:
            meta.cost_and_grad(...)
    """

    def __init__(self):
        self.events = []
        self._cb = _TRACE_FN(lambda name, push, user: self.events.append(
            (name.decode(), int(push))))

    def __enter__(self):
        rc = _load().meta_trace_set(self._cb, None)
        if rc:
            raise MetaError(rc, "meta_trace_set")
        return self.events

    def __exit__(self, *exc):
        _load().meta_trace_set(_TRACE_FN(), None)
        return False


def lbfgs_workspace_size(dims: Sequence[int], batch: int, m: int = 5) -> int:
    """Bytes of the L-BFGS workspace (m pairs) of a batch of this shape."""
    n = ctypes.c_size_t(0)
    rc = _load().meta_lbfgs_workspace_size(
        ctypes.byref(_problem(len(dims), dims, batch, 1, 1.0)), int(m), ctypes.byref(n))
    if rc:
        raise MetaError(rc, "meta_lbfgs_workspace_size")
    return int(n.value)


def lbfgs_direction(g: torch.Tensor, S: Sequence[torch.Tensor], Y: Sequence[torch.Tensor],
                    m: Optional[int] = None, ndim: Optional[int] = None) -> torch.Tensor:
    """d = -H g by the two-loop recursion over the pairs S[i], Y[i] (oldest first) of
    every instance (meta_lbfgs_direction)."""
    gb, nd, dims, sq = _shape(_as_batch(g, "g")[0], ndim)
    B, dev = gb.shape[0], gb.device
    if len(S) != len(Y):
        raise ValueError("%d s vectors but %d y vectors" % (len(S), len(Y)))
    m = int(m or max(1, len(S)))
    Sb = [_like(_as_batch(x, "s")[0], gb, "s") for x in S]
    Yb = [_like(_as_batch(x, "y")[0], gb, "y") for x in Y]
    arr = lambda ts: (ctypes.c_void_p * max(1, len(ts)))(*[t.data_ptr() for t in ts])
    lws = torch.empty(lbfgs_workspace_size(dims, B, m), dtype=torch.uint8, device=dev)
    d = torch.empty_like(gb)
    rc = _load().meta_lbfgs_direction(ctypes.byref(_problem(nd, dims, B, 1, 1.0)), m, len(Sb),
                                      arr(Sb), arr(Yb), _p(gb), _p(d),
                                      ctypes.c_void_p(lws.data_ptr()), lws.numel(), _stream(dev))
    if rc:
        raise MetaError(rc, "meta_lbfgs_direction")
    return d[0] if sq else d


def lbfgs_minimize(I0: torch.Tensor, J: torch.Tensor, p0: torch.Tensor, T: int, sigma: float,
                   mu, rho=1.0, lam=1e-3, iters: int = 10, m: int = 5, h0: float = 0.05,
                   ndim: Optional[int] = None, ckpt: int = 0, p_update=0, scheme: str = "sl"):
    """L-BFGS on the Eq. 4 cost from p0 (meta_lbfgs_minimize).  Returns (p, costs
    [iters + 1, B] float64 numpy, last moving iteration per instance)."""
    I0b, nd, dims, sq = _shape(_as_batch(I0, "I0")[0], ndim)
    Jb = _like(_as_batch(J, "J")[0], I0b, "J")
    p = _like(_as_batch(p0, "p0")[0], I0b, "p0").clone()
    B, dev = I0b.shape[0], I0b.device
    ws = _workspace(dims, B, T, sigma, dev, None, ckpt, scheme)
    lws = torch.empty(lbfgs_workspace_size(dims, B, m), dtype=torch.uint8, device=dev)
    mu_t, rho_t, lam_t = _coef(mu, B, dev), _coef(rho, B, dev), _coef(lam, B, dev)
    hist = np.zeros((iters + 1, B), dtype=np.float64)
    done = np.zeros(B, dtype=np.int32)
    rc = _load().meta_lbfgs_minimize(
        ctypes.byref(_problem(nd, dims, B, T, sigma, ws.ckpt, p_update, scheme)), _p(I0b), _p(Jb),
        _p(p),
        _p(mu_t), _p(rho_t), _p(lam_t), int(iters), int(m), float(h0), ctypes.c_void_p(ws.ptr()),
        ws.nbytes, ctypes.c_void_p(lws.data_ptr()), lws.numel(),
        hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        done.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _stream(dev))
    if rc:
        raise MetaError(rc, "meta_lbfgs_minimize")
    return (p[0] if sq else p), hist, done


def gd_minimize(I0: torch.Tensor, J: torch.Tensor, p0: torch.Tensor, T: int, sigma: float,
                mu, rho=1.0, lam=1e-3, iters: int = 10, h0: float = 0.05,
                ndim: Optional[int] = None, ckpt: int = 0, p_update=0, scheme: str = "sl"):
    """Gradient descent on the Eq. 4 cost from p0, the paper's optimiser (Sec. 3),
    with the normalised step p <- p - h0 g / max|g| (meta_gd_minimize).  Returns
    (p, costs [iters + 1, B] float64 numpy)."""
    reg = Registration(I0, J, p0, T, sigma, mu, rho, lam, optimizer="gd", h0=h0, ndim=ndim,
                       ckpt=ckpt, p_update=p_update, scheme=scheme)
    hist = reg.run(iters)
    return reg.p, hist


class Registration:
    """An iterative registration of I0 to J: the Eq. 4 cost minimised over p0 by
    gradient descent (optimizer "gd", meta_gd_minimize) or L-BFGS ("lbfgs",
    meta_lbfgs_minimize / meta_lbfgs_resume), whose state can be saved to a host
    file and resumed in another process.  A run of a + b iterations and a run of
    a iterations, saved, resumed and run for b more give the same iterates bit for
    bit.  ``p`` is the current iterate, ``costs`` the cost history
    [iterations + 1, B] (float64 numpy)."""

    def __init__(self, I0, J, p0, T: int, sigma: float, mu, rho=1.0, lam=1e-3,
                 optimizer: str = "lbfgs", m: int = 5, h0: float = 0.05, ckpt: int = 0,
                 ndim: Optional[int] = None, p_update=0, scheme: str = "sl"):
        if optimizer not in ("gd", "lbfgs"):
            raise ValueError("optimizer must be 'gd' or 'lbfgs'")
        I0b, nd, dims, sq = _shape(_as_batch(I0, "I0")[0], ndim)
        self.I0 = I0b.contiguous()
        self.J = _like(_as_batch(J, "J")[0], I0b, "J").contiguous()
        self._p = _like(_as_batch(p0, "p0")[0], I0b, "p0").clone()
        self._sq = sq
        B, dev = I0b.shape[0], I0b.device
        self.optimizer, self.ndim, self.dims, self.batch = optimizer, nd, tuple(dims), B
        self.T, self.sigma, self.m, self.h0 = int(T), float(sigma), int(m), float(h0)
        self.p_update, self.scheme = _pupd(p_update), scheme
        self.ws = Workspace(dims, B, T, sigma, dev, ckpt, scheme)
        self.ckpt = self.ws.ckpt
        self.lws = torch.empty(lbfgs_workspace_size(dims, B, m if optimizer == "lbfgs" else 1),
                               dtype=torch.uint8, device=dev)
        self._mu, self._rho, self._lam = _coef(mu, B, dev), _coef(rho, B, dev), _coef(lam, B, dev)
        self.iterations = 0
        self.costs: Optional[np.ndarray] = None
        self._started = False  # the L-BFGS state in lws is valid

    @property
    def p(self) -> torch.Tensor:
        return self._p[0] if self._sq else self._p

    def _prob(self) -> _Problem:
        return _problem(self.ndim, self.dims, self.batch, self.T, self.sigma, self.ckpt,
                        self.p_update, self.scheme)

    def run(self, iters: int) -> np.ndarray:
        """`iters` more iterations; returns their cost history [iters + 1, B]."""
        iters = int(iters)
        if iters < 0:
            raise ValueError("iters must be >= 0")
        lib, dev = _load(), self.I0.device
        hist = np.zeros((iters + 1, self.batch), dtype=np.float64)
        hp = hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        common = (ctypes.byref(self._prob()), _p(self.I0), _p(self.J), _p(self._p), _p(self._mu),
                  _p(self._rho), _p(self._lam))
        with torch.cuda.device(dev):
            if self.optimizer == "gd":
                rc = lib.meta_gd_minimize(*common, iters, self.h0, ctypes.c_void_p(self.ws.ptr()),
                                          self.ws.nbytes, ctypes.c_void_p(self.lws.data_ptr()),
                                          self.lws.numel(), hp, _stream(dev))
                what = "meta_gd_minimize"
            else:
                fn = lib.meta_lbfgs_resume if self._started else lib.meta_lbfgs_minimize
                what = "meta_lbfgs_resume" if self._started else "meta_lbfgs_minimize"
                done = np.zeros(self.batch, dtype=np.int32)
                rc = fn(*common, iters, self.m, self.h0, ctypes.c_void_p(self.ws.ptr()),
                        self.ws.nbytes, ctypes.c_void_p(self.lws.data_ptr()), self.lws.numel(), hp,
                        done.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _stream(dev))
        if rc:
            raise MetaError(rc, what)
        self._started = True
        self.costs = hist if self.costs is None else np.concatenate([self.costs, hist[1:]])
        self.iterations += iters
        return hist

    def _settings(self) -> dict:
        f = lambda t: [float(x) for x in t.cpu().tolist()]
        return dict(optimizer=self.optimizer, ndim=self.ndim, dims=list(self.dims),
                    batch=self.batch, T=self.T, sigma=self.sigma, mu=f(self._mu),
                    rho=f(self._rho), lam=f(self._lam), m=self.m, h0=self.h0, ckpt=self.ckpt,
                    p_update=self.p_update, scheme=self.scheme, iterations=self.iterations)

    def save(self, path) -> None:
        """Writes p, the iteration count, the cost history and (L-BFGS) the optimiser
        state to a host file (paper_2106_08817_gb300.checkpoint)."""
        from . import checkpoint
        if self.costs is None:
            self.run(0)  # the cost at p0 (and, for L-BFGS, its gradient and an empty state)
        blob = None
        if self.optimizer == "lbfgs":
            lib, dev = _load(), self.I0.device
            n = ctypes.c_size_t(0)
            rc = lib.meta_lbfgs_state_size(ctypes.byref(self._prob()), self.m, ctypes.byref(n))
            if rc:
                raise MetaError(rc, "meta_lbfgs_state_size")
            buf = (ctypes.c_ubyte * n.value)()
            with torch.cuda.device(dev):
                rc = lib.meta_lbfgs_state_save(ctypes.byref(self._prob()), self.m,
                                               ctypes.c_void_p(self.lws.data_ptr()),
                                               self.lws.numel(), buf, n.value, _stream(dev))
            if rc:
                raise MetaError(rc, "meta_lbfgs_state_save")
            blob = bytes(buf)
        digest = checkpoint.images_digest(self.I0.cpu().numpy(), self.J.cpu().numpy())
        checkpoint.write(path, self._settings(), self._p.cpu().numpy(), self.costs, digest, blob)

    @classmethod
    def resume(cls, path, I0, J, device=None) -> "Registration":
        """A registration continued from a file written by save(), on the same images
        (checked by their SHA-256)."""
        from . import checkpoint
        st = checkpoint.read(path)
        dev = torch.device(device) if device is not None else (
            I0.device if isinstance(I0, torch.Tensor) else torch.device("cuda"))
        I0t = torch.as_tensor(I0, dtype=torch.float32).to(dev)
        Jt = torch.as_tensor(J, dtype=torch.float32).to(dev)
        shape = (st["batch"],) + tuple(st["dims"])
        I0t, Jt = I0t.reshape(shape), Jt.reshape(shape)
        if checkpoint.images_digest(I0t.cpu().numpy(), Jt.cpu().numpy()) != st["images_sha256"]:
            raise ValueError("these are not the images the registration was saved with")
        reg = cls(I0t, Jt, torch.from_numpy(st["p"]).to(dev), st["T"], st["sigma"], st["mu"],
                  st["rho"], st["lam"], optimizer=st["optimizer"], m=st["m"], h0=st["h0"],
                  ckpt=st["ckpt"], ndim=st["ndim"], p_update=st["p_update"], scheme=st["scheme"])
        reg.iterations, reg.costs = st["iterations"], st["costs"]
        reg._started = True
        if reg.optimizer == "lbfgs":
            blob = st["lbfgs_state"]
            buf = (ctypes.c_ubyte * len(blob)).from_buffer_copy(blob)
            with torch.cuda.device(dev):
                rc = _load().meta_lbfgs_state_load(ctypes.byref(reg._prob()), reg.m, buf,
                                                   len(blob),
                                                   ctypes.c_void_p(reg.lws.data_ptr()),
                                                   reg.lws.numel(), _stream(dev))
            if rc:
                raise MetaError(rc, "meta_lbfgs_state_load")
        return reg


class CostAndGradPlan:
    """A cost_and_grad call recorded once into a CUDA graph (meta_plan_*).

    The plan owns fixed input/output tensors (I0, J, p0, mu, rho, lam, cost,
    grad) and its workspace: update the inputs in place (e.g. ``plan.p0.sub_(...)``)
    and call ``launch()``; results appear in ``plan.cost`` / ``plan.grad``.
    """

    def __init__(self, I0, J, p0, T: int, sigma: float, mu, rho=1.0, lam=1e-3,
                 ndim: Optional[int] = None, ckpt: int = 0, p_update=0, scheme: str = "sl"):
        I0b, nd, dims, _ = _shape(_as_batch(I0, "I0")[0], ndim)
        B, dev = I0b.shape[0], I0b.device
        self.I0 = I0b.clone()
        self.J = _like(_as_batch(J, "J")[0], I0b, "J").clone()
        self.p0 = _like(_as_batch(p0, "p0")[0], I0b, "p0").clone()
        self.mu, self.rho, self.lam = (_coef(mu, B, dev).clone(), _coef(rho, B, dev).clone(),
                                       _coef(lam, B, dev).clone())
        self.cost = torch.empty((B, 3), dtype=torch.float64, device=dev)
        self.grad = torch.empty_like(I0b)
        self.ws = Workspace(dims, B, T, sigma, dev, ckpt, scheme)
        self.device = dev
        pr = _problem(nd, dims, B, T, sigma, ckpt, p_update, scheme)
        h = ctypes.c_void_p(0)
        torch.cuda.synchronize(dev)
        rc = _load().meta_plan_create(ctypes.byref(pr), _p(self.I0), _p(self.J), _p(self.p0),
                                      _p(self.mu), _p(self.rho), _p(self.lam), _p(self.cost),
                                      _p(self.grad), ctypes.c_void_p(self.ws.ptr()),
                                      self.ws.nbytes, ctypes.byref(h))
        if rc:
            raise MetaError(rc, "meta_plan_create")
        self._h = h

    def launch(self):
        rc = _load().meta_plan_launch(self._h, _stream(self.device))
        if rc:
            raise MetaError(rc, "meta_plan_launch")
        return self.cost, self.grad

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.meta_plan_destroy(h)
            self._h = None


class GroupPlan:
    """Many independent problems of different shapes / T / sigma (2-D and 3-D
    mixed) recorded into one CUDA graph as parallel branches (meta_plan_create_group),
    or, with ``persistent=True``, run by ONE persistent kernel launch
    (meta_plan_create_persistent: the semi-Lagrangian scheme, default momentum update).

    `problems` is a list of dicts with keys I0, J, p0 ([B, *dims] CUDA tensors),
    T, sigma, mu, rho, lam (optional: ckpt, p_update, scheme).  Each item keeps its own copies of the inputs
    (``plan.items[k]["p0"]`` etc.), cost [B, 3] and grad; ``launch()`` runs all.
    """

    def __init__(self, problems, streams: int = 8, persistent: bool = False):
        self.persistent = bool(persistent)
        self.items = []
        n = len(problems)
        probs = (_Problem * n)()
        ptr = lambda: (ctypes.c_void_p * n)()
        I0s, Js, p0s, mus, rhos, lams, costs, grads, wss = (ptr() for _ in range(9))
        wsb = (ctypes.c_size_t * n)()
        dev = None
        for k, pb in enumerate(problems):
            I0b, nd, dims, _ = _shape(_as_batch(pb["I0"], "I0")[0], pb.get("ndim"))
            B, dev = I0b.shape[0], I0b.device
            it = {"I0": I0b.clone(), "J": _like(_as_batch(pb["J"], "J")[0], I0b, "J").clone(),
                  "p0": _like(_as_batch(pb["p0"], "p0")[0], I0b, "p0").clone(),
                  "mu": _coef(pb["mu"], B, dev).clone(), "rho": _coef(pb.get("rho", 1.0), B, dev).clone(),
                  "lam": _coef(pb.get("lam", 1e-3), B, dev).clone(),
                  "cost": torch.empty((B, 3), dtype=torch.float64, device=dev),
                  "grad": torch.empty_like(I0b), "T": int(pb["T"]), "sigma": float(pb["sigma"]),
                  "dims": dims, "B": B}
            it["ckpt"] = int(pb.get("ckpt", 0))
            it["scheme"] = pb.get("scheme", "sl")
            it["ws"] = Workspace(dims, B, it["T"], it["sigma"], dev, it["ckpt"], it["scheme"])
            probs[k] = _problem(nd, dims, B, it["T"], it["sigma"], it["ckpt"],
                                pb.get("p_update", 0), it["scheme"])
            for arr, key in ((I0s, "I0"), (Js, "J"), (p0s, "p0"), (mus, "mu"), (rhos, "rho"),
                             (lams, "lam"), (costs, "cost"), (grads, "grad")):
                arr[k] = it[key].data_ptr()
            wss[k] = it["ws"].ptr()
            wsb[k] = it["ws"].nbytes
            self.items.append(it)
        self.device = dev
        h = ctypes.c_void_p(0)
        torch.cuda.synchronize(dev)
        with torch.cuda.device(dev):
            if self.persistent:
                rc = _load().meta_plan_create_persistent(n, probs, I0s, Js, p0s, mus, rhos, lams,
                                                         costs, grads, wss, wsb, ctypes.byref(h))
            else:
                rc = _load().meta_plan_create_group(n, probs, I0s, Js, p0s, mus, rhos, lams,
                                                    costs, grads, wss, wsb, int(streams),
                                                    ctypes.byref(h))
        if rc:
            raise MetaError(rc, "meta_plan_create_persistent" if self.persistent
                            else "meta_plan_create_group")
        self._h = h

    def launch(self):
        rc = _load().meta_plan_launch(self._h, _stream(self.device))
        if rc:
            raise MetaError(rc, "meta_plan_launch")

    def status(self, clear: bool = False) -> int:
        """The plan's own status bits (meta_plan_status; persistent plans: bit 0 = a
        dependency wait ran out and a launch was abandoned).  Synchronises the stream."""
        bits = ctypes.c_uint(0)
        rc = _load().meta_plan_status(self._h, int(clear), _stream(self.device),
                                      ctypes.byref(bits))
        if rc not in (0, 5):
            raise MetaError(rc, "meta_plan_status")
        return int(bits.value)

    def selftest_timeout(self, hold: int = 0, limit_ns: int = 50_000_000) -> None:
        """One persistent launch in which problem `hold`'s first phase never reports
        completion: its next phase's bounded wait runs out (meta_plan_selftest_timeout)."""
        rc = _load().meta_plan_selftest_timeout(self._h, int(hold), int(limit_ns),
                                                _stream(self.device))
        if rc:
            raise MetaError(rc, "meta_plan_selftest_timeout")

    def voxel_steps(self) -> int:
        return sum(it["B"] * int(np.prod(it["dims"])) * it["T"] for it in self.items)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.meta_plan_destroy(h)
            self._h = None


NOALLOC_MAX_BYTES = 64 << 20


def cost_and_grad_noalloc(I0: torch.Tensor, J: torch.Tensor, p0: torch.Tensor, T: int,
                          sigma: float, mu, rho=1.0, lam=1e-3, ndim: Optional[int] = None,
                          out: Optional[Tuple[torch.Tensor, torch.Tensor]] = None, ckpt: int = 0,
                          p_update=0, scheme: str = "sl", check_status: bool = False
                          ) -> Tuple[torch.Tensor, torch.Tensor]:
    """cost_and_grad on the library's fixed 64 MiB device scratch: no workspace
    argument.  For callers that cannot allocate device memory; pass `out` (and
    device tensors for mu, rho, lam) so that this call allocates nothing either.
    Calls share the scratch: order them on one stream.  The call runs with the
    images' device current (the library picks that device's scratch).
    check_status: wait for the call and raise MetaError (status 5) if a device-side
    wait ran out; otherwise read noalloc_status() before the next call."""
    I0b, nd, dims, sq = _shape(_as_batch(I0, "I0")[0], ndim)
    Jb = _like(_as_batch(J, "J")[0], I0b, "J")
    p0b = _like(_as_batch(p0, "p0")[0], I0b, "p0")
    B, dev = I0b.shape[0], I0b.device
    mu_t, rho_t, lam_t = _coef(mu, B, dev), _coef(rho, B, dev), _coef(lam, B, dev)
    if out is not None:
        cost, grad = _outputs(out, I0b)
    else:
        cost = torch.empty((B, 3), dtype=torch.float64, device=dev)
        grad = torch.empty_like(I0b)
    pr = _problem(nd, dims, B, T, sigma, ckpt, p_update, scheme)
    with torch.cuda.device(dev):
        rc = _load().meta_cost_and_grad_noalloc(ctypes.byref(pr), _p(I0b), _p(Jb), _p(p0b),
                                                _p(mu_t), _p(rho_t), _p(lam_t), _p(cost),
                                                _p(grad), _stream(dev))
        if rc:
            raise MetaError(rc, "meta_cost_and_grad_noalloc")
        if check_status and noalloc_status(device=dev) & 1:
            raise MetaError(5, "meta_cost_and_grad_noalloc")
    if sq and out is None:
        grad = grad[0]
    return cost, grad


def noalloc_status(clear: bool = False, device=None) -> int:
    """Device fault bits of the no-allocation scratch of `device` (default: the current
    one) latched since the last cost_and_grad_noalloc began (meta_noalloc_status;
    synchronises the stream).  Bit 0: a bounded device wait ran out (that call's results
    are invalid); bit 1: an adjoint step used the atomic scatter (order not fixed)."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None \
        else torch.device(device)
    bits = ctypes.c_uint(0)
    with torch.cuda.device(dev):
        rc = _load().meta_noalloc_status(int(clear), _stream(dev), ctypes.byref(bits))
    if rc not in (0, 5):
        raise MetaError(rc, "meta_noalloc_status")
    return int(bits.value)


def noalloc_selftest_timeout(limit_ns: int = 50_000_000, device=None) -> None:
    """Enqueues a bounded device wait that runs out on the no-allocation scratch
    (meta_noalloc_selftest_timeout): the timeout bit then shows in noalloc_status()."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None \
        else torch.device(device)
    with torch.cuda.device(dev):
        rc = _load().meta_noalloc_selftest_timeout(int(limit_ns), _stream(dev))
    if rc:
        raise MetaError(rc, "meta_noalloc_selftest_timeout")


class Shoot(torch.autograd.Function):
    """(I0, p0) -> (I_T, p_T) with the hand-written adjoint as backward.

    forward keeps the trajectory in a fresh workspace; backward runs the
    discrete transpose of every step on it (no recomputation needed).
    """

    @staticmethod
    def forward(ctx, I0, p0, T, sigma, mu, rho, p_update=0, scheme="sl"):
        I0c, p0c = I0.detach().contiguous(), p0.detach().contiguous()
        b_, nd, dims, sq = _shape(I0c, None)
        ws = Workspace(dims, b_.shape[0], T, sigma, I0c.device, 0, scheme)
        I1, p1, _ = shoot_forward(I0c, p0c, T, sigma, mu, rho, workspace=ws, p_update=p_update,
                                  scheme=scheme)
        ctx.ws, ctx.args, ctx.shape = ws, (T, sigma, mu, rho, p_update, scheme), I0c.shape
        return I1, p1

    @staticmethod
    def backward(ctx, gI1, gp1):
        T, sigma, mu, rho, p_update, scheme = ctx.args
        if gI1 is None:
            gI1 = torch.zeros(ctx.shape, device=ctx.ws.buf.device)
        gI0, gp0 = shoot_adjoint(gI1.contiguous(), None if gp1 is None else gp1.contiguous(),
                                 ctx.ws, T, sigma, mu, rho, want_gI0=ctx.needs_input_grad[0],
                                 p_update=p_update, scheme=scheme)
        return gI0, gp0, None, None, None, None, None, None


def shoot(I0, p0, T: int, sigma: float, mu, rho=1.0, p_update=0, scheme: str = "sl"):
    """Differentiable shooting: torch autograd calls the library's adjoint."""
    return Shoot.apply(I0, p0, T, sigma, mu, rho, p_update, scheme)


def timer_start(cap: int = 1 << 16) -> None:
    """Bracket every following library launch with CUDA events (profiling aid)."""
    rc = _load().meta_timer_start(int(cap))
    if rc:
        raise MetaError(rc, "meta_timer_start")


def timer_stop() -> dict:
    """{kernel class: (summed device ms, scopes timed, kernels launched)} since timer_start."""
    n = len(KERNEL_CLASSES)
    ms = (ctypes.c_float * n)()
    cnt = (ctypes.c_int * n)()
    rc = _load().meta_timer_stop(ms, cnt)
    if rc:
        raise MetaError(rc, "meta_timer_stop")
    return {k: (float(ms[i]), int(cnt[i]), int(cnt[i]) * _LAUNCHES_PER_SCOPE.get(k, 1))
            for i, k in enumerate(KERNEL_CLASSES)}
