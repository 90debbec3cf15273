"""C-ABI checks that need no GPU: the library loads, exports every symbol that
include/meta.h declares, and rejects bad arguments with error codes before any
CUDA call."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def meta():
    from paper_2106_08817_gb300 import _build
    _build.build()
    import paper_2106_08817_gb300 as m
    return m


def declared_functions():
    text = open(os.path.join(ROOT, "include", "meta.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(meta_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("meta_shoot_forward", "meta_shoot_adjoint", "meta_cost_and_grad",
                 "meta_workspace_size", "meta_status_string", "meta_workspace_status"):
        assert must in names


def test_library_exports_every_declared_symbol(meta):
    lib = meta._load()
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings(meta):
    lib = meta._load()
    for code in range(10):
        assert lib.meta_status_string(code).decode() != "unknown status", code
        assert meta.STATUS[code]
    assert lib.meta_status_string(99).decode() == "unknown status"


@pytest.mark.parametrize("kw,code", [
    (dict(ndim=4), 1), (dict(ndim=1), 1), (dict(batch=0), 1), (dict(T=0), 1),
    (dict(T=5000), 1), (dict(sigma=0.0), 1), (dict(sigma=-1.0), 1), (dict(sigma=19.0), 1),
    (dict(sigma=float("nan")), 1), (dict(dims=(1, 5)), 2), (dict(dims=(5, 70000)), 2),
])
def test_invalid_problems_are_rejected(meta, kw, code):
    prm = dict(ndim=2, dims=(16, 16), batch=1, T=4, sigma=2.0)
    prm.update(kw)
    pr = meta._problem(prm["ndim"], prm["dims"], prm["batch"], prm["T"], prm["sigma"])
    n = ctypes.c_size_t(0)
    assert meta._load().meta_workspace_size(ctypes.byref(pr), ctypes.byref(n)) == code


def test_momentum_update_values(meta):
    n = ctypes.c_size_t(0)
    for val, code in ((0, 0), (1, 0), (2, 1), (-1, 1)):
        pr = meta._problem(2, (16, 16), 1, 4, 2.0)
        pr.p_update = val
        assert meta._load().meta_workspace_size(ctypes.byref(pr), ctypes.byref(n)) == code
    with pytest.raises(ValueError):
        meta._problem(2, (16, 16), 1, 4, 2.0, 0, "exact")
    assert meta._problem(2, (16, 16), 1, 4, 2.0, 0, "det").p_update == 1


def test_schemes_and_their_workspace(meta):
    lib = meta._load()
    n = ctypes.c_size_t(0)
    for sch, pu, code in ((0, 0, 0), (1, 0, 0), (2, 0, 0), (3, 0, 1), (1, 1, 1), (2, 1, 1)):
        pr = meta._problem(2, (16, 16), 1, 4, 2.0)
        pr.scheme, pr.p_update = sch, pu
        assert lib.meta_workspace_size(ctypes.byref(pr), ctypes.byref(n)) == code
    # the Eulerian and hybrid adjoints pass raw (I^, p^) between steps: two more fields
    sl = meta.workspace_size((16, 16), 3, 4, 2.0)
    for sch in ("euler", "hybrid"):
        pr = meta._problem(2, (16, 16), 3, 4, 2.0, scheme=sch)
        assert lib.meta_workspace_size(ctypes.byref(pr), ctypes.byref(n)) == 0
        assert n.value == sl + 2 * 3 * 16 * 16 * 4
    # with step checkpoints too: the semi-Lagrangian adjoint recomputes each segment
    # before the gradp that needs it and passes no raw adjoints
    assert (meta.workspace_size((16, 16), 3, 6, 2.0, 3, "euler")
            == meta.workspace_size((16, 16), 3, 6, 2.0, 3, "sl") + 2 * 3 * 16 * 16 * 4)
    with pytest.raises(ValueError):
        meta._problem(2, (16, 16), 1, 4, 2.0, scheme="lagrangian")


def test_workspace_size_grows_with_T_and_batch(meta):
    a = meta.workspace_size((64, 64), 1, 10, 3.0)
    b = meta.workspace_size((64, 64), 2, 10, 3.0)
    c = meta.workspace_size((64, 64), 1, 20, 3.0)
    assert b > a and c > a
    # the trajectory (2 (T+1) + d T fields) dominates: check the order of magnitude
    fields = 2 * 11 + 2 * 10 + 4 * 2 + 6
    assert fields * 64 * 64 * 4 <= a < (fields + 8) * 64 * 64 * 4


def test_checkpointing_shrinks_the_workspace(meta):
    """ckpt_stride k keeps ceil(T/k) checkpoints plus two segments (2k states, 2k + 1
    velocity fields) instead of T+1 states and T velocity fields."""
    full = meta.workspace_size((64, 64, 64), 1, 20, 5.0)
    k5 = meta.workspace_size((64, 64, 64), 1, 20, 5.0, ckpt=5)
    f = 64 * 64 * 64 * 4
    assert full >= (2 * 21 + 3 * 20) * f
    assert (2 * (4 + 10) + 3 * 11) * f <= k5 <= (2 * (4 + 10) + 3 * 11 + 4 * 3 + 8 + 1) * f
    assert k5 < full
    assert meta.workspace_size((64, 64, 64), 1, 20, 5.0, ckpt=1) == full
    assert meta.workspace_size((64, 64, 64), 1, 20, 5.0, ckpt=20) == full
    pr = meta._problem(3, (8, 8, 8), 1, 4, 1.0, -1)
    n = ctypes.c_size_t(0)
    assert meta._load().meta_workspace_size(ctypes.byref(pr), ctypes.byref(n)) == 1


def test_tuning_table_round_trip_and_validation(meta):
    """Tile shapes per problem shape: built-in equal tiles, set / get / forget,
    and range checks before anything runs."""
    dims, B, s = (160, 192, 160), 1, 6.0
    meta.set_tuning(dims, B, s, None)
    t0 = meta.tuning(dims, B, s)
    assert (t0["ly"], t0["lz"], t0["txw"]) == (96, 80, 80)  # 192 = 2 x 96, 160 = 2 x 80
    assert 1 <= t0["zc_transport"] <= 160 and 1 <= t0["zc_advect"] <= 160 and t0["split"] == 1
    mine = dict(zc_transport=8, zc_advect=16, ly=64, lz=48, txw=64, split=1)
    meta.set_tuning(dims, B, s, mine)
    assert meta.tuning(dims, B, s) == mine
    meta.set_tuning(dims, B, s, dict(ly=32))  # zero fields: built-in choice
    assert meta.tuning(dims, B, s)["ly"] == 32 and meta.tuning(dims, B, s)["lz"] == 80
    # a whole 160-wide row per x tile: staged row 160 + 2 x 20 + 4 = 204 <= 256 (halo 20:
    # r = 18, r4 = 20, taps to 40 = r4 + 20)
    meta.set_tuning(dims, B, s, dict(txw=160))
    assert meta.tuning(dims, B, s)["txw"] == 160
    # strided tiles up to 192 whose window (tile + taps, 40 at sigma 6) one TMA box holds
    meta.set_tuning(dims, B, s, dict(ly=192, lz=160))
    assert (meta.tuning(dims, B, s)["ly"], meta.tuning(dims, B, s)["lz"]) == (192, 160)
    for bad in (dict(ly=40), dict(ly=208), dict(txw=12), dict(zc_transport=161),
                dict(lz=-16), dict(zc_advect=-1), dict(split=2),  # split <= batch (1 here)
                dict(txw=224), dict(txw=264)):  # staged rows of 264 and 304 floats
        with pytest.raises(meta.MetaError):
            meta.set_tuning(dims, B, s, bad)
    with pytest.raises(meta.MetaError):  # sigma 18: halo 56, so 144 + 112 = 256 fits no wider
        meta.set_tuning(dims, B, 18.0, dict(txw=152))
    meta.set_tuning(dims, B, 18.0, dict(txw=144))
    with pytest.raises(meta.MetaError):  # sigma 18: 112 taps, so 160 + 112 > 256
        meta.set_tuning(dims, B, 18.0, dict(ly=160))
    meta.set_tuning(dims, B, 18.0, dict(ly=144, lz=144))
    meta.set_tuning(dims, B, 18.0, None)
    with pytest.raises(meta.MetaError):
        meta.set_tuning((64, 64), 1, 2.0, dict(lz=16))  # 2-D problems have no z tiles
    with pytest.raises(meta.MetaError):  # y tiles x nz beyond the launch grid limit
        meta.set_tuning((4000, 2000, 64), 1, 2.0, dict(ly=16))
    meta.set_tuning(dims, B, s, None)
    assert meta.tuning(dims, B, s) == t0
    t2 = meta.tuning((256, 256), 16, 6.0)
    assert (t2["ly"], t2["txw"], t2["lz"], t2["zc_transport"], t2["split"]) == (128, 128, 0, 0, 1)
    meta.set_tuning((256, 256), 16, 6.0, dict(split=4))
    assert meta.tuning((256, 256), 16, 6.0)["split"] == 4
    with pytest.raises(meta.MetaError):
        meta.set_tuning((256, 256), 16, 6.0, dict(split=17))
    meta.set_tuning((256, 256), 16, 6.0, None)


def test_workspace_covers_every_batch_split(meta):
    """A split plan runs sub-batch k in its own aligned region of the caller's
    workspace: meta_workspace_size covers the sum for every split."""
    one = meta.workspace_size((37, 141), 1, 5, 2.3)
    for B in (2, 5, 16):  # split into B regions of one instance each
        n = meta.workspace_size((37, 141), B, 5, 2.3)
        assert B * one <= n <= B * one + 64 * 1024
    n = meta.workspace_size((37, 141), 40, 5, 2.3)  # at most 16 regions
    assert abs(n - 40 * one) <= 64 * 1024


def test_null_pointers_and_bad_workspace_fail_before_any_cuda_call(meta):
    lib = meta._load()
    pr = meta._problem(2, (16, 16), 1, 4, 2.0)
    fake = ctypes.c_void_p(0x1000)
    null = ctypes.c_void_p(0)
    need = meta.workspace_size((16, 16), 1, 4, 2.0)
    # null inputs
    assert lib.meta_cost_and_grad(ctypes.byref(pr), null, fake, fake, fake, fake, fake, fake,
                                  fake, fake, need, null) == 1
    assert lib.meta_shoot_forward(ctypes.byref(pr), fake, null, fake, fake, fake, fake, fake,
                                  need, null) == 1
    assert lib.meta_shoot_adjoint(ctypes.byref(pr), fake, fake, fake, fake, fake, null, fake,
                                  need, null) == 1
    # deformation: neither phi nor jac asked for, a null input, a short workspace
    assert lib.meta_shoot_deform(ctypes.byref(pr), fake, fake, fake, fake, fake, fake, null,
                                 null, fake, need, null) == 1
    assert lib.meta_shoot_deform(ctypes.byref(pr), null, fake, fake, fake, null, null, fake,
                                 null, fake, need, null) == 1
    assert lib.meta_shoot_deform(ctypes.byref(pr), fake, fake, fake, fake, null, null, null,
                                 fake, fake, need - 1, null) == 3
    # workspace: null, misaligned, too small
    assert lib.meta_cost_and_grad(ctypes.byref(pr), fake, fake, fake, fake, fake, fake, fake,
                                  fake, null, need, null) == 3
    assert lib.meta_cost_and_grad(ctypes.byref(pr), fake, fake, fake, fake, fake, fake, fake,
                                  fake, ctypes.c_void_p(0x1010), need, null) == 3
    assert lib.meta_cost_and_grad(ctypes.byref(pr), fake, fake, fake, fake, fake, fake, fake,
                                  fake, fake, need - 1, null) == 3


def test_lbfgs_arguments_fail_before_any_cuda_call(meta):
    lib = meta._load()
    pr = meta._problem(2, (16, 16), 2, 4, 2.0)
    n = ctypes.c_size_t(0)
    assert lib.meta_lbfgs_workspace_size(ctypes.byref(pr), 0, ctypes.byref(n)) == 1
    assert lib.meta_lbfgs_workspace_size(ctypes.byref(pr), 65, ctypes.byref(n)) == 1
    assert lib.meta_lbfgs_workspace_size(ctypes.byref(pr), 5, ctypes.byref(n)) == 0
    need = n.value
    # 2 x 5 pairs + 6 vectors of 2 x 256 floats, plus the per-instance scalars
    assert need >= (2 * 5 + 6) * 2 * 256 * 4
    assert meta.lbfgs_workspace_size((16, 16), 2, 5) == need
    fake, null = ctypes.c_void_p(0x1000), ctypes.c_void_p(0)
    ws = meta.workspace_size((16, 16), 2, 4, 2.0)
    args = [ctypes.byref(pr), fake, fake, fake, fake, fake, fake]
    # h0 <= 0, a null input, a short or misaligned L-BFGS workspace
    assert lib.meta_lbfgs_minimize(*args, 3, 5, 0.0, fake, ws, fake, need, None, None, null) == 1
    assert lib.meta_lbfgs_minimize(ctypes.byref(pr), null, fake, fake, fake, fake, fake, 3, 5,
                                   0.1, fake, ws, fake, need, None, None, null) == 1
    assert lib.meta_lbfgs_minimize(*args, 3, 5, 0.1, fake, ws, fake, need - 1, None, None,
                                   null) == 3
    assert lib.meta_lbfgs_minimize(*args, 3, 5, 0.1, fake, ws, ctypes.c_void_p(0x1010), need,
                                   None, None, null) == 3
    assert lib.meta_lbfgs_direction(ctypes.byref(pr), 5, 6, None, None, fake, fake, fake, need,
                                    null) == 1


def test_workspace_cache_can_be_cleared(meta):
    meta._ws_cache[("probe",)] = object()
    meta.clear_workspaces()
    assert meta._ws_cache == {}
    assert "clear_workspaces" in meta.__all__


def test_arrays_must_match_the_image_shape(meta):
    """Every array of a call has the image batch's shape [B, *dims] (or [*dims] when
    B = 1); a transposed or otherwise reshaped array raises instead of being read in
    the wrong order."""
    import torch
    ref = torch.zeros(2, 5, 7)
    assert meta._like(torch.ones(2, 5, 7), ref, "J").shape == (2, 5, 7)
    one = torch.zeros(1, 5, 7)
    assert meta._like(torch.ones(5, 7), one, "J").shape == (1, 5, 7)
    for bad in (torch.ones(2, 7, 5), torch.ones(5, 7), torch.ones(2, 35), torch.ones(70),
                torch.ones(3, 5, 7), torch.empty(2, 5, 7, device="meta")):
        with pytest.raises(ValueError):
            meta._like(bad, ref, "J")


def test_caller_outputs_are_checked(meta):
    """cost_and_grad(out=(cost, grad)): the kernels write cost [B, 3] (float64) and grad
    (float32, the images' shape) whole, so anything else raises before the call."""
    import torch
    ref = torch.zeros(2, 5, 7)
    cost, grad = torch.zeros(2, 3, dtype=torch.float64), torch.zeros(2, 5, 7)
    assert meta._outputs((cost, grad), ref)[1] is grad
    assert meta._outputs((cost, None), ref)[1] is None
    bad = [(torch.zeros(2, 3), grad), (torch.zeros(3, 3, dtype=torch.float64), grad),
           (torch.zeros(3, 2, dtype=torch.float64).t(), grad),
           (cost, torch.zeros(2, 5, 7, dtype=torch.float64)), (cost, torch.zeros(2, 7, 5)),
           (cost, torch.zeros(2, 7, 5).transpose(1, 2)), (cost, torch.zeros(2, 5, 6))]
    for c, g in bad:
        with pytest.raises(ValueError):
            meta._outputs((c, g), ref)


def test_lbfgs_pairs_must_come_in_pairs(meta):
    """lbfgs_direction with unequal numbers of s and y vectors raises before the C call
    (which would otherwise read past the shorter pointer array)."""
    import torch
    real = meta._as_batch
    meta._as_batch = lambda x, name: (x.contiguous(), False)  # CPU tensors for the check
    try:
        g = torch.zeros(1, 4, 5)
        with pytest.raises(ValueError):
            meta.lbfgs_direction(g, [g, g], [g])
    finally:
        meta._as_batch = real
