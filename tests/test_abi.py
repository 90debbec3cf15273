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
    for code in range(8):
        assert lib.meta_status_string(code).decode()
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
    # with step checkpoints the raw buffer is there already: no second one
    assert (meta.workspace_size((16, 16), 3, 6, 2.0, 3, "euler")
            == meta.workspace_size((16, 16), 3, 6, 2.0, 3, "sl"))
    with pytest.raises(ValueError):
        meta._problem(2, (16, 16), 1, 4, 2.0, scheme="lagrangian")


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
