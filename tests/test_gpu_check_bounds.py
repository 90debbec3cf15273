"""The bounds-checked debug build (META_CHECK_BOUNDS, libmeta_check.so, loaded with
META_LIB=check): every index the kernels compute from the data -- the lower
corner of each foot, the record cells the transports decode -- is checked against
its range, and a violation is clamped and latched in the workspace status word
(bit 2) instead of reaching memory outside its buffer.  On ordinary inputs
nothing is out of range: the checked build, run in a child process, must give
the ordinary build's costs and gradients and leave bit 2 clear, including steps
whose adjoint uses the gather window (1 < R) and the atomic scatter (R beyond
the window), and a checkpointed 3-D call."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (dims, batch, T, sigma, ckpt, p0 scale, seed, mu, rho, lam): small steps; a gather
# window of a few voxels; per-step displacements of 0.2 to 17 voxels (the scatter);
# 3-D checkpointed; a 3-D gather window of up to 4 voxels
CASES = [((48, 40), 2, 5, 2.0, 0, 5.0, 700, 0.1, 1.0, 1e-3),
         ((48, 52), 1, 3, 2.0, 0, 60.0, 710, 0.1, 1.0, 1e-3),
         ((70, 33), 1, 5, 3.0, 0, 200.0, 21, 0.2, 0.8, 1e-2),
         ((12, 20, 16), 1, 6, 1.5, 2, 5.0, 720, 0.1, 1.0, 1e-3),
         ((14, 16, 18), 1, 5, 1.5, 0, 220.0, 31, 0.1, 1.0, 1e-3)]

RUN = r"""
import json, os, sys
import numpy as np
import torch
sys.path.insert(0, {root!r})
sys.path.insert(0, os.path.join({root!r}, "tests"))
from paper_2106_08817_gb300 import _build
_build.build(check={check})
import paper_2106_08817_gb300 as meta
import phantoms
from scipy import ndimage
out = {{}}
for k, (dims, B, T, sigma, ckpt, scale, seed, mu, rho, lam) in enumerate(json.loads({cases!r})):
    dims = tuple(dims)
    I0, _ = phantoms.random_fields(seed, B, dims)
    J, _ = phantoms.random_fields(seed + 1, B, dims)
    r = np.random.default_rng(seed + 2)
    p0 = np.stack([ndimage.gaussian_filter(r.normal(size=dims), 2.0) * scale
                   for _ in range(B)]).astype(np.float32)
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    ws = meta.Workspace(dims, B, T, sigma, "cuda", ckpt)
    c, g = meta.cost_and_grad(f(I0), f(J), f(p0), T, sigma, [mu] * B, [rho] * B, [lam] * B,
                              workspace=ws, ckpt=ckpt)
    torch.cuda.synchronize()
    out["cost%d" % k] = c.cpu().numpy()
    out["grad%d" % k] = g.cpu().numpy()
    out["status%d" % k] = np.array(ws.status())
np.savez({path!r}, **out)
print("lib", meta.library_path())
"""


def run(tmp_path, check):
    path = str(tmp_path / ("check.npz" if check else "plain.npz"))
    code = RUN.format(root=ROOT, check=check, cases=json.dumps(CASES), path=path)
    env = dict(os.environ)
    if check:
        env["META_LIB"] = "check"
    else:
        env.pop("META_LIB", None)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    assert ("libmeta_check.so" in r.stdout) == check
    return np.load(path)


def test_checked_build_gives_the_same_results_and_no_bounds_bit(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    plain = run(tmp_path, False)
    chk = run(tmp_path, True)
    for k in range(len(CASES)):
        assert int(chk["status%d" % k]) & 4 == 0, k  # no index left its range
        assert int(chk["status%d" % k]) & 1 == 0, k
        assert (int(chk["status%d" % k]) & 2) == (int(plain["status%d" % k]) & 2), k
        np.testing.assert_allclose(chk["cost%d" % k], plain["cost%d" % k], rtol=1e-6, atol=0)
        g0, g1 = plain["grad%d" % k], chk["grad%d" % k]
        assert np.linalg.norm(g1 - g0) <= 1e-5 * np.linalg.norm(g0), k
    assert int(plain["status2"]) & 2  # that case did take the atomic scatter
