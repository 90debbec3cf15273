"""Host-side pieces of bench.py that need no GPU: the byte models behind
`path_roofline`, the source hash that guards the committed ncu traffic, and the
traffic lookup."""
import json
import os
import shutil

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_model_bytes_per_voxel_step():
    # forward F = 24 + 8 d^2, adjoint A = 48 + 12 d + 8 d^2, recompute F + 4d
    assert bench.model_bytes_per_voxel_step(2) == 224
    assert bench.model_bytes_per_voxel_step(3) == 360


def test_own_bytes_add_the_recomputed_forward_steps():
    keep2, keep3 = bench.own_bytes_per_voxel_step(2, 20, 0), bench.own_bytes_per_voxel_step(3, 20, 0)
    assert (keep2, keep3) == (196.0, 296.0)
    fwd3 = (bench.bytes_per_voxel("xpass_m", 3) + 2 * bench.bytes_per_voxel("strided_fwd", 3)
            + bench.bytes_per_voxel("advect", 3))
    # T = 20, k = 5: segments 0 and 1 are recomputed (10 of 20 steps), the last two
    # stay in place after the forward
    assert bench.own_bytes_per_voxel_step(3, 20, 5) == pytest.approx(keep3 + 10 / 20 * fwd3)
    # T = 10, k = 4: segment [0,4) recomputed, [4,8) and [8,10) kept: 4 of 10 steps
    assert bench.own_bytes_per_voxel_step(3, 10, 4) == pytest.approx(keep3 + 4 / 10 * fwd3)
    # 2-D, T = 7, k = 3: two sets of segment slots would not be smaller than the whole
    # trajectory, so one set: [0,3), [3,6) recomputed, [6,7) kept: 6 of 7 steps
    fwd2 = (bench.bytes_per_voxel("xpass_m", 2) + bench.bytes_per_voxel("strided_fwd", 2)
            + bench.bytes_per_voxel("advect", 2))
    assert bench.own_bytes_per_voxel_step(2, 7, 3) == pytest.approx(keep2 + 6 / 7 * fwd2)
    # T = 40, k = 5: two sets, segments 0..5 recomputed (30 of 40 steps)
    assert bench.own_bytes_per_voxel_step(3, 40, 5) == pytest.approx(keep3 + 30 / 40 * fwd3)
    # strides of 0, 1 or >= T keep the whole trajectory
    for k in (0, 1, 20, 25):
        assert bench.own_bytes_per_voxel_step(3, 20, k) == keep3


def test_source_hash_ignores_comments_but_not_code(tmp_path):
    src = os.path.join(ROOT, "paper_2106_08817_gb300", "csrc")
    dst = tmp_path / "csrc"
    shutil.copytree(src, dst)
    h0 = bench.kernel_sources_hash(str(dst))
    assert h0 == bench.kernel_sources_hash()
    f = dst / "meta_blur.cu"
    text = f.read_text()
    f.write_text("// an added comment\n" + text.replace("namespace meta {", "namespace meta {  /* x */", 1))
    assert bench.kernel_sources_hash(str(dst)) == h0
    f.write_text(text.replace("kBX", "kBX + 0", 1))
    assert bench.kernel_sources_hash(str(dst)) != h0


def test_committed_traffic_is_scaled_by_voxels_and_keyed_by_dimension():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        d = json.load(fh)
    if d.get("sources_hash") != bench.kernel_sources_hash():
        pytest.skip("traffic.json was taken on other kernel sources")
    k2 = d["kernels"]["adj_gather@2"]
    full = bench.ncu_traffic("adj_gather", 2, k2["voxels_per_launch"])
    assert full == pytest.approx(k2["dram_bytes_per_launch"])
    assert bench.ncu_traffic("adj_gather", 2, k2["voxels_per_launch"] // 2) == pytest.approx(full / 2)
    assert bench.ncu_traffic("no_such_class", 2, 1000) is None


def test_reference_arm_prints_one_complete_line():
    """bench.py --impl reference: the FP64 oracle on the host cores prints one JSON line with
    the same metric and workload as the GPU arm, its own cpu_baseline and e2e."""
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "disk64", "--steps", "2", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 3 and d["higher_is_better"]
    assert d["config"]["workload"] == "disk64"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0


def test_cpu_baseline_reports_all_cores_and_one_thread():
    """cpu_baseline: the oracle on every host core (value, cores), and on one thread when
    an instance fits in a third of the sample time (null otherwise)."""
    import oracle
    w = bench.workload("disk64")
    d = bench.cpu_baseline_entry(w, 0.6)
    assert d["kind"] == "oracle" and d["unit"] == bench.UNIT and d["value"] > 0
    assert d["cores"] == oracle.max_threads()
    assert d["single_thread"]["cores"] == 1 and d["single_thread"]["value"] > 0
    assert oracle.max_threads() == d["cores"]  # the thread count is restored
    assert bench.cpu_baseline_entry(w, 1e-9)["single_thread"] is None


def test_model_bytes_per_kernel_class_add_up_to_the_model():
    """The roofline's per-class bytes are the parts of the fixed model: forward
    F = (8 + 4d) + (d - 1) 8d + (16 + 4d), adjoint (24 + 8d) + 8d + (d - 1) 8d + (24 + 4d),
    and the path is 2F + 4d + A."""
    for d in (2, 3):
        m = lambda k: bench.model_bytes_per_voxel(k, d)
        F = m("xpass_m") + (d - 1) * m("strided_fwd") + m("advect")
        A = m("adj_gather") + m("xpass_adj") + (d - 1) * m("strided_adj") + m("adj_gradp")
        assert F == 24 + 8 * d * d and A == 48 + 12 * d + 8 * d * d
        assert 2 * F + 4 * d + A == bench.model_bytes_per_voxel_step(d)
    assert bench.model_bytes_per_voxel("adj_gather", 3) == 48
    # classes outside the model fall back to the implementation's own count
    assert bench.model_bytes_per_voxel("cost", 3) == bench.bytes_per_voxel("cost", 3)


def test_downsampled_copy_halves_extent_and_kernel_width():
    w = bench.workload("head16")
    h = bench.downsampled_copy(w)
    assert bench.single_volume(w) and not bench.single_volume(bench.workload("disk64"))
    assert h.dims == (8, 8, 8) and h.sigma == w.sigma / 2 and h.T == w.T
    assert h.I0.shape == (1, 8, 8, 8)
    assert abs(float(h.I0.mean()) - float(w.I0.mean())) < 1e-6  # block means keep the mean


def test_cpu_baseline_of_a_single_volume_runs_it_whole_and_its_2x_copy():
    """A single volume: the oracle once on the full volume (the value), once on its 2x
    block-averaged copy, and the library's result on the copy compared with the
    oracle's (here a stand-in that returns the oracle's own result: zero error)."""
    import oracle
    w = bench.workload("head16")

    def same(h):
        return oracle.cost_and_grad(h.I0[0], h.J[0], h.p0[0], h.T, h.sigma, float(h.mu[0]),
                                    float(h.rho[0]), float(h.lam[0]))

    d = bench.cpu_baseline_entry(w, 3.0, same)
    assert d["kind"] == "oracle" and d["value"] > 0 and d["cores"] == oracle.max_threads()
    assert "16x16x16" in d["sample"]
    ds = d["downsampled_2x"]
    assert ds["value"] > 0 and "8x8x8" in ds["sample"]
    assert ds["vs_gpu"]["grad_relL2"] == 0.0 and max(ds["vs_gpu"]["cost_rel_err"]) == 0.0
    assert d["single_thread"]["cores"] == 1


def test_reference_arm_samples_a_single_volume_by_its_2x_copy():
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "head16", "--steps", "2", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    d = json.loads(lines[0])
    assert d["config"]["workload"] == "head16" and d["config"]["dims"] == [16, 16, 16]
    assert "2x block-averaged copy" in d["cpu_baseline"]["sample"]
    assert d["ms_per_step"] > 0 and d["value"] > 0
