"""Host-side logic that needs no GPU: the seeded input recipes (shapes, ranges, seed
stability) and the benchmark's reference arm, whose JSON line other tools read."""
import json
import os
import subprocess
import sys

import numpy as np

from paper_1401_7962_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_mixed_batch_recipe_ranges_and_layout():
    sizes, kappas, offsets = wl.mixed_batch_params(4096, wl.SEED_BASE + 5)
    assert sizes.dtype == np.int32 and sizes.min() >= 128 and sizes.max() <= 1024
    # uniform orders: every eighth of the range is used, the mean is near the middle
    assert abs(sizes.mean() - 576) < 15
    counts, _ = np.histogram(sizes, bins=8, range=(128, 1025))
    assert counts.min() > 0.8 * 512 and counts.max() < 1.2 * 512
    assert kappas.min() >= 1e2 and kappas.max() <= 1e8
    lk = np.log10(kappas)
    assert abs(lk.mean() - 5.0) < 0.1          # log-uniform in [2, 8]
    assert offsets[0] == 0 and np.array_equal(np.diff(offsets), sizes[:-1].astype(np.int64) ** 2)
    # seed-stable: the same call gives the same batch; another seed does not
    s2, k2, _ = wl.mixed_batch_params(4096, wl.SEED_BASE + 5)
    assert np.array_equal(sizes, s2) and np.array_equal(kappas, k2)
    s3, _, _ = wl.mixed_batch_params(4096, wl.SEED_BASE + 6)
    assert not np.array_equal(sizes, s3)


def test_mixed_batch_host_matrices_have_the_recipe_spectrum():
    sizes = np.array([5, 12, 9], dtype=np.int32)
    kappas = np.array([1e2, 1e4, 1e3])
    offsets = np.array([0, 25, 25 + 144], dtype=np.int64)
    packed = wl.mixed_batch_host(sizes, kappas, offsets, seed=7)
    assert packed.dtype == np.float32 and packed.size == 25 + 144 + 81
    for m in range(3):
        A = wl.unpack(sizes, packed, offsets, m).astype(np.float64)
        sv = np.linalg.svd(A, compute_uv=False)
        # singular values log-spaced from 1 to kappa (up to the FP32 rounding of A)
        want = np.logspace(0.0, np.log10(kappas[m]), int(sizes[m]))[::-1]
        assert np.allclose(sv, want, rtol=1e-4 * kappas[m])
        # matrix m is the single-matrix recipe with its own seed
        B = wl.svd_conditioned(int(sizes[m]), float(kappas[m]), wl.mixed_batch_seed(7, m))
        assert np.array_equal(A, B.astype(np.float64))


def test_reference_arm_prints_one_json_line():
    env = dict(os.environ)
    env.pop("WORLD_SIZE", None)
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "inv128", "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600,
                         env=env, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [x for x in out.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "GFLOP/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
