"""bench.py's reference arm (the FP64 oracle on the host cores) prints the contract's JSON line (CPU)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--workload", "tiny"], capture_output=True, text=True, env=env, cwd=ROOT,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["unit"] == d["unit"]


def test_committed_traffic_lookup():
    """The bench's `traffic` comes from the committed ncu record when it was taken on the current
    kernel source: per bucket and grid type, scaled by the bucket's ligand count; a bucket kernel
    with another warps-per-item count reads its bucket's figure; an unrecorded bucket gives None."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2209_05069_gb300 import synth
    rec = json.load(open(os.path.join(ROOT, "profiles", "dock_kernel_traffic.json")))
    src = os.path.join(ROOT, "paper_2209_05069_gb300", "csrc", "dock_kernels.cuh")
    if rec["kernel_source_sha1"] != bench.kernel_source_sha1(src):
        pytest.skip("the record was taken on another kernel source (the bench reports traffic: null)")
    db = synth.make_db(synth.WORKLOADS["uneven"], rec["captured_ligands"])
    k = next(iter(rec["records"]["f32"]["per_kernel"]))   # e.g. dock_kernel<64, 0, 2, 1>
    maxn = int(k.split("<")[1].split(",")[0])
    bucket = maxn // 32 - 1
    n = np.diff(db.atom_off)
    in_bucket = int(((n - 1) // 32 == bucket).sum())
    got = bench.committed_kernel_traffic("f32", k, db, bucket, in_bucket)
    assert got == pytest.approx(rec["records"]["f32"]["per_kernel"][k])
    other_g = "dock_kernel<" + ",".join(k.split("<", 1)[1].split(",")[:2]) + ", 8, 1>"
    assert bench.committed_kernel_traffic("f32", other_g, db, bucket, 2 * in_bucket) == pytest.approx(2 * got)
    wide = "dock_kernel_wide<" + ",".join(k.split("<", 1)[1].split(",")[:2]) + ", 1, 2>"
    assert bench.committed_kernel_traffic("f32", wide, db, bucket, in_bucket) == pytest.approx(got)
    assert bench.committed_kernel_traffic("f32", "dock_kernel<160, 0, 2, 1>", db, 4, 10) is None
