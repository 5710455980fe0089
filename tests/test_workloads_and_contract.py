"""Host-side checks, no GPU: the synthetic workloads have the sizes and
structure the benchmark's descriptions state (5-tet box grids; the bar, the
two-blocks scene, the 256-mesh batch), and the reference arm of bench.py
prints one JSON line with the keys of the benchmark contract."""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("n,nv,ne", [(10, 1331, 5000), (48, 117649, 552960), (64, 274625, 1310720)])
def test_box_grid_counts(n, nv, ne):
    X, tets = W.box_grid(n, n, n, 1.0 / n)
    assert X.shape == (nv, 3) and tets.shape == (ne, 4)
    # every tet has positive volume with the builder's orientation
    d = X[tets[:, 1:]] - X[tets[:, :1]]
    vol = np.einsum("ij,ij->i", d[:, 0], np.cross(d[:, 1], d[:, 2])) / 6.0
    assert np.all(vol > 0) and np.isclose(vol.sum(), 1.0)


def test_bar_and_blocks_sizes():
    bar = W.contact_bar()
    assert (bar.nv, bar.ne) == (337881, 1600000)
    assert len(bar.spr_idx) == round(0.02 * bar.nv) and bar.k_contact == 1e8
    blocks = W.two_blocks_hanging(64, 48, k=1e5)
    assert (blocks.nv, blocks.ne) == (392274, 1863680)
    idx, w, kn, kt, nrm = blocks.meta["weak"]
    assert idx.shape == (2401, 8) and np.allclose(w[:, :4].sum(1), 1.0) and np.allclose(w[:, 4:].sum(1), 1.0)


def test_batch_is_uneven_and_seeded():
    probs = W.batched_blocks()
    sides = [q.meta["cells"][0] for q in probs]
    assert len(probs) == 256 and min(sides) >= 8 and max(sides) <= 32 and len(set(sides)) > 10
    again = W.batched_blocks()
    assert all(np.array_equal(a.x0, b.x0) for a, b in zip(probs[:8], again[:8]))


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config",
                          "twist10", "--steps", "2", "--warmup", "1"], capture_output=True, text=True, cwd=ROOT,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "e2e", "cpu_baseline", "impl"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert "workload" in d["config"]
