"""The pivot search's launch variants give bit-identical results.

Every variant of the full-search pivot kernel forms each entry with the same operations
(l = S[r, j] x (1 / pivot) with one reciprocal per step, S[r, c] - l S[i, c] fused, ties to the
lowest row x n + col), so the variant chosen for a launch shape must not change a single bit of
the pivots, D, L, U or of a whole product. The variant is fixed per process by environment
variables read once by the library (ACI_PRRLU_2D = 0: never the 2D register kernel, 2: wherever it
fits; ACI_PRRLU_GRIDC / ACI_PRRLU_CLUSTER: its column groups / the cluster size; ACI_PRRLU_MBX:
its candidate exchange through mbarriers or the cluster barrier), so each
configuration runs in a child process; the default configuration is compared with the oracle in
test_gpu_kernels.py and test_gpu_aci.py."""

import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (m, n, chimax, complex): 2D grids 4 x 4 (tiles 4 x 8, 2 x 4, 1 x 8), 8 x 2, 2 x 8, 2 x 2; the
# 1D kernel at 480 x 480, 480 x 246 and 160 x 400
CASES = [(480, 480, 240, False), (256, 256, 128, False), (200, 200, 100, True), (128, 300, 128, True),
         (700, 100, 90, False), (100, 700, 90, False), (37, 53, 30, False), (480, 246, 200, False),
         (160, 400, 150, False)]

CHILD = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_2604_00037_gb300.binding import Context
from synthetic.tt import tt_random_uniform
cases = eval(sys.argv[3])
ctx = Context(0)
out = {}
for (m, n, k, cp) in cases:
    rng = np.random.default_rng(m * 1000 + n)
    r = min(m, n)
    U = rng.standard_normal((m, r))
    V = rng.standard_normal((r, n))
    if cp:
        U = U + 1j * rng.standard_normal(U.shape)
        V = V + 1j * rng.standard_normal(V.shape)
    M = (U * (10.0 ** -np.linspace(0, 12, r))) @ V
    g = ctx.prrlu(torch.from_numpy(M).cuda(), 1e-13 * np.abs(M).max(), k)
    for key in ("I", "J", "D", "L", "U"):
        out[f"{m}x{n}{'c' if cp else 'r'}_{key}"] = g[key]
rng = np.random.default_rng(7)
a = tt_random_uniform(rng, 10, 2, 24, low=-1, high=1)
b = tt_random_uniform(rng, 10, 2, 24, low=-1, high=1)
dev = lambda tt: [torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in tt]
y, info = ctx.elementwise(dev(a), dev(b), "mul", 1e-12, 256)
for i, c in enumerate(y):
    out[f"product_core{i}"] = c.cpu().numpy()
np.savez(sys.argv[2], **out)
"""


def _run(env_extra, path):
    env = dict(os.environ)
    for v in ("ACI_PRRLU_2D", "ACI_PRRLU_GRIDC", "ACI_PRRLU_CLUSTER", "ACI_PRRLU_MBX"):
        env.pop(v, None)
    env.update(env_extra)
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, str(path), repr(CASES)], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    return np.load(path)


@pytest.fixture(scope="module")
def default_run(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return _run({}, tmp_path_factory.mktemp("piv") / "default.npz")


@pytest.mark.parametrize("env", [{"ACI_PRRLU_2D": "0"}, {"ACI_PRRLU_2D": "2"},
                                 {"ACI_PRRLU_2D": "2", "ACI_PRRLU_GRIDC": "2"},
                                 {"ACI_PRRLU_2D": "2", "ACI_PRRLU_GRIDC": "8"},
                                 {"ACI_PRRLU_2D": "2", "ACI_PRRLU_CLUSTER": "4"}, {"ACI_PRRLU_CLUSTER": "8"},
                                 {"ACI_PRRLU_2D": "2", "ACI_PRRLU_MBX": "1"},
                                 {"ACI_PRRLU_2D": "2", "ACI_PRRLU_MBX": "0"}])
def test_variants_are_bit_identical(default_run, env, tmp_path):
    other = _run(env, tmp_path / "variant.npz")
    assert sorted(default_run.files) == sorted(other.files)
    for key in default_run.files:
        x, y = default_run[key], other[key]
        assert x.shape == y.shape, key
        assert np.ascontiguousarray(x).tobytes() == np.ascontiguousarray(y).tobytes(), key
