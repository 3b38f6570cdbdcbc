"""GPU parity when the power spectrum splits its fields into several chunks
whose sizes are not multiples of the fields a block takes (the paired row
pass takes four): run in a child process with a 1 MiB chunk target
(CF_PK_CHUNK_MB, read once per process), 70 fields of 64^2 -> chunks of 62
and 8 fields, binary32 fields and count maps, against the oracle."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU collection
    pytest.skip("needs a CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, %(root)r)
from paper_1406_6072_gb300 import cf
from paper_1406_6072_gb300 import workloads as W
dev = torch.device("cuda:0")
n, F, nb = (64, 64), 70, 16
x = W.gaussian_field_values((F,) + n, seed=81, scale=1.0).astype(np.float32)
c = np.random.default_rng(82).poisson(2.0, size=(F,) + n).astype(np.int32)
g = cf.make_grid(n)
bins = cf.make_bins(nb)
wsb = cf.cf_power_spectrum_workspace_size(g, F, bins, cf.CF_F32)
out = {}
for name, arr in (("fields", x), ("counts", c)):
    ws = torch.full((wsb + (64 << 20),), 0xA5, dtype=torch.uint8, device=dev)  # tail guard beyond the workspace
    pk = torch.empty((F, nb), dtype=torch.float64, device=dev)
    nm = torch.empty(nb, dtype=torch.int64, device=dev)
    t = torch.from_numpy(arr).to(dev)
    if name == "fields":
        cf.cf_power_spectrum(t, cf.CF_F32, g, F, bins, pk, nm, None, None, ws, wsb)
    else:
        cf.cf_power_spectrum_counts(t, None, g, F, bins, pk, nm, None, None, ws, wsb)
    torch.cuda.synchronize()
    out[name] = pk.cpu().numpy().tolist()
    out[name + "_guard_intact"] = bool((ws[wsb:] == 0xA5).all().item())
print(json.dumps(out))
"""


def test_power_spectrum_chunks_not_multiple_of_four(orc):
    from paper_1406_6072_gb300 import workloads as W
    env = dict(os.environ, CF_PK_CHUNK_MB="1")
    p = subprocess.run([sys.executable, "-c", CHILD % {"root": ROOT}], capture_output=True, text=True, env=env,
                       timeout=600)
    assert p.returncode == 0, p.stderr[-3000:]
    got = json.loads(p.stdout.strip().splitlines()[-1])
    assert got["fields_guard_intact"] and got["counts_guard_intact"]
    n, F, nb = (64, 64), 70, 16
    x = W.gaussian_field_values((F,) + n, seed=81, scale=1.0).astype(np.float32)
    c = np.random.default_rng(82).poisson(2.0, size=(F,) + n).astype(np.int32)
    edges = orc.bin_edges(orc.BINS_LINEAR, nb, 0.0, n[0] / 2)
    opk, _ = orc.power_spectrum(x.astype(np.float64), n, edges)
    assert np.allclose(np.array(got["fields"]), opk, rtol=2e-5, atol=1e-9 * opk.max())
    dg = orc.counts_to_delta(c.reshape(F, -1), None).reshape((F,) + n)
    opkg, _ = orc.power_spectrum(dg, n, edges)
    assert np.allclose(np.array(got["counts"]), opkg, rtol=2e-5, atol=1e-9 * opkg.max())
