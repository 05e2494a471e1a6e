"""Device memory of the trace's working pool, through the C-ABI.

The walk's record slots and each model's ray buffer come from a memory pool of
the library that keeps them reserved between traces (of the same or another
model) and returns them to the driver when the last model on the device is
destroyed.  The test traces two
models in turn, checks that the second trace reuses the reserve instead of
taking more memory, that the rays are unchanged by the reuse, and that
destroying both models gives the memory back.  It runs in a fresh process, so
that no model of another test keeps the reserve alive.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_2411_03040_gb300 import build, mgt, synth
build.build()
mgt.load()
torch.zeros(1, device="cuda")
torch.cuda.synchronize()
free0, _ = torch.cuda.mem_get_info()
m = synth.shell_model(20000, 3, 2, 5, seed=21, name="pool-20k")
a = mgt.mgt_model_create(m)
st_a = mgt.mgt_trace_rays(a)
off_a, idx_a = mgt.mgt_get_rays(a)
torch.cuda.synchronize()
free1, _ = torch.cuda.mem_get_info()
b = mgt.mgt_model_create(m)
st_b = mgt.mgt_trace_rays(b)
mgt.mgt_trace_rays(a)
torch.cuda.synchronize()
free2, _ = torch.cuda.mem_get_info()
off_a2, idx_a2 = mgt.mgt_get_rays(a)
same = bool(np.array_equal(off_a, off_a2) and np.array_equal(idx_a, idx_a2))
a.close()
b.close()
torch.cuda.synchronize()
free3, _ = torch.cuda.mem_get_info()
print(json.dumps({"free": [free0, free1, free2, free3], "same_rays": same,
                  "steps": [st_a["total_steps"], st_b["total_steps"]]}))
"""


def test_trace_pool_is_reused_and_released():
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    free0, free1, free2, free3 = out["free"]
    MiB = 1 << 20
    # after the first trace: model a's arrays and rays plus the reserved walk
    # scratch (48 x 20,000 walks x 128-record slots x 16 B = 1.97 GB)
    scratch = 48 * 20000 * 128 * 16
    assert free0 - free1 > scratch, (free0 - free1) / MiB
    # model b adds its own arrays and rays, not a second scratch
    assert free1 - free2 < 0.5 * (free0 - free1), ((free1 - free2) / MiB, (free0 - free1) / MiB)
    assert out["same_rays"]
    assert out["steps"][0] == out["steps"][1]
    # all of it back once the last model is gone (within the driver's granularity)
    assert free0 - free3 < 64 * MiB, (free0 - free3) / MiB
