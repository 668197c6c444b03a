"""The index-checked debug build (liblfa_debug.so, -DLFA_DEBUG): every kernel route on valid inputs
records no failed index check (lfa_info_t.debug_error == 0) and still matches the FP64 oracle. The
checks record a site id and skip the access; none traps. Runs in a child interpreter with
LFA_DEBUG=1, which makes the binding load the debug library."""
import os
import subprocess
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
import lfa_workloads as W
import oracle as O
from paper_2506_05617_gb300 import lfa as C
from paper_2506_05617_gb300.torch_api import LfaPlan
assert C.LIB_PATH.endswith("liblfa_debug.so"), C.LIB_PATH
out = []
# (c_out, c_in, k, n, m, stride, option variant): single-CTA, cluster, rotation-log, blocked, strided
cases = [(16, 16, 3, 4, 4, 1, None), (256, 128, 3, 2, 3, 1, None), (512, 256, 3, 2, 2, 1, None),
         (512, 512, 3, 2, 2, 1, C.LFA_VARIANT_BLOCKED), (32, 16, 3, 4, 4, 2, None), (128, 160, 3, 2, 2, 1, None)]
for co, ci, k, n, m, st, var in cases:
    rng = np.random.default_rng(co + ci)
    w = (rng.standard_normal((co, ci, k, k)) / np.sqrt(ci * k * k)).astype(np.float32)
    desc = (co, ci, k, k, n, m, -1, -1, st, st)
    kw = {} if var is None else {"variant": var}
    plan = LfaPlan([desc], vectors=True, **kw)
    sig, U, V = plan.svd([torch.from_numpy(w).cuda()])
    g = torch.ones_like(sig[0])
    dw = plan.backward([g], U, V)
    r = min(co, ci * st * st)
    uh, vh = plan.expand(0, U[0], V[0], 0, min(4, n * m * r))
    torch.cuda.synchronize()
    status, info = plan.info()
    if st == 1:
        s_ref = O.lfa_svd(w, n, m, compute_uv=False)
    else:
        s_ref = O.lfa_svd_strided(w, n, m, st, st, compute_uv=False)
    err = float(np.max(np.abs(sig[0].cpu().numpy() - s_ref)) / s_ref.max())
    out.append({"case": [co, ci, k, n, m, st], "variant": plan.meta[0]["variant_name"], "status": status,
                "debug_error": info["debug_error"], "sigma_err": err})
    plan.close()
print(json.dumps(out))
'''


def test_debug_build_reports_no_failed_index_check():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_05617_gb300 import build as B
    B.build(debug=True)
    env = dict(os.environ, LFA_DEBUG="1")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    import json
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert len(res) == 6
    for case in res:
        assert case["debug_error"] == 0, case
        assert case["status"] == 0, case
        assert case["sigma_err"] <= 1e-5, case
