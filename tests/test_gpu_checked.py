"""The checked build (libstap compiled with -DSTAP_CHECKED) on the GPU: every
kernel index into a global buffer, and every shared- and tensor-memory offset
of the tensor-core kernels, is compared with its extent; an access outside it
would be skipped and recorded (nothing traps).  These runs cover the plain
and mixed-precision paths, the edge shapes, the training and snapshot options
and a small batch; they must skip no access and still match the oracle.  The
checked library is loaded in a child process (STAP_CHECKED=1)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu

CHILD = r'''
import json, sys
sys.path.insert(0, "tests")
import numpy as np
import torch
import oracle
from paper_2203_06233_gb300 import stap, synth
from _parity import EDGE_SPECS, power_errors
assert stap.stap_checked_build()
res = []
def case(name, spec, okw, **kw):
    d = oracle.Dims(*spec.dims())
    cube = synth.make_cube(spec)
    ref = oracle.run(d, cube, **okw)["out"]
    plan = stap.Plan(spec.dims(), **kw)
    out = plan.run_cpi(torch.from_numpy(cube).cuda()).cpu().numpy()
    code, failed = plan.status()
    plan.close()
    e_cell, e_norm = power_errors(out, ref)
    n, site, idx, ext = stap.stap_check_report()
    res.append(dict(name=name, code=code, failed=failed, e_norm=e_norm, skipped=n, site=site,
                    index=idx, extent=ext))
specs = [("small", synth.small_cpi()), ("standard", synth.standard_cpi())] + \
        [(f"edge{i}", s) for i, s in enumerate(EDGE_SPECS)]
for name, spec in specs:
    case(name, spec, {})
for prec in (1, 2, 3):
    for name, spec in [("small", synth.small_cpi()), ("edge3", EDGE_SPECS[3]), ("edge8", EDGE_SPECS[8])]:
        case(f"{name} prec {prec}", spec, {}, precision=prec)
case("window", synth.CPISpec(3, 20, 32, 96, 2, 4, 5, cnr_db=30.0, seed=33), dict(training=2, guard=1, half=3),
     training=2, train_guard=1, train_half=3)
case("neighbours", synth.standard_cpi(), dict(training=1), training=1)
case("staggered", synth.small_cpi(), dict(staggered=True), snapshots=1)
case("mixed_ir D64", EDGE_SPECS[3], {}, solver=1, refine_steps=2)
specs = [synth.CPISpec(4, 64, 64, 256, 3, 64, 8, cnr_db=30.0, seed=41),
         synth.CPISpec(8, 32, 64, 128, 2, 64, 16, cnr_db=35.0, seed=42)]
cubes = [torch.from_numpy(synth.make_cube(s)).cuda() for s in specs]
plan = stap.Plan([s.dims() for s in specs], precision=1)
outs = plan.run_cpi(cubes)
torch.cuda.synchronize()
plan.close()
n, site, idx, ext = stap.stap_check_report()
res.append(dict(name="batch bf16x3", code=0, failed=0, e_norm=0.0, skipped=n, site=site, index=idx, extent=ext))
print("RESULT " + json.dumps(res))
'''


def test_checked_build_skips_no_access_and_matches_the_oracle():
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, capture_output=True, text=True,
                       env=dict(os.environ, STAP_CHECKED="1"), timeout=1800)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    res = json.loads(line[len("RESULT "):])
    for c in res:
        print(c)
    assert all(c["skipped"] == 0 for c in res), [c for c in res if c["skipped"]]
    assert all(c["code"] == 0 and c["failed"] == 0 for c in res)
    assert all(c["e_norm"] <= 1e-3 for c in res)
