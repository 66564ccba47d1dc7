"""Full-size parity: the mixed-workload and large-workload shapes through
stap_run_cpi (the plain FP32 path), checked against the oracle on seeded
range blocks.  Blocks are independent (the Doppler transform is per range
cell), so the oracle's result for a block's window is exact for those cells.
The cube is generated on the device and copied back, so both sides see the
same complex64 input."""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2203_06233_gb300 import stap, synth

from _parity import power_errors

pytestmark = pytest.mark.gpu


def growth(spec):
    return max(1.0, (spec.D + 2) / 14.0)


@pytest.mark.parametrize("name,nblocks", [("mixed", 4), ("large", 2)])
def test_full_size_workload_on_sampled_blocks(name, nblocks):
    spec = synth.WORKLOADS[name]()
    d = oracle.Dims(*spec.dims())
    cube_d = synth.make_cube_torch(spec, "cuda")
    plan = stap.Plan(spec.dims(), device="cuda")
    out_d = plan.run_cpi(cube_d)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan.run_cpi(cube_d, out_d)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    code, failed = plan.status()
    assert code == stap.STAP_OK and failed == 0
    print(f"{name}: {spec.dims()} one CPI in {el * 1e3:.1f} ms "
          f"({spec.cells / el:.3e} cells/s)")
    cube = cube_d.cpu().numpy()
    B = spec.training_block
    rng = np.random.default_rng(1234 + spec.seed)
    blocks = sorted(int(b) for b in rng.choice(spec.NB, nblocks, replace=False))
    g = growth(spec)
    for b in blocks:
        ref = oracle.run(d, cube, r0=b * B, nr=B)
        assert ref["n_failed"] == 0
        got = out_d[:, :, b * B:(b + 1) * B].cpu().numpy()
        e_cell, e_norm = power_errors(got, ref["out"])
        print(f"  block {b}: max-cell/floor={e_cell:.3e} normwise={e_norm:.3e}")
        assert e_norm <= 1e-5 * g and e_cell <= 1e-3 * g, (b, e_cell, e_norm)
    plan.close()
