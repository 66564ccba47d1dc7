"""Full-size parity: the D = 64 CPI (C16 P256 K256 R16384 T4 B128 S32) and
the large CPI (C32 P512 K512 R32768 T4 B256 S64, D = 128, about 4.3 GB)
through stap_run_cpi, on the plain FP32 path and on every mixed-precision
path, checked against the oracle on seeded range blocks.  Blocks are
independent (the Doppler transform is per range cell), so the oracle's
result for a block's window is exact for those cells.  The cube is generated
on the device and copied back, so both sides see the same complex64 input;
each block's oracle result serves every path.

Bars per block: plain normwise <= 1e-5 g and worst cell <= PLAIN_CELL_BAR g,
with g = (D + 2)/14 (the FP32 dot products' error growth with D); mixed
normwise <= 1e-3 and worst cell <= mixed_cell_bar (2 x 2^-21 (D/lf + 1), the
first-order effect of the split products' covariance error under the
conditioning that the diagonal load allows)."""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2203_06233_gb300 import stap, synth

from _parity import MIXED_NORM_BAR, MIXED_PRECISIONS, PLAIN_CELL_BAR, mixed_cell_bar, power_errors

pytestmark = pytest.mark.gpu


def growth(spec):
    return max(1.0, (spec.D + 2) / 14.0)


@pytest.mark.parametrize("name,nblocks", [("mixed", 4), ("large", 8)])
def test_full_size_workload_on_sampled_blocks(name, nblocks):
    spec = synth.WORKLOADS[name]()
    d = oracle.Dims(*spec.dims())
    cube_d = synth.make_cube_torch(spec, "cuda")
    paths = [("plain", stap.STAP_PREC_FP32)] + MIXED_PRECISIONS
    outs = {}
    for pname, prec in paths:
        plan = stap.Plan(spec.dims(), device="cuda", precision=prec)
        out_d = plan.run_cpi(cube_d)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.run_cpi(cube_d, out_d)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        code, failed = plan.status()
        assert code == stap.STAP_OK and failed == 0, (pname, code, failed)
        print(f"{name} {pname}: {spec.dims()} one CPI in {el * 1e3:.1f} ms "
              f"({spec.cells / el:.3e} cells/s)")
        outs[pname] = out_d
        plan.close()
    cube = cube_d.cpu().numpy()
    B = spec.training_block
    rng = np.random.default_rng(1234 + spec.seed)
    blocks = sorted(int(b) for b in rng.choice(spec.NB, nblocks, replace=False))
    g = growth(spec)
    bad = []
    for b in blocks:
        ref = oracle.run(d, cube, r0=b * B, nr=B)
        assert ref["n_failed"] == 0
        for pname, _ in paths:
            got = outs[pname][:, :, b * B:(b + 1) * B].cpu().numpy()
            e_cell, e_norm = power_errors(got, ref["out"])
            print(f"  block {b} {pname}: max-cell/floor={e_cell:.3e} normwise={e_norm:.3e}")
            if pname == "plain":
                ok = e_norm <= 1e-5 * g and e_cell <= PLAIN_CELL_BAR * g
            else:
                ok = e_norm <= MIXED_NORM_BAR and e_cell <= mixed_cell_bar(spec)
            if not ok:
                bad.append((pname, b, e_cell, e_norm))
    assert not bad, bad
