"""Autotuner (GPU): the tuned configuration is stored and used, and results
stay identical to the oracle under it."""
import numpy as np
import pytest

import oracle
from oracle import exact
from paper_1109_1264_gb300 import inputs
from paper_1109_1264_gb300 import programs as P

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_autotune_program_and_nrm2(saltlib, cuda_dev):
    s = saltlib
    s.salt_tune_clear()
    try:
        n = (1 << 20) + 3
        for dt, tdt, code in ((np.float32, torch.float32, s.F32), (np.float64, torch.float64, s.F64)):
            vecs = inputs.uniform_vectors(31, n, 5, dt)
            tv = [torch.from_numpy(v).to(cuda_dev) for v in vecs]
            cfg, ms = s.salt_autotune(s.KERNEL_PROGRAM, P.PROG_E, tv, [1.5, -0.25], reps=2)
            assert ms > 0 and s.salt_tune_get(P.PROG_E, code, n) == cfg
            tv[4].zero_()
            s.salt_eval(P.PROG_E, tv, [1.5, -0.25])
            want = [v.copy() for v in vecs]
            oracle.eval_program(P.PROG_E, want, [1.5, -0.25])
            assert np.array_equal(tv[4].cpu().numpy().view(np.uint8), want[4].view(np.uint8))
            out = torch.zeros(1, dtype=torch.float64, device=cuda_dev)
            cfg, ms = s.salt_autotune(s.KERNEL_NRM2, None, [tv[0]], red_out=out, reps=2)
            s.salt_nrm2(tv[0], out)
            ref = exact.exact_nrm2(vecs[0])
            tol = 1e-6 if dt == np.float32 else 1e-13
            assert abs(out.item() - ref) <= tol * ref
    finally:
        s.salt_tune_clear()
