"""pclb_diagnostics_noalloc against pclb_diagnostics (GPU).

The no-allocation entry point serves callers that cannot call cudaMalloc
(inside a stream capture, inside an allocator's callbacks, plug-ins without a
memory pool): it keeps its reduction scratch in a fixed device array instead
of a caller workspace.  Its results must equal those of the workspace-based
entry point, call after call (the shared array keeps the previous call's
contents).  This file is collected last so that a stop-at-first-failure run
has run every other test first.
"""
import numpy as np
import pytest

from paper_1302_7104_gb300 import inputs as I
from paper_1302_7104_gb300 import pclb as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# same tolerances as the diagnostics parity tests
TOL = {"fp64": 1e-13, "fp32": 2e-7}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_diagnostics_match_workspace_entry_point(prec):
    cases = [I.random_smooth(45, 23, seed=21), I.kh(n_r=96, n_theta=64)]
    for w in cases:
        with P.PCLB(w, precision=prec) as g:
            g.set_state().step(3)
            want = g.diagnostics()
            f = g.get_f()
            for _ in range(2):   # two calls in a row share the static scratch
                got = P.diagnostics_noalloc(w, f, prec, stream=g.stream)
                assert got[:6] == pytest.approx(want[:6], rel=TOL[prec], abs=TOL[prec] * want[0])
                assert got[6] == want[6] == w.n_r * w.n_theta


def test_noalloc_rejects_grids_beyond_its_scratch():
    w = I.random_smooth(8, 16385, seed=3)
    f = torch.zeros((33, 16385, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(P.PCLBError) as e:
        P.diagnostics_noalloc(w, f, "fp32")
    assert e.value.code == 1 and "16384" in str(e.value)
