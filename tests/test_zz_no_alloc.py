"""pclb_diagnostics_noalloc against pclb_diagnostics and the oracle (GPU).

The no-allocation entry point serves callers that cannot call cudaMalloc
(inside an allocator's own callbacks, plug-ins without a memory pool, hosts
that gave all device memory to another framework): it keeps its reduction
scratch in a fixed device array instead of a caller workspace.  Its results
must equal those of the workspace-based entry point and of the oracle, call
after call (the shared array keeps the previous call's contents), and a call
must not change the device's free memory.  This file is collected last so
that a stop-at-first-failure run has run every other test first.
"""
import numpy as np
import pytest

import oracle as O
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


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_diagnostics_match_oracle(prec):
    """The oracle sees exactly the values the device array holds."""
    w = I.random_smooth(40, 24, seed=13)
    f = O.set_state(w)
    f = f * (1.0 + 0.01 * np.random.default_rng(5).normal(size=f.shape))
    dtype = torch.float32 if prec == "fp32" else torch.float64
    fd = torch.as_tensor(f, dtype=dtype, device="cuda")
    want = O.diagnostics(w, fd.double().cpu().numpy())
    for _ in range(2):
        got = P.diagnostics_noalloc(w, fd, prec)
        assert got[:6] == pytest.approx(want, rel=TOL[prec], abs=TOL[prec] * want[0])
        assert got[6] == w.n_r * w.n_theta


def test_noalloc_call_leaves_device_memory_alone():
    """After the first call on the device (which loads the library's module,
    static array included), further calls change neither the device's free
    memory nor PyTorch's allocations."""
    w = I.random_smooth(45, 23, seed=22)
    f = torch.as_tensor(O.set_state(w), dtype=torch.float32, device="cuda")
    P.diagnostics_noalloc(w, f, "fp32")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        P.diagnostics_noalloc(w, f, "fp32")
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0


def test_noalloc_refuses_a_capturing_stream():
    """The call waits for its stream and copies to the host, so on a stream
    under capture it returns PCLB_EUNSUPPORTED and queues nothing; the capture
    itself stays valid."""
    w = I.random_smooth(20, 12, seed=23)
    f = torch.as_tensor(O.set_state(w), dtype=torch.float32, device="cuda")
    x = torch.zeros(4, device="cuda")
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        x.add_(1.0)
        with pytest.raises(P.PCLBError) as e:
            P.diagnostics_noalloc(w, f, "fp32", stream=s)
    assert e.value.code == 8 and "captured" in str(e.value)
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(x.cpu(), torch.ones(4))
    got = P.diagnostics_noalloc(w, f, "fp32")   # an ordinary call afterwards still works
    assert got[6] == w.n_r * w.n_theta


def test_noalloc_rejects_grids_beyond_its_scratch():
    w = I.random_smooth(8, 16385, seed=3)
    f = torch.zeros((33, 16385, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(P.PCLBError) as e:
        P.diagnostics_noalloc(w, f, "fp32")
    assert e.value.code == 1 and "16384" in str(e.value)
