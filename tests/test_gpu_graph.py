"""pclb_step_graph: the steps of pclb_step launched as one captured CUDA
graph give bitwise the same states, for odd and even step counts (the
ping-pong buffers), on replay, interleaved with plain steps, after a scheme
change (which drops the captured graphs), and for the generic velocity-set
kernels."""
import numpy as np
import pytest

import oracle as O
from paper_1302_7104_gb300 import inputs as I
from paper_1302_7104_gb300 import pclb as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _f0(w, dtype, seed=11):
    f = O.set_state(w)
    f = f * (1.0 + 0.01 * np.random.default_rng(seed).normal(size=f.shape))
    return torch.as_tensor(f, dtype=dtype, device="cuda")


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_graph_steps_equal_plain_steps(prec):
    w = I.random_smooth(70, 35, seed=41, bc_kind=(I.BC_WALL, I.BC_DIRICHLET))
    dtype = torch.float32 if prec == "fp32" else torch.float64
    f0 = _f0(w, dtype)
    with P.PCLB(w, precision=prec) as a, P.PCLB(w, precision=prec) as b:
        a.set_f(f0)
        b.set_f(f0)
        # odd and even counts, replays (the second 3 and 2 hit the cache),
        # and a plain step in between (changes the starting buffer)
        for n, plain in ((3, False), (2, False), (3, False), (1, True), (2, False), (5, False)):
            a.step(n)
            if plain:
                b.step(n)
            else:
                b.step_graph(n)
            assert torch.equal(a.get_f(), b.get_f()), n
        assert a.status_flags() == 0 and b.status_flags() == 0


def test_graph_follows_a_scheme_change():
    w = I.random_smooth(40, 24, seed=42)
    f0 = _f0(w, torch.float64)
    with P.PCLB(w, precision="fp64") as a, P.PCLB(w, precision="fp64") as b:
        a.set_f(f0).step(2)
        b.set_f(f0).step_graph(2)
        a.set_scheme(P.SCHEME_LW, P.RELAX_EULER).step(2)
        b.set_scheme(P.SCHEME_LW, P.RELAX_EULER).step_graph(2)
        assert torch.equal(a.get_f(), b.get_f())


def test_graph_with_the_generic_velocity_set():
    w = I.random_smooth(37, 19, seed=43, n_dirs=16, n_f=16)
    f0 = _f0(w, torch.float64)
    with P.PCLB(w, precision="fp64") as a, P.PCLB(w, precision="fp64") as b:
        a.set_f(f0).step(3)
        b.set_f(f0).step_graph(3)
        assert torch.equal(a.get_f(), b.get_f())
