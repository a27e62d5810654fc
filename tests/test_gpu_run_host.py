"""pclb_run_host with page-locked buffers: the host transfers run slab by slab
(azimuthal slabs of whole tile rows) on copy streams under the set-state,
step and moment kernels of other slabs.  The fields it returns equal, bit for
bit, those of the device path (the same entry points on device tensors, whole
grid) for 0 to 3 steps, with 4 slabs (the last of one row) and 16 slabs (a
ragged last tile), outputs omitted, outputs that alias the inputs, a sector
grid and a non-default scheme."""
import pytest

from paper_1302_7104_gb300 import inputs as I
from paper_1302_7104_gb300 import pclb as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# (n_r, n_theta): 524,300 nodes and 4 tile rows -> 4 slabs, rows 16/16/16/1;
# 2,109,440 nodes and 65 tile rows -> 16 slabs, the last tile 6 rows high
CASES = [(10700, 49), (2048, 1030)]


def _dtype(prec):
    return torch.float32 if prec == "fp32" else torch.float64


def _pinned(w, dtype):
    return [torch.as_tensor(x, dtype=dtype).pin_memory() for x in w.fields()]


def _device_path(g, ins, n):
    g.set_state(*[x.cuda() for x in ins]).step(n)
    return [x.cpu() for x in g.moments()]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("n_r,n_theta", CASES)
def test_slabs_equal_the_device_path(prec, n_r, n_theta):
    w = I.random_smooth(n_r, n_theta, seed=51, bc_kind=(I.BC_WALL, I.BC_EXTRAP))
    dtype = _dtype(prec)
    ins = _pinned(w, dtype)
    with P.PCLB(w, precision=prec) as g:
        for n in (0, 1, 2, 3):
            want = _device_path(g, ins, n)
            outs = [torch.full((n_theta, n_r), float("nan"), dtype=dtype).pin_memory() for _ in range(4)]
            got = g.run_host(*ins, n, outs)
            for a, b in zip(got, want):
                assert torch.equal(a, b), n
        assert g.status_flags() == 0


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_omitted_and_aliased_outputs(prec):
    n_r, n_theta = CASES[0]
    w = I.random_smooth(n_r, n_theta, seed=52, bc_kind=(I.BC_EXTRAP, I.BC_DIRICHLET))
    dtype = _dtype(prec)
    ins = _pinned(w, dtype)
    with P.PCLB(w, precision=prec) as g:
        want = _device_path(g, ins, 1)
        # only u_theta and T asked for
        outs = [None, None] + [torch.zeros((n_theta, n_r), dtype=dtype).pin_memory() for _ in range(2)]
        got = g.run_host(*ins, 1, outs)
        assert torch.equal(got[2], want[2]) and torch.equal(got[3], want[3])
        # results written over the inputs (each slab is read before it is written)
        alias = [x.clone().pin_memory() for x in ins]
        got = g.run_host(*alias, 1, alias)
        for a, b in zip(got, want):
            assert torch.equal(a, b)


def test_sector_grid_and_scheme():
    """A quarter sector (rotated labels at the azimuthal seam) under the
    Lax-Wendroff scheme with forward-Euler relaxation, 2 steps."""
    w = I.random_smooth(9000, 60, seed=53, n_f=2, bc_kind=(I.BC_WALL, I.BC_WALL))
    ins = _pinned(w, torch.float32)
    with P.PCLB(w, precision="fp32") as g:
        g.set_scheme(P.SCHEME_LW, P.RELAX_EULER)
        want = _device_path(g, ins, 2)
        got = g.run_host(*ins, 2, [torch.empty_like(x).pin_memory() for x in ins])
        for a, b in zip(got, want):
            assert torch.equal(a, b)


def test_nonphysical_input_is_flagged():
    """A row with rho <= 0 inside a middle slab: the pipelined call completes
    and the status word reports the non-physical state."""
    n_r, n_theta = CASES[0]
    w = I.random_smooth(n_r, n_theta, seed=54)
    ins = _pinned(w, torch.float32)
    ins[0][20, 100:110] = -1.0          # row 20 lies in the second of the four slabs
    outs = [torch.empty_like(x).pin_memory() for x in ins]
    with P.PCLB(w, precision="fp32") as g:
        g.run_host(*ins, 1, outs)
        assert g.status_flags() & P.FLAG_NONPHYS


def test_on_the_legacy_default_stream():
    """A context on the legacy default stream (handle 0): the copy streams
    are ordered against it by events only, and the results still equal the
    device path."""
    n_r, n_theta = CASES[0]
    w = I.random_smooth(n_r, n_theta, seed=55)
    ins = _pinned(w, torch.float32)
    with P.PCLB(w, precision="fp32", stream=torch.cuda.default_stream()) as g:
        assert g.stream.cuda_stream == 0
        want = _device_path(g, ins, 1)
        got = g.run_host(*ins, 1, [torch.empty_like(x).pin_memory() for x in ins])
        for a, b in zip(got, want):
            assert torch.equal(a, b)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("n_r,n_theta,n_dirs", [(3, 2, 8), (37, 17, 8), (40, 24, 16)])
def test_small_grids_and_the_generic_set(prec, n_r, n_theta, n_dirs):
    """One slab whose stencil rows wrap around the seam (3 x 2), a last slab of
    one row (37 x 17: two slabs), and N_i = 16 (page-locked buffers, which
    take the sequential path for the generic kernels): 0 to 2 steps."""
    w = I.random_smooth(n_r, n_theta, seed=56, n_dirs=n_dirs, n_f=n_dirs)
    dtype = _dtype(prec)
    ins = _pinned(w, dtype)
    with P.PCLB(w, precision=prec) as g:
        for n in (0, 1, 2):
            want = _device_path(g, ins, n)
            got = g.run_host(*ins, n, [torch.empty_like(x).pin_memory() for x in ins])
            for a, b in zip(got, want):
                assert torch.equal(a, b), n
        assert g.status_flags() == 0
