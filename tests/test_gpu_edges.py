"""Edge cases of the CUDA path through the C ABI: zero steps, interleaved
contexts on one stream, a large grid ragged in both directions (sampled nodes
against the oracle), a sector of one period with walls on a ragged grid, and
forward and adjoint steps interleaved on the caller's stream (the adjoint's
wall work runs on a side stream joined back before the next launch)."""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_1302_7104_gb300 import inputs as I
from paper_1302_7104_gb300 import pclb as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _noisy(w, seed=11, scale=0.01):
    f = O.set_state(w)
    return np.ascontiguousarray(f * (1.0 + scale * np.random.default_rng(seed).normal(size=f.shape)))


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_zero_steps_change_nothing(prec):
    w = I.random_smooth(37, 19, seed=31)
    dtype = torch.float32 if prec == "fp32" else torch.float64
    f0 = torch.as_tensor(_noisy(w), dtype=dtype, device="cuda")
    with P.PCLB(w, precision=prec) as g:
        a = g.set_f(f0).step(0).get_f()
        assert torch.equal(a, f0)
        host = g.run_host(*[torch.as_tensor(x, dtype=dtype) for x in w.fields()], 0)
        dev = [x.cpu() for x in g.set_state().moments()]
    for x, y in zip(host, dev):
        assert torch.equal(x, y)


def test_interleaved_contexts_are_independent():
    wa = I.random_smooth(40, 24, seed=32, bc_kind=(I.BC_DIRICHLET, I.BC_WALL))
    wb = I.random_smooth(33, 17, seed=33, n_f=3)
    fa, fb = _noisy(wa, 1), _noisy(wb, 2)
    with P.PCLB(wa, precision="fp64") as ga, P.PCLB(wb, precision="fp64") as gb:
        ga.set_f(torch.as_tensor(fa, device="cuda"))
        gb.set_f(torch.as_tensor(fb, device="cuda"))
        for _ in range(3):
            ga.step(1)
            gb.step(1)
        got_a, got_b = ga.get_f().cpu().numpy(), gb.get_f().cpu().numpy()
    for w, f, got in ((wa, fa, got_a), (wb, fb, got_b)):
        want = O.run(w, f, 3)
        assert np.max(np.abs(got - want)) / np.max(np.abs(want)) <= 1e-12


def _sample(w, seed=5):
    nt, nr = w.n_theta, w.n_r
    rng = np.random.default_rng(seed)
    it, ir = [], []
    for c in (0, 1, 2, 3, nr - 4, nr - 3, nr - 2, nr - 1):   # walls
        rows = rng.integers(0, nt, 24)
        it += list(rows) + [0, 1, nt - 2, nt - 1]
        ir += [c] * (len(rows) + 4)
    for t in (0, 1, 2, 3, nt - 4, nt - 3, nt - 2, nt - 1):   # seam rows
        cols = rng.integers(0, nr, 24)
        it += [t] * len(cols)
        ir += list(cols)
    # the ragged last tile in r (columns past the last multiple of 32) and in theta
    it += list(rng.integers(0, nt, 128))
    ir += list(rng.integers(32 * (nr // 32) - 2, nr, 128))
    it += list(rng.integers(16 * (nt // 16) - 2, nt, 128))
    ir += list(rng.integers(0, nr, 128))
    it += list(rng.integers(0, nt, 512))
    ir += list(rng.integers(0, nr, 512))
    return np.asarray(it, dtype=np.int64), np.asarray(ir, dtype=np.int64)


@pytest.mark.parametrize("prec,tol", [("fp32", 2e-6), ("fp64", 1e-12)])
def test_large_ragged_grid_sampled_nodes_match_oracle(prec, tol):
    # 1999 x 1013: 63 tiles in r with a 15-node tail, 64 tiles in theta with a 5-row tail
    w = I.random_smooth(1999, 1013, seed=34, bc_kind=(I.BC_WALL, I.BC_DIRICHLET))
    f = _noisy(w, 3)
    if prec == "fp32":
        f = f.astype(np.float32).astype(np.float64)
    dtype = torch.float32 if prec == "fp32" else torch.float64
    it, ir = _sample(w)
    with P.PCLB(w, precision=prec) as g:
        got_f = g.set_f(torch.as_tensor(f, dtype=dtype, device="cuda")).step(1).get_f()
        assert g.status_flags() == 0
        got = got_f[:, torch.as_tensor(it, device="cuda"), torch.as_tensor(ir, device="cuda")].double().cpu().numpy().T
    want = O.step_nodes(w, f, it, ir)
    assert np.max(np.abs(got - want)) / np.max(np.abs(f)) <= tol


def test_forward_and_adjoint_interleave_on_the_stream():
    """Alternating steps and adjoint steps on one stream equal the same calls
    made one by one with a synchronisation after each."""
    w = I.random_smooth(70, 36, seed=35, bc_kind=(I.BC_WALL, I.BC_EXTRAP))
    f0 = torch.as_tensor(_noisy(w), device="cuda")
    lam0 = torch.as_tensor(np.random.default_rng(4).normal(size=(w.q, w.n_theta, w.n_r)), device="cuda")

    def run(sync):
        with P.PCLB(w, precision="fp64") as g:
            g.set_f(f0)
            g.lambda_set(lam0)
            for _ in range(3):
                st = g.save_state()
                g.step(1)
                if sync:
                    g.sync()
                g.adjoint_state(st)
                if sync:
                    g.sync()
            return g.get_f().cpu(), g.lambda_get().cpu()

    a_f, a_l = run(False)
    b_f, b_l = run(True)
    assert torch.equal(a_f, b_f) and torch.equal(a_l, b_l)


def test_alu_peaks_are_plausible():
    """The benchmark's multiply-add rate helper: packed FP32 and FP64 rates
    within a factor of a few of GB300's nominal rates (152 SMs at up to
    2.07 GHz: 80 and 1.26 TFLOP/s)."""
    import bench
    P.lib()   # builds the product and the benchmark helper library
    pk = bench._alu_peaks(torch.cuda.current_stream())
    assert 20.0 < pk["ffma2_tflops"] < 120.0
    assert 0.3 < pk["dfma_tflops"] < 3.0


@pytest.mark.parametrize("prec,n_dirs", [("fp32", 8), ("fp64", 8), ("fp64", 16)])
def test_step_states_equals_step(prec, n_dirs):
    """pclb_step_states: one step between saved-state buffers equals pclb_step
    bit for bit and leaves the context's own state alone."""
    w = I.random_smooth(45, 21, seed=36, n_dirs=n_dirs, n_f=n_dirs, bc_kind=(I.BC_WALL, I.BC_EXTRAP))
    dtype = torch.float32 if prec == "fp32" else torch.float64
    with P.PCLB(w, precision=prec) as g:
        g.set_f(torch.as_tensor(_noisy(w), dtype=dtype, device="cuda"))
        s0 = g.save_state()
        s1, s2 = g.new_state(), g.new_state()
        g.step_states(s0, s1).step_states(s1, s2)
        assert torch.equal(g.save_state(), s0)          # the context's state is untouched
        want = g.step(2).get_f()
        got = g.load_state(s2).get_f()                  # the nodes (buffer padding is not state)
        assert torch.equal(got, want)


def test_misaligned_pointers_are_refused_before_any_launch():
    """Pointers the kernels would read or write element by element must be
    aligned to the element size: a misaligned one is refused on the host
    (PCLB_EINVAL) and nothing is launched."""
    import ctypes
    w = I.random_smooth(20, 12, seed=37)
    with P.PCLB(w, precision="fp32") as g:
        g.set_state()
        buf = torch.zeros(4 * w.n_theta * w.n_r + 4, dtype=torch.float32, device="cuda")
        bad = ctypes.c_void_p(buf.data_ptr() + 2)
        ok = ctypes.c_void_p(buf.data_ptr())
        assert P.lib().pclb_set_state(g.ctx, bad, ok, ok, ok) == 1
        assert P.lib().pclb_moments(g.ctx, bad, None, None, None) == 1
        f = torch.zeros(w.q * w.n_theta * w.n_r + 4, dtype=torch.float32, device="cuda")
        assert P.lib().pclb_get_f(g.ctx, ctypes.c_void_p(f.data_ptr() + 2)) == 1
        st = g.new_state()
        assert P.lib().pclb_adjoint_state(g.ctx, ctypes.c_void_p(st.data_ptr() + 8)) in (1, 8)
        assert g.status_flags() == 0


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_window_wait_that_runs_out_reports_timeout(prec):
    """A step whose wait for its own window copies runs out (limit 0: every
    tile is given up without waiting) sets PCLB_FLAG_TIMEOUT;
    pclb_status_flags returns PCLB_ETIMEOUT; the context stays usable: with
    the default limit restored, a reloaded state steps exactly as a fresh
    context does.  Nothing faults or hangs: the copies of a tile given up get
    the default limit to land before its block exits."""
    w = I.kh(n_r=1024, n_theta=512)
    dtype = torch.float32 if prec == "fp32" else torch.float64
    f0 = torch.as_tensor(O.set_state(w), dtype=dtype, device="cuda")
    with P.PCLB(w, precision=prec) as g:
        g.set_f(f0).set_wait_limit(0).step(3)
        flags = ctypes.c_uint32()
        code = P.lib().pclb_status_flags(g.ctx, ctypes.byref(flags), 1)
        assert code == 5 and flags.value & P.FLAG_TIMEOUT, (code, flags.value)
        with pytest.raises(P.PCLBError):
            g.set_wait_limit(61_000_000_000)          # above the maximum
        g.set_wait_limit().set_f(f0).step(2)
        assert g.status_flags() == 0
        got = g.get_f()
    with P.PCLB(w, precision=prec) as h:
        want = h.set_f(f0).step(2).get_f()
    assert torch.equal(got, want)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_adjoint_window_wait_that_runs_out_reports_timeout(prec):
    """The adjoint kernels give a tile up the same way when the wait for its
    f and lam windows runs out: PCLB_FLAG_TIMEOUT, PCLB_ETIMEOUT from
    pclb_status_flags, and with the default limit restored the next adjoint
    step equals a fresh context's bit for bit."""
    w = I.kh(n_r=1024, n_theta=512)
    dtype = torch.float32 if prec == "fp32" else torch.float64
    f0 = torch.as_tensor(O.set_state(w), dtype=dtype, device="cuda")
    gen = torch.Generator(device="cpu").manual_seed(11)
    lam = torch.randn(f0.shape, generator=gen, dtype=torch.float64).to(dtype=dtype, device="cuda")
    with P.PCLB(w, precision=prec) as g:
        g.set_wait_limit(0)
        g.adjoint_step(f0, lam)
        flags = ctypes.c_uint32()
        code = P.lib().pclb_status_flags(g.ctx, ctypes.byref(flags), 1)
        assert code == 5 and flags.value & P.FLAG_TIMEOUT, (code, flags.value)
        g.set_wait_limit()
        got = g.adjoint_step(f0, lam)
        g.sync()
        assert g.status_flags() == 0
    with P.PCLB(w, precision=prec) as h:
        want = h.adjoint_step(f0, lam)
        h.sync()
    assert torch.equal(got, want)


@pytest.mark.parametrize("n_dirs", [16, 24])
def test_tiled_step_wait_that_runs_out_reports_timeout(n_dirs):
    """The FP32 step of the 16- and 24-direction sets (plane pairs streamed
    through a TMA ring) gives a tile up the same way when a wait runs out:
    PCLB_FLAG_TIMEOUT, PCLB_ETIMEOUT, and with the default limit restored a
    reloaded state steps bit for bit like a fresh context."""
    w = I.random_smooth(200, 96, seed=31, n_dirs=n_dirs, n_f=n_dirs)
    f0 = torch.as_tensor(O.set_state(w), dtype=torch.float32, device="cuda")
    with P.PCLB(w, precision="fp32") as g:
        g.set_f(f0).set_wait_limit(0).step(2)
        flags = ctypes.c_uint32()
        code = P.lib().pclb_status_flags(g.ctx, ctypes.byref(flags), 1)
        assert code == 5 and flags.value & P.FLAG_TIMEOUT, (code, flags.value)
        g.set_wait_limit().set_f(f0).step(3)
        assert g.status_flags() == 0
        got = g.get_f()
    with P.PCLB(w, precision="fp32") as h:
        want = h.set_f(f0).step(3).get_f()
    assert torch.equal(got, want)


def test_host_sync_that_runs_out_reports_timeout():
    """pclb_sync with a limit shorter than the queued work returns
    PCLB_ETIMEOUT and leaves the work running; a second sync with the default
    limit waits it out."""
    w = I.kh(n_r=4096, n_theta=4096)
    with P.PCLB(w, precision="fp32") as g:
        g.set_state()
        g.sync()
        g.step(30)                                      # about 35 ms of work
        assert P.lib().pclb_sync(g.ctx, 1) == 5         # PCLB_ETIMEOUT after 1 ms
        assert "did not finish" in P.lib().pclb_last_error(g.ctx).decode()
        g.sync()
        assert g.status_flags() == 0
