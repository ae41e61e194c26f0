"""GPU parity of the leakage-calibration model and its adjoint (polaris_adj_*): Stokes and
loss against the FP64 oracle, gradients against the oracle's FP64 gradient (itself pinned by
central differences) element by element and against central differences of the FP64 oracle
loss, and the torch.autograd wrapper against the direct call.

Gradient bound, per element: |g - g_ref| <= 1e-3 |g_ref| + 4e-6 max|g_ref| (max over the
gradient's family: window taps, gains or leakage terms).  The relative part is the 1e-3 the
calibration asks for; the floor covers elements that nearly cancel.  An FP32 transform of
log2 N <= 14 radix-2 stages gives the spectral sums a relative error of up to about
log2 N * 2^-24 = 8.3e-7; a leakage-gradient element adds four products of those sums
(2a|gR|^2 B DR, 2a|gR|^2 C, c conj(gR) gL B, c conj(gR) gL DL C), none larger than its
family's largest element, so one that cancels keeps up to about 4 x 8.3e-7 = 3.3e-6 of that
maximum (measured: up to 2.0e-6 of it over 500-520 random segments at 2^14, with either
kernel set; the median relative error of the gradients is 3e-7..1.5e-6)."""
import numpy as np
import pytest

from paper_1412_1256_gb300 import synth

pytestmark = pytest.mark.gpu
REL, FLOOR = 1e-3, 4e-6


def _assert_grad(got, ref, what):
    got = np.asarray(got, np.float64).reshape(-1)
    ref = np.asarray(ref, np.float64).reshape(-1)
    bound = REL * np.abs(ref) + FLOOR * np.abs(ref).max()
    bad = np.abs(got - ref) > bound
    assert not bad.any(), (what, int(bad.sum()), float(np.max(np.abs(got - ref) / bound)))


def _fd_checks(orc, host, bits, n_fft, n, w, g, d, target, r, taps, leaks, h=1e-3):
    """The GPU gradient against central differences (step h) of the FP64 oracle loss, for the
    four gain components, the given window taps and the given leakage terms, within 1e-3
    relative.  The loss is a quartic polynomial in each parameter, so the truncation error
    h^2 f'''/6 stays far below that."""
    w64, g64, d64 = (np.asarray(x, np.float64) for x in (w, g, d))

    def L(w_, g_, d_):
        return orc.leak_forward(host, bits, n_fft, n, w_, g_, d_, target)[1]

    ggr, gwr, gdr = (r[k].cpu().numpy().astype(np.float64) for k in ("grad_gains", "grad_window", "grad_leak"))
    for i in range(4):
        e = np.zeros(4)
        e[i] = h
        fd = (L(w64, g64 + e, d64) - L(w64, g64 - e, d64)) / (2 * h)
        assert ggr[i] == pytest.approx(fd, rel=REL), ("gain", i)
    for i in taps:
        e = np.zeros(n_fft)
        e[i] = h
        fd = (L(w64 + e, g64, d64) - L(w64 - e, g64, d64)) / (2 * h)
        assert gwr[i] == pytest.approx(fd, rel=REL), ("tap", i)
    for (f, k, c) in leaks:
        e = np.zeros_like(d64)
        e[f, k, c] = h
        fd = (L(w64, g64, d64 + e) - L(w64, g64, d64 - e)) / (2 * h)
        assert gdr[f, k, c] == pytest.approx(fd, rel=REL), ("leak", f, k, c)


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_1256_gb300 import polaris

    polaris.load()
    return torch, polaris


def _case(torch, n_fft, nseg, bits, seed):
    rng = np.random.default_rng(seed)
    n = n_fft * nseg
    if bits == 8:
        host = [synth.pack(synth.quantize_int8(rng.standard_normal(n) * 20.0), 8) for _ in range(2)]
    else:
        host = [synth.pack(synth.quantize(rng.standard_normal(n), bits), bits) for _ in range(2)]
    nbin = n_fft // 2 + 1
    w = 0.5 - 0.5 * np.cos(2 * np.pi * np.arange(n_fft) / n_fft) + 0.05 * rng.standard_normal(n_fft)
    mag, ph = rng.uniform(0.8, 1.2, 2), rng.uniform(-np.pi, np.pi, 2)
    gains = np.array([mag[0] * np.cos(ph[0]), mag[0] * np.sin(ph[0]), mag[1] * np.cos(ph[1]), mag[1] * np.sin(ph[1])])
    leak = rng.uniform(-0.035, 0.035, (2, nbin, 2))
    # float32 copies (what the GPU sees); the oracle runs on the same rounded values
    w32, g32, d32 = (x.astype(np.float32) for x in (w, gains, leak))
    dev = [torch.from_numpy(h.view(np.int32)).cuda() for h in host]
    return host, dev, n, w32, g32, d32


def _t(torch, x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


# log2 N 6 runs the kernels for any N, 9..14 the size-specialised ones (every width; at 2^9
# and 2^12 more segments than the grid has CTAs, so that each CTA sums several)
@pytest.mark.parametrize("logn,bits,nseg", [(6, 8, 6), (9, 1, 1300), (10, 2, 12), (11, 4, 10), (12, 2, 500),
                                            (13, 4, 5), (14, 8, 8), (14, 1, 3)])
def test_forward_and_gradients_match_oracle(env, orc, logn, bits, nseg):
    torch, pol = env
    n_fft = 1 << logn
    host, dev, n, w, g, d = _case(torch, n_fft, nseg, bits, 40 + logn)
    st_ref, _ = orc.leak_forward(host, bits, n_fft, n, w, g, d)
    rng = np.random.default_rng(9)
    target = (st_ref * 0.9 + rng.standard_normal(st_ref.shape) * 0.05 * np.abs(st_ref).mean()).astype(np.float32)
    _, loss_ref = orc.leak_forward(host, bits, n_fft, n, w, g, d, target)
    gw_ref, gg_ref, gd_ref = orc.leak_grad(host, bits, n_fft, n, w, g, d, target)
    with pol.Adjoint(n_fft, bits) as adj:
        r = adj.run(dev, n, _t(torch, w), _t(torch, g), _t(torch, d), _t(torch, target), grads=True)
        torch.cuda.synchronize()
    st = r["stokes"].cpu().numpy()
    scale = np.abs(st_ref).max()
    assert np.abs(st - st_ref).max() <= 1e-5 * scale
    assert float(r["loss"].cpu()[0]) == pytest.approx(loss_ref, rel=1e-3)
    for name, got, ref in (("window", r["grad_window"], gw_ref), ("gains", r["grad_gains"], gg_ref),
                           ("leak", r["grad_leak"], gd_ref)):
        _assert_grad(got.cpu().numpy(), ref, name)


def test_every_run_writes_loss_and_gain_gradients(env, orc):
    """A sequence of runs on one handle (loss only, Stokes only, with gradients twice, loss
    only) writes the loss and the gain gradients on every run that asks for them, into
    outputs that start as NaN, and no loss on the run that does not: bitwise equal from run
    to run (every sum has a fixed order) and equal to the oracle's."""
    import ctypes

    torch, pol = env
    n_fft, nseg, bits = 1 << 12, 40, 2
    host, dev, n, w, g, d = _case(torch, n_fft, nseg, bits, 77)
    st_ref, _ = orc.leak_forward(host, bits, n_fft, n, w, g, d)
    target = (st_ref * 0.95).astype(np.float32)
    _, loss_ref = orc.leak_forward(host, bits, n_fft, n, w, g, d, target)
    _, gg_ref, _ = orc.leak_grad(host, bits, n_fft, n, w, g, d, target)
    lib = pol.load()
    nb = n_fft // 2 + 1
    W, G, D, T = (_t(torch, x) for x in (w, g, d, target))
    arr = (ctypes.c_void_p * 2)(*[p.data_ptr() for p in dev])
    nan = float("nan")
    losses, gains = [], []
    with pol.Adjoint(n_fft, bits) as adj:
        for kind in ("loss", "stokes", "grads", "grads", "loss"):
            st = torch.full((4, nb), nan, device="cuda")
            loss = torch.full((1,), nan, dtype=torch.float64, device="cuda")
            gw = torch.full((n_fft,), nan, device="cuda")
            gg = torch.full((4,), nan, device="cuda")
            gd = torch.full((2, nb, 2), nan, device="cuda")
            grads = kind == "grads"
            rc = lib.polaris_adj_run(adj._h, arr, n, W.data_ptr(), G.data_ptr(), D.data_ptr(),
                                     None if kind == "stokes" else T.data_ptr(), st.data_ptr(),
                                     None if kind == "stokes" else loss.data_ptr(),
                                     gw.data_ptr() if grads else None, gg.data_ptr() if grads else None,
                                     gd.data_ptr() if grads else None, None)
            assert rc == 0
            torch.cuda.synchronize()
            assert torch.isfinite(st).all(), kind
            if kind == "stokes":
                assert torch.isnan(loss).all()  # not requested, not written
                continue
            losses.append(loss.cpu().numpy().copy())
            assert np.isfinite(losses[-1]).all(), kind
            if grads:
                gains.append(gg.cpu().numpy().copy())
                assert np.isfinite(gains[-1]).all()
    assert all(x.tobytes() == losses[0].tobytes() for x in losses)
    assert gains[0].tobytes() == gains[1].tobytes()
    assert float(losses[0][0]) == pytest.approx(loss_ref, rel=1e-3)
    _assert_grad(gains[0], gg_ref, "gains")


def test_unaligned_buffers_take_the_general_kernels(env, orc):
    """The size-specialised kernels (2^9..2^14) read inputs and window by 16-byte vector loads;
    a call whose buffers are not 16-byte aligned runs the kernels for any N instead, with the
    same results within the bounds above."""
    torch, pol = env
    n_fft, bits, nseg = 4096, 2, 7
    host, dev, n, w, g, d = _case(torch, n_fft, nseg, bits, 51)
    st_ref, _ = orc.leak_forward(host, bits, n_fft, n, w, g, d)
    target = (st_ref * 0.9).astype(np.float32)
    gw_ref, gg_ref, gd_ref = orc.leak_grad(host, bits, n_fft, n, w, g, d, target)
    # the same values one 4-byte element past a 16-byte boundary
    w_off = torch.zeros(n_fft + 1, dtype=torch.float32, device="cuda")[1:]
    w_off.copy_(_t(torch, w))
    dev_off = []
    for x in dev:
        y = torch.zeros(x.numel() + 1, dtype=x.dtype, device="cuda")[1:]
        y.copy_(x)
        dev_off.append(y)
    assert w_off.data_ptr() % 16 and all(y.data_ptr() % 16 for y in dev_off)
    with pol.Adjoint(n_fft, bits) as adj:
        for ins, win in ((dev, _t(torch, w)), (dev_off, w_off)):
            r = adj.run(ins, n, win, _t(torch, g), _t(torch, d), _t(torch, target), grads=True)
            torch.cuda.synchronize()
            assert np.abs(r["stokes"].cpu().numpy() - st_ref).max() <= 1e-5 * np.abs(st_ref).max()
            for name, got, ref in (("window", r["grad_window"], gw_ref), ("gains", r["grad_gains"], gg_ref),
                                   ("leak", r["grad_leak"], gd_ref)):
                _assert_grad(got.cpu().numpy(), ref, name)


def test_many_random_segments_2p14(env, orc):
    """520 random 2-bit segments of 2^14 (each CTA sums three or four): the case that sets the
    gradient floor above (near-cancelling leakage terms keep up to about 2e-6 of their
    family's maximum)."""
    torch, pol = env
    n_fft, bits, nseg = 1 << 14, 2, 520
    host, dev, n, w, g, d = _case(torch, n_fft, nseg, bits, 61)
    st_ref, _ = orc.leak_forward(host, bits, n_fft, n, w, g, d)
    target = (st_ref * 0.9).astype(np.float32)
    gw_ref, gg_ref, gd_ref = orc.leak_grad(host, bits, n_fft, n, w, g, d, target)
    with pol.Adjoint(n_fft, bits) as adj:
        r = adj.run(dev, n, _t(torch, w), _t(torch, g), _t(torch, d), _t(torch, target), grads=True)
        torch.cuda.synchronize()
    assert np.abs(r["stokes"].cpu().numpy() - st_ref).max() <= 1e-5 * np.abs(st_ref).max()
    for name, got, ref in (("window", r["grad_window"], gw_ref), ("gains", r["grad_gains"], gg_ref),
                           ("leak", r["grad_leak"], gd_ref)):
        _assert_grad(got.cpu().numpy(), ref, name)


def test_autograd_wrapper_matches_direct_call(env):
    torch, pol = env
    n_fft, bits = 1024, 8
    host, dev, n, w, g, d = _case(torch, n_fft, 6, bits, 77)
    with pol.Adjoint(n_fft, bits) as adj:
        st = adj.run(dev, n, _t(torch, w), _t(torch, g), _t(torch, d))["stokes"]
        target = (st * 0.8).contiguous()
        direct = adj.run(dev, n, _t(torch, w), _t(torch, g), _t(torch, d), target, grads=True)
        W = _t(torch, w).requires_grad_()
        G = _t(torch, g).requires_grad_()
        D = _t(torch, d).requires_grad_()
        loss = pol.leakage_loss(adj, dev, n, W, G, D, target)
        (2.0 * loss).backward()
        torch.cuda.synchronize()
        # every sum has a fixed order: the two runs agree bit for bit
        assert float(loss.detach()) == float(direct["loss"][0])
        for got, ref in ((W.grad, direct["grad_window"]), (G.grad, direct["grad_gains"]), (D.grad, direct["grad_leak"])):
            assert torch.equal(got, 2.0 * ref)


def test_argument_errors(env):
    torch, pol = env
    with pytest.raises(pol.PolarisError) as ei:
        pol.Adjoint(100, 8)
    assert ei.value.code == pol.EINVAL
    host, dev, n, w, g, d = _case(torch, 64, 2, 8, 1)
    with pol.Adjoint(64, 8) as adj:
        with pytest.raises(pol.PolarisError):
            adj.run(dev, n + 64 // 2, _t(torch, w), _t(torch, g), _t(torch, d))
        with pytest.raises(pol.PolarisError):
            adj.run(dev, n, _t(torch, w), _t(torch, g), _t(torch, d), None, grads=True)


def _params(torch, rng, n_fft):
    nb = n_fft // 2 + 1
    w = (0.5 - 0.5 * np.cos(2 * np.pi * np.arange(n_fft) / n_fft)).astype(np.float32)
    mag, ph = rng.uniform(0.8, 1.2, 2), rng.uniform(-np.pi, np.pi, 2)
    g = np.array([mag[0] * np.cos(ph[0]), mag[0] * np.sin(ph[0]), mag[1] * np.cos(ph[1]), mag[1] * np.sin(ph[1])],
                 dtype=np.float32)
    d = (rng.uniform(0, 0.05, (2, nb)) * np.exp(1j * rng.uniform(-np.pi, np.pi, (2, nb))))
    d = np.stack([d.real, d.imag], -1).astype(np.float32)
    return w, g, d


def test_full_size_circular_source_against_oracle(env, orc):
    """The differentiable workload at full size: 2 circular-feed IFs (int8) carrying a line
    with known fractional Q, U, V, 16384-point segments, 256 of them; injected gains
    (|g| 0.8..1.2) and leakage (|D| <= 0.05); target = the model at other parameters."""
    torch, pol = env
    packed, cfg = synth.config_circular()
    n_fft, n = cfg["n_fft"], cfg["n_samples"]
    rng = np.random.default_rng(5)
    w, g, d = _params(torch, rng, n_fft)
    w0, g0, d0 = _params(torch, rng, n_fft)
    target, _ = orc.leak_forward(packed, 8, n_fft, n, w0, g0, d0)
    target = target.astype(np.float32)
    st_ref, loss_ref = orc.leak_forward(packed, 8, n_fft, n, w, g, d, target)
    gw_ref, gg_ref, gd_ref = orc.leak_grad(packed, 8, n_fft, n, w, g, d, target)
    dev = [torch.from_numpy(p.view(np.int32)).cuda() for p in packed]
    with pol.Adjoint(n_fft, 8) as adj:
        r = adj.run(dev, n, _t(torch, w), _t(torch, g), _t(torch, d), _t(torch, target), grads=True)
        torch.cuda.synchronize()
    st = r["stokes"].cpu().numpy()
    assert np.abs(st - st_ref).max() <= 1e-5 * np.abs(st_ref).max()
    assert float(r["loss"].cpu()[0]) == pytest.approx(loss_ref, rel=1e-3)
    for name, got, ref in (("window", r["grad_window"], gw_ref), ("gains", r["grad_gains"], gg_ref),
                           ("leak", r["grad_leak"], gd_ref)):
        _assert_grad(got.cpu().numpy(), ref, name)
    nb = n_fft // 2 + 1
    _fd_checks(orc, packed, 8, n_fft, n, w, g, d, target, r, taps=(3, 8191, 12371),
               leaks=[(0, 3, 0), (1, nb // 3, 1), (0, nb - 1, 0)])


@pytest.mark.parametrize("logn,bits,nseg", [(6, 8, 6), (8, 8, 24), (10, 2, 12)])
def test_gradients_match_central_differences_of_fp64_loss(env, orc, logn, bits, nseg):
    """d loss / d parameter from the adjoint against central differences (h = 1e-3) of the
    FP64 oracle loss at the same parameters: every gain component, taps and leakage terms
    across the band, DC and Nyquist included, within 1e-3 relative."""
    torch, pol = env
    n_fft = 1 << logn
    host, dev, n, w, g, d = _case(torch, n_fft, nseg, bits, 123 + logn)
    nb = n_fft // 2 + 1
    st_ref, _ = orc.leak_forward(host, bits, n_fft, n, w, g, d)
    target = (st_ref * 0.85).astype(np.float32)  # (the oracle's model, never the GPU's)
    with pol.Adjoint(n_fft, bits) as adj:
        r = adj.run(dev, n, _t(torch, w), _t(torch, g), _t(torch, d), _t(torch, target), grads=True)
        torch.cuda.synchronize()
    _fd_checks(orc, host, bits, n_fft, n, w, g, d, target, r,
               taps=(0, 1, n_fft // 3, n_fft // 2, n_fft - 1),
               leaks=[(0, 0, 0), (0, 3, 0), (1, 7, 1), (0, nb // 2, 1), (1, nb - 1, 0)])


def test_calibration_by_gradient_descent(env):
    """Fitting gains and leakage to target Stokes through torch.autograd and Adam: the loss
    falls by two orders of magnitude and the fitted model reproduces the target."""
    torch, pol = env
    packed, cfg = synth.config_circular(seed=7, n_fft=1024, n_segments=64, center=200.0, fwhm=40.0)
    n_fft, n = cfg["n_fft"], cfg["n_samples"]
    rng = np.random.default_rng(11)
    w, g_true, d_true = _params(torch, rng, n_fft)
    dev = [torch.from_numpy(p.view(np.int32)).cuda() for p in packed]
    with pol.Adjoint(n_fft, 8) as adj:
        target = adj.run(dev, n, _t(torch, w), _t(torch, g_true), _t(torch, d_true))["stokes"].contiguous()
        W = _t(torch, w)
        G = _t(torch, g_true * np.float32(1.06) + np.float32(0.03)).requires_grad_()
        D = _t(torch, d_true * np.float32(0.5)).requires_grad_()
        opt = torch.optim.Adam([G, D], lr=3e-3)
        first = None
        for _ in range(300):
            opt.zero_grad()
            loss = pol.leakage_loss(adj, dev, n, W, G, D, target)
            loss.backward()
            opt.step()
            first = float(loss.detach()) if first is None else first
        final = float(pol.leakage_loss(adj, dev, n, W, G.detach(), D.detach(), target).detach())
        torch.cuda.synchronize()
    assert final < 1e-2 * first
