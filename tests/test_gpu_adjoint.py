"""GPU parity of the leakage-calibration model and its adjoint (polaris_adj_*): Stokes and
loss against the FP64 oracle, gradients against the oracle's FP64 gradient (itself pinned by
central differences), and the torch.autograd wrapper against the direct call."""
import numpy as np
import pytest

from paper_1412_1256_gb300 import synth

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("logn,bits,nseg", [(6, 8, 6), (10, 2, 12), (14, 8, 8)])
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
    for got, ref in ((r["grad_window"], gw_ref), (r["grad_gains"], gg_ref), (r["grad_leak"], gd_ref)):
        got = got.cpu().numpy().astype(np.float64)
        assert np.abs(got - ref).max() <= 2e-3 * np.abs(ref).max()


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
        assert float(loss.detach()) == pytest.approx(float(direct["loss"][0]), rel=1e-6)
        # two runs accumulate their float atomics in different orders: agreement to ~1e-5
        for got, ref in ((W.grad, direct["grad_window"]), (G.grad, direct["grad_gains"]), (D.grad, direct["grad_leak"])):
            assert float((got - 2.0 * ref).abs().max()) <= 1e-4 * float(ref.abs().max() * 2.0)


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
