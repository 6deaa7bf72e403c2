"""GPU checks of the exact energy gradient (reverse-mode adjoint) and its autograd binding:
against the FP64 oracle's reverse-mode gradient, against central finite differences of the
library's own energy, with and without checkpointed forward maps, on a batch of 128^3 pairs."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_02060_gb300 import build
    build.build()
    from paper_1605_02060_gb300 import lddmm as L
    L.load()
    return L


def _blobs(shape):
    Z, Y, X = shape
    gz, gy, gx = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    I0 = np.exp(-((gx - X / 2) ** 2 / 12 + (gy - Y / 2) ** 2 / 9 + (gz - Z / 2) ** 2 / 7))
    I1 = np.exp(-((gx - X / 2 - 1) ** 2 / 10 + (gy - Y / 2) ** 2 / 9 + (gz - Z / 2 + 0.5) ** 2 / 8))
    return I0.astype(np.float32), I1.astype(np.float32)


@pytest.mark.parametrize("flags", [0, 2])
@pytest.mark.parametrize("shape,T", [((8, 8, 8), 3), ((11, 9, 13), 5)])
def test_gradient_matches_oracle(L, shape, T, flags):
    from oracle import lddmm as O
    from paper_1605_02060_gb300 import synth
    I0, I1 = _blobs(shape)
    M = (0.5 + 0.5 * np.random.default_rng(3).random(shape)).astype(np.float32)
    v = synth.smooth_velocity(T, shape, 0.8, seed=8)
    h = (1.0, 1.1, 0.9)
    Z, Y, X = shape
    p = L.default_params(X, Y, Z, T=T, sigma=0.5, alpha=0.05, hx=h[0], hy=h[1], hz=h[2], flags=flags)
    po = O.Params(T=T, sigma=0.5, alpha=0.05, h=h)
    Eo, go = O.energy_grad_exact(v, I0, I1, M, po)
    with L.Lddmm(p, I0, I1, M) as ctx:
        E, g = ctx.energy_grad(v)
    assert abs(E - Eo) <= 1e-5 * abs(Eo)
    assert _rel(g, go) < 1e-4


def test_autograd_function_and_finite_differences(L):
    from paper_1605_02060_gb300 import synth
    from paper_1605_02060_gb300.autograd import LddmmEnergy
    pair = synth.ellipsoid_pair(seed=0)
    T = 10
    p = L.default_params(32, 32, 32, T=T)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    with L.Lddmm(p, dev(pair.I0), dev(pair.I1), dev(pair.M)) as ctx:
        v = dev(synth.smooth_velocity(T, (32, 32, 32), 1.5, seed=21)).requires_grad_(True)
        E = LddmmEnergy.apply(v, ctx)
        E.backward()
        g = v.grad.detach().clone()
        E2, g2 = ctx.energy_grad(v.detach(), torch.empty_like(g))
        assert abs(float(E.detach()) - E2) <= 1e-9 * abs(E2)
        assert _rel(g.cpu().numpy(), g2.cpu().numpy()) < 1e-5    # atomics: FP32 rounding only
        rng = np.random.default_rng(5)
        hstep = 1e-3
        for k in range(4):
            d = dev(synth.smooth_velocity(T, (32, 32, 32), 1.0, seed=100 + k))
            Ep = float(LddmmEnergy.apply(v.detach() + hstep * d, ctx))
            Em = float(LddmmEnergy.apply(v.detach() - hstep * d, ctx))
            fd = (Ep - Em) / (2 * hstep)
            an = float((g.double() * d.double()).sum())
            assert abs(fd - an) <= 2e-2 * abs(an) + 1e-6, (k, fd, an)


def test_batch_of_128cubed_pairs_fd_16_directions(L):
    """Eight independent 128^3 ellipsoid-union pairs (T = 10): the adjoint gradient of each,
    with checkpointed maps, checked by central finite differences on 16 random smooth
    directions in total (h = 1e-3), two per pair."""
    from paper_1605_02060_gb300 import synth
    from paper_1605_02060_gb300.autograd import LddmmEnergy
    T = 10
    shape = (128, 128, 128)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    worst = 0.0
    for i in range(8):
        pair = synth.union_pair(shape, seed=100 + i, amplitude=5.0)
        p = L.default_params(128, 128, 128, T=T, flags=2)
        with L.Lddmm(p, dev(pair.I0), dev(pair.I1), dev(pair.M)) as ctx:
            for _ in range(5):
                ctx.step(want_energy=False)       # move away from v = 0
            v = torch.empty((T, 3) + shape, device="cuda")
            ctx.get_velocity(v)
            v.requires_grad_(True)
            E = LddmmEnergy.apply(v, ctx)
            E.backward()
            g = v.grad.detach()
            for k in range(2):
                d = dev(synth.smooth_velocity(T, shape, 1.0, seed=200 + 2 * i + k))
                Ep = float(LddmmEnergy.apply(v.detach() + 1e-3 * d, ctx))
                Em = float(LddmmEnergy.apply(v.detach() - 1e-3 * d, ctx))
                fd = (Ep - Em) / 2e-3
                an = float((g.double() * d.double()).sum())
                worst = max(worst, abs(fd - an) / abs(an))
    assert worst < 5e-2, worst
