"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on seeded inputs.

Tolerances (relative L2 unless stated): K and one iteration <= 1e-4 (K in FP32 products:
<= 1e-5), final deformed image after 20 iterations <= 1e-3, labels bit-exact on the same
phi_10, Dice within 0.005.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_02060_gb300 import build
    build.build()
    from paper_1605_02060_gb300 import lddmm as L
    L.load()
    return L


@pytest.fixture(scope="module")
def O():
    from oracle import lddmm as O
    return O


@pytest.fixture(scope="module")
def synth():
    from paper_1605_02060_gb300 import synth
    return synth


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


K_MODES = {"fp32": (0, 1e-5), "bf16x3": (1, 2e-5)}
MODES = ["fp32", "bf16x3"]     # K implementations under test
PROD = K_MODES[MODES[-1]][0]   # the mode the benchmark runs


# --------------------------------------------------------------------------- K operator

@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("shape,h,alpha,gamma", [((32, 32, 32), (1, 1, 1), 0.02, 1.0),
                                                 ((29, 20, 33), (4, 4, 4), 0.02, 1.0),
                                                 ((9, 11, 17), (1.0, 2.0, 0.5), 0.5, 1.7),
                                                 ((2, 3, 5), (1, 1, 1), 1.0, 1.0),
                                                 # x lengths past 256: FP32 tail columns
                                                 ((6, 5, 264), (1, 1, 1), 0.02, 1.0),
                                                 ((4, 7, 260), (1, 1, 1), 0.3, 1.2),
                                                 # y/z passes on split fields: several
                                                 # k-blocks, resident and streamed B, and
                                                 # padded rows (z = 100, 230)
                                                 ((100, 72, 64), (1, 1, 1), 0.3, 1.0),
                                                 ((40, 200, 32), (1, 1, 1), 0.3, 1.0),
                                                 ((230, 24, 16), (1, 1, 1), 0.3, 1.0)])
def test_K_matches_oracle(L, O, mode, shape, h, alpha, gamma):
    code, tol = K_MODES[mode]
    rng = np.random.default_rng(1)
    f = rng.standard_normal(shape).astype(np.float32)
    Z, Y, X = shape
    p = L.default_params(X, Y, Z, hx=h[0], hy=h[1], hz=h[2], alpha=alpha, gamma=gamma, k_mode=code)
    a = np.zeros(shape, np.float32)
    with L.Lddmm(p, a, a) as ctx:
        got = ctx.apply_K(_dev(f))
    ref = O.apply_K(f, alpha, gamma, h)
    assert _rel(got.cpu().numpy() if hasattr(got, "cpu") else got, ref) < tol


@pytest.mark.parametrize("shape", [(32, 32, 32), (29, 20, 33), (228, 160, 264)])
def test_K_plain_bf16_products(L, O, shape):
    """Plain bf16 products (no split): the error of an 8-bit mantissa, ~1e-3 relative."""
    rng = np.random.default_rng(2)
    f = rng.standard_normal(shape).astype(np.float32)
    Z, Y, X = shape
    p = L.default_params(X, Y, Z, k_mode=2)
    a = np.zeros(shape, np.float32)
    with L.Lddmm(p, a, a) as ctx:
        got = ctx.apply_K(_dev(f))
    err = _rel(got, O.apply_K(f, 0.02, 1.0, (1, 1, 1), workers=-1))
    assert 1e-5 < err < 1e-2


def test_K_single_mode_full_size(L):
    X, Y, Z = 264, 160, 228
    k = (7, 3, 11)
    gz, gy, gx = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    f = np.cos(2 * np.pi * (k[0] * gx / X + k[1] * gy / Y + k[2] * gz / Z)).astype(np.float32)
    lam = sum(2 - 2 * np.cos(2 * np.pi * k[d] / n) for d, n in enumerate((X, Y, Z)))
    s = 1.0 / (1.0 + 0.02 * lam) ** 2
    for mode in MODES:
        code, tol = K_MODES[mode]
        p = L.default_params(X, Y, Z, k_mode=code)
        a = np.zeros((Z, Y, X), np.float32)
        with L.Lddmm(p, a, a) as ctx:
            out = torch.empty((Z, Y, X), device="cuda")
            ctx.apply_K(_dev(f), out)
            assert _rel(out.cpu().numpy(), s * f.astype(np.float64)) < 4 * tol


def test_K_tensor_modes_full_size_deterministic(L):
    """At 264x160x228 on random data (all frequencies, every pipeline stage and ring wrap of the
    tensor-core passes): each tensor-core mode gives bit-identical results run to run, and
    agrees with the FP32-product K (itself matched to the oracle above) within its precision:
    bf16x3 1e-4, plain bf16 1e-2."""
    X, Y, Z = 264, 160, 228
    rng = np.random.default_rng(5)
    f = torch.from_numpy(rng.standard_normal((Z, Y, X)).astype(np.float32)).cuda()
    a = torch.zeros((Z, Y, X), device="cuda")
    res = {}
    for code in (0, 1, 2):
        p = L.default_params(X, Y, Z, k_mode=code)
        with L.Lddmm(p, a, a) as ctx:
            runs = []
            for _ in range(2):
                out = torch.empty_like(f)
                ctx.apply_K(f, out)
                runs.append(out)
            torch.cuda.synchronize()
        assert torch.equal(runs[0], runs[1]), "k_mode %d is not deterministic" % code
        res[code] = runs[0].double()
    ref = res[0]
    assert float((res[1] - ref).norm() / ref.norm()) < 1e-4
    assert float((res[2] - ref).norm() / ref.norm()) < 1e-2


@pytest.mark.parametrize("shape", [(40, 260, 300), (258, 12, 36), (20, 24, 270)])
def test_K_outside_the_pre_split_path_deterministic_and_matches_oracle(L, O, shape):
    """Axes longer than the pre-split pass takes (x > 264, y or z > 256): the fp32-input
    tensor-core pass.  Each tensor-core mode repeats bit for bit and matches the oracle (bf16x3
    2e-5, plain bf16 1e-2)."""
    Z, Y, X = shape
    rng = np.random.default_rng(8)
    f = rng.standard_normal(shape).astype(np.float32)
    ref = O.apply_K(f, 0.02, 1.0, (1, 1, 1), workers=-1)
    fd = _dev(f)
    a = torch.zeros(shape, device="cuda")
    for code, tol in ((1, 2e-5), (2, 1e-2)):
        p = L.default_params(X, Y, Z, k_mode=code)
        with L.Lddmm(p, a, a) as ctx:
            outs = []
            for _ in range(3):
                out = torch.empty_like(fd)
                ctx.apply_K(fd, out)
                outs.append(out)
            torch.cuda.synchronize()
        assert all(torch.equal(outs[0], o) for o in outs[1:]), code
        assert _rel(outs[0].cpu().numpy(), ref) < tol, code


# --------------------------------------------------------------------------- one iteration

def _pair_small(synth, shape=(32, 32, 32)):
    return synth.ellipsoid_pair(shape=shape, seed=0)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("shape,T,h", [((32, 32, 32), 10, (1, 1, 1)),
                                       ((20, 17, 23), 3, (1.0, 1.25, 0.8)),
                                       ((8, 10, 260), 3, (1, 1, 1))])
def test_one_step_matches_oracle(L, O, synth, mode, shape, T, h):
    Z, Y, X = shape
    pair = synth.ellipsoid_pair(shape=shape, centre=((X - 1) / 2, (Y - 1) / 2, (Z - 1) / 2),
                                semi_axes=(X / 3.2, Y / 4.0, Z / 4.5), width=X / 5.0,
                                amplitude=2.0, seed=3)
    v0 = synth.smooth_velocity(T, shape, 2.0, seed=4)
    code, _ = K_MODES[mode]
    p = L.default_params(X, Y, Z, T=T, hx=h[0], hy=h[1], hz=h[2], k_mode=code)
    po = O.Params(T=T, h=h)
    ref = O.lddmm_step(v0, pair.I0, pair.I1, pair.M, po)
    with L.Lddmm(p, _dev(pair.I0), _dev(pair.I1), _dev(pair.M)) as ctx:
        ctx.set_velocity(_dev(v0))
        u10 = ctx.get_field(L.LDDMM_FIELD_U10)
        u01 = ctx.get_field(L.LDDMM_FIELD_U01)
        J0 = ctx.get_field(L.LDDMM_FIELD_J0)
        e = ctx.step()
        v1 = ctx.get_velocity()
    assert _rel(u10, ref.u10) < 1e-5
    assert _rel(u01, ref.u01) < 1e-5
    assert _rel(J0, ref.J0T) < 1e-5
    assert _rel(v1, ref.v_new) < 1e-4
    assert abs(e["reg"] - ref.E_reg) <= 1e-5 * ref.E_reg
    assert abs(e["data"] - ref.E_data) <= 1e-5 * ref.E_data
    assert abs(e["min_det"] - ref.min_det) <= 1e-4
    # the update itself: v1 - v0 against the oracle's increment
    assert _rel(v1 - v0, ref.v_new - v0) < 1e-4


@pytest.mark.parametrize("shape,T,h", [((32, 32, 32), 4, (1, 1, 1)),
                                       ((20, 17, 23), 3, (1.0, 1.25, 0.8)),
                                       ((8, 10, 260), 4, (1, 1, 1))])
def test_one_step_rk4_matches_oracle(L, O, synth, shape, T, h):
    """flags bit 2: RK4 along each time step (the paper's integrator); the maps, the deformed
    template, the energies and the update against the oracle run with integrator='rk4'."""
    Z, Y, X = shape
    pair = synth.ellipsoid_pair(shape=shape, centre=((X - 1) / 2, (Y - 1) / 2, (Z - 1) / 2),
                                semi_axes=(X / 3.2, Y / 4.0, Z / 4.5), width=X / 5.0,
                                amplitude=2.0, seed=3)
    v0 = synth.smooth_velocity(T, shape, 3.0, seed=5)
    p = L.default_params(X, Y, Z, T=T, hx=h[0], hy=h[1], hz=h[2], k_mode=PROD, flags=4)
    po = O.Params(T=T, h=h, integrator="rk4")
    ref = O.lddmm_step(v0, pair.I0, pair.I1, pair.M, po)
    sl = O.lddmm_step(v0, pair.I0, pair.I1, pair.M, O.Params(T=T, h=h))
    with L.Lddmm(p, _dev(pair.I0), _dev(pair.I1), _dev(pair.M)) as ctx:
        ctx.set_velocity(_dev(v0))
        u10 = ctx.get_field(L.LDDMM_FIELD_U10)
        u01 = ctx.get_field(L.LDDMM_FIELD_U01)
        J0 = ctx.get_field(L.LDDMM_FIELD_J0)
        e = ctx.step()
        v1 = ctx.get_velocity()
        with pytest.raises(L.LddmmError) as ei:
            ctx.energy_grad(None, torch.empty((T, 3) + shape, device="cuda"))
        assert ei.value.code == L.LDDMM_ERR_INVALID_ARG
    assert _rel(u10, ref.u10) < 1e-5 and _rel(u01, ref.u01) < 1e-5
    assert _rel(u10, sl.u10) > 1e-4          # the integrators differ at this velocity
    assert _rel(J0, ref.J0T) < 1e-5
    assert _rel(v1 - v0, ref.v_new - v0) < 1e-4
    assert abs(e["reg"] - ref.E_reg) <= 1e-5 * ref.E_reg
    assert abs(e["data"] - ref.E_data) <= 1e-5 * ref.E_data


def _pair_centred(synth, shape):
    Z, Y, X = shape
    return synth.ellipsoid_pair(shape=shape, centre=((X - 1) / 2, (Y - 1) / 2, (Z - 1) / 2),
                                semi_axes=(X / 3.2, Y / 4.0, Z / 4.5), width=X / 5.0,
                                amplitude=2.0, seed=3)


@pytest.mark.parametrize("mode", MODES)
def test_degenerate_steps(L, O, synth, mode):
    """Cases the method reduces to a closed form: an empty mask (b = 0, so v <- (1 - 2 eps) v and
    E_data = 0); identical images from v = 0 (no residual: v stays 0 and E = 0); one time step
    (T = 1) and the smallest grid (2 x 2 x 2) against the oracle."""
    code, _ = K_MODES[mode]
    shape = (12, 10, 16)
    Z, Y, X = shape
    pair = _pair_centred(synth, shape)
    v0 = synth.smooth_velocity(3, shape, 1.5, seed=6)
    p = L.default_params(X, Y, Z, T=3, k_mode=code)
    eps = np.float32(p.epsilon)
    # empty mask
    with L.Lddmm(p, _dev(pair.I0), _dev(pair.I1), _dev(np.zeros(shape, np.float32))) as ctx:
        ctx.set_velocity(_dev(v0))
        e = ctx.step()
        v1 = ctx.get_velocity()
    ref = O.lddmm_step(v0, pair.I0, pair.I1, np.zeros(shape), O.Params(T=3))
    assert e["data"] == 0.0
    assert abs(e["reg"] - ref.E_reg) <= 1e-5 * ref.E_reg
    assert _rel(v1, v0 - eps * (np.float32(2) * v0)) < 1e-6
    # identical images from v = 0
    with L.Lddmm(p, _dev(pair.I0), _dev(pair.I0), _dev(pair.M)) as ctx:
        e = ctx.step()
        v1 = ctx.get_velocity()
    assert e["total"] == 0.0 and not v1.any()
    # T = 1, and the smallest grid
    rng = np.random.default_rng(9)
    tiny = [rng.random((2, 2, 2)).astype(np.float32) for _ in range(2)] + [np.ones((2, 2, 2), np.float32)]
    for shp, T, (I0, I1, M) in (((12, 10, 16), 1, (pair.I0, pair.I1, pair.M)),
                                ((2, 2, 2), 2, tiny)):
        z, y, x = shp
        vv = synth.smooth_velocity(T, shp, 0.5, seed=7)
        pp = L.default_params(x, y, z, T=T, k_mode=code)
        ref = O.lddmm_step(vv, I0, I1, M, O.Params(T=T))
        with L.Lddmm(pp, _dev(I0), _dev(I1), _dev(M)) as ctx:
            ctx.set_velocity(_dev(vv))
            e = ctx.step()
            v1 = ctx.get_velocity()
        assert _rel(v1, ref.v_new) < 1e-4
        assert abs(e["reg"] - ref.E_reg) <= 1e-5 * max(ref.E_reg, 1e-30)
        assert abs(e["data"] - ref.E_data) <= 1e-5 * max(ref.E_data, 1e-30) + 1e-12


def test_twenty_iterations_config1(L, O, synth):
    pair = _pair_small(synth)
    T = 10
    p = L.default_params(32, 32, 32, k_mode=PROD)
    with L.Lddmm(p, _dev(pair.I0), _dev(pair.I1), _dev(pair.M)) as ctx:
        eg = [ctx.step()["total"] for _ in range(20)]
        J0 = ctx.get_field(L.LDDMM_FIELD_J0)
        v = ctx.get_velocity()
    po = O.Params(T=T)
    vo = np.zeros((T, 3, 32, 32, 32))
    eo = []
    for _ in range(20):
        r = O.lddmm_step(vo, pair.I0, pair.I1, pair.M, po)
        eo.append(r.E)
        vo = r.v_new
    J1, W, _, _ = O.backward_sweep(vo, pair.I1, pair.M, po)
    _, _, J0o, _ = O.forward_sweep(vo, pair.I0, pair.I1, pair.M, J1, W, po)
    assert _rel(J0, J0o) < 1e-3
    assert _rel(v, vo) < 1e-3
    for a, b in zip(eg, eo):
        assert abs(a - b) <= 1e-4 * b
    assert all(b < a for a, b in zip(eg, eg[1:]))


# --------------------------------------------------------------------------- outputs

@pytest.fixture(scope="module")
def brain_small(synth):
    pair, atlas = synth.brain_pair(shape=(29, 20, 33), base_shape=(114, 80, 132), seed=1)
    return pair


def test_labels_bit_exact_and_warp(L, O, synth, brain_small):
    pair = brain_small
    Z, Y, X = pair.I0.shape
    T = 5
    v0 = synth.smooth_velocity(T, (Z, Y, X), 3.0, seed=7)
    p = L.default_params(X, Y, Z, T=T, k_mode=PROD)
    with L.Lddmm(p, _dev(pair.I0), _dev(pair.I1), _dev(pair.M)) as ctx:
        ctx.set_velocity(_dev(v0))
        labels = ctx.transfer_labels(_dev(pair.L0.view(np.int16)),
                                     torch.empty((Z, Y, X), dtype=torch.int16, device="cuda"))
        labels = labels.cpu().numpy().view(np.uint16)
        labels_host = ctx.transfer_labels(pair.L0)           # host in, host out
        u10 = ctx.get_field(L.LDDMM_FIELD_U10)
        u01 = ctx.get_field(L.LDDMM_FIELD_U01)
        img = pair.image1
        w0 = ctx.warp(img, 0)
        w1 = ctx.warp(_dev(img), 1, torch.empty((Z, Y, X), device="cuda")).cpu().numpy()
        d = ctx.dice(pair.L0, labels_host)
    ref = O.transfer_labels(pair.L0, u10)
    np.testing.assert_array_equal(labels, ref)
    np.testing.assert_array_equal(labels_host, ref)
    assert _rel(w0, O.warp(img, u10)) < 1e-6
    assert _rel(w1, O.warp(img, u01)) < 1e-6
    assert abs(d - O.dice(pair.L0, ref)) < 1e-12
    # and the maps themselves against the oracle's flows
    po = O.Params(T=T)
    J1, W, u01o, _ = O.backward_sweep(v0, pair.I1, pair.M, po)
    _, u10o, _, _ = O.forward_sweep(v0, pair.I0, pair.I1, pair.M, J1, W, po)
    assert _rel(u10, u10o) < 1e-5 and _rel(u01, u01o) < 1e-5


def test_multiscale_register_matches_oracle(L, O, synth):
    shape = (23, 18, 26)            # ragged at every level: 6x5x7, 12x9x13, 23x18x26
    Z, Y, X = shape
    pair = synth.ellipsoid_pair(shape=shape, centre=(12.5, 8.5, 11), semi_axes=(8, 6, 7),
                                width=5.0, amplitude=2.0, seed=5)
    T, iters = 4, 3
    p = L.default_params(X, Y, Z, T=T, iterations=iters, level_factor=[4, 2, 1], k_mode=PROD)
    with L.Lddmm(p, _dev(pair.I0), _dev(pair.I1), _dev(pair.M)) as ctx:
        trace = ctx.register()
        v = ctx.get_velocity()
        assert ctx.grid()[:3] == (X, Y, Z)
    vo, eo, _ = O.register(pair.I0, pair.I1, pair.M, O.Params(T=T), iters, factors=(4, 2, 1))
    assert len(trace) == 3 * iters
    assert _rel(v, vo) < 1e-4
    for t, (f, er, ed) in zip(trace, eo):
        assert abs(t["total"] - (er + ed)) <= 1e-5 * (er + ed)


# --------------------------------------------------------------------------- full size

@pytest.mark.parametrize("mode", MODES[-1:])
def test_full_size_first_step(L, O, synth, mode):
    """264x160x228, T = 10 (the benchmark's grid and launch configuration): from v = 0 every
    time step sees J0 = I0, J1 = I1, W = M, so v_new_j = eps K[(2/sigma^2) M (I0 - I1) grad I0]
    for all j; the oracle evaluates that in FP64 (pointwise residual + FFT)."""
    pair, _ = synth.brain_pair(shape=(228, 160, 264), base_shape=(114, 80, 132), seed=1)
    Z, Y, X = pair.I0.shape
    code, _ = K_MODES[mode]
    p = L.default_params(X, Y, Z, k_mode=code)
    po = O.Params()
    with L.Lddmm(p, _dev(pair.I0), _dev(pair.I1), _dev(pair.M)) as ctx:
        e = ctx.step()
        v = torch.empty((10, 3, Z, Y, X), device="cuda")
        ctx.get_velocity(v)
    I0 = pair.I0.astype(np.float64)
    r = 2.0 / po.sigma ** 2 * pair.M * (I0 - pair.I1)
    g = O.fd_gradient(I0)
    ref = np.stack([po.epsilon * O.apply_K(r * g[e_], po.alpha, po.gamma, po.h, workers=-1)
                    for e_ in range(3)])
    v0 = v[0].cpu().numpy()
    assert _rel(v0, ref) < 1e-4
    for j in (1, 5, 9):
        assert torch.equal(v[j], v[0])
    Ed = float((pair.M * (I0 - pair.I1) ** 2).sum()) / po.sigma ** 2
    assert abs(e["data"] - Ed) <= 1e-6 * Ed
    assert e["reg"] == 0.0 and e["min_det"] == 1.0


# --------------------------------------------------------------------------- API behaviour

def test_host_and_device_pointers_agree(L, synth):
    pair = synth.ellipsoid_pair(shape=(16, 16, 16), centre=(7.5, 7.5, 7.5), semi_axes=(5, 4, 3.5),
                                width=3.0, amplitude=1.5, seed=0)
    p = L.default_params(16, 16, 16, T=4, k_mode=PROD)
    with L.Lddmm(p, pair.I0, pair.I1, pair.M) as a, \
            L.Lddmm(p, _dev(pair.I0), _dev(pair.I1), _dev(pair.M)) as b:
        ea = [a.step()["total"] for _ in range(2)]
        eb = [b.step()["total"] for _ in range(2)]
        va = a.get_velocity()
        vb = torch.empty((4, 3, 16, 16, 16), device="cuda")
        b.get_velocity(vb)
    # the energies are FP64 sums with atomics (summation order varies); v is deterministic
    np.testing.assert_allclose(ea, eb, rtol=1e-12)
    np.testing.assert_array_equal(va, vb.cpu().numpy())


def test_nonfinite_input_rejected(L):
    a = np.zeros((8, 8, 8), np.float32)
    b = a.copy()
    b[3, 4, 5] = np.nan
    p = L.default_params(8, 8, 8)
    with pytest.raises(L.LddmmError) as ei:
        L.Lddmm(p, a, b)
    assert ei.value.code == L.LDDMM_ERR_NONFINITE


def test_bounded_wait_reports_timeout_and_context_survives(L, synth):
    """A host wait shorter than the queued work returns LDDMM_ERR_TIMEOUT (nothing hangs); once
    the stream drains, the same context keeps working."""
    shape = (96, 96, 96)
    pair = synth.ellipsoid_pair(shape=shape, centre=(47.5, 47.5, 47.5), semi_axes=(30, 24, 21),
                                width=18.0, amplitude=6.0, seed=0)
    p = L.default_params(96, 96, 96, k_mode=0)
    with L.Lddmm(p, _dev(pair.I0), _dev(pair.I1), _dev(pair.M)) as ctx:
        ctx.set_timeout(1e-6)
        for _ in range(3):
            ctx.step(want_energy=False)
        with pytest.raises(L.LddmmError) as ei:
            ctx.step()
        assert ei.value.code == L.LDDMM_ERR_TIMEOUT
        torch.cuda.synchronize()
        ctx.set_timeout(60.0)
        e = ctx.step()
        assert np.isfinite(e["total"]) and e["iter"] == 4   # 0-based: the fifth


def test_backtracking_never_increases_energy(L, synth):
    pair = synth.ellipsoid_pair(seed=0)
    p = L.default_params(32, 32, 32, T=4, epsilon=0.05, flags=1, k_mode=PROD)
    with L.Lddmm(p, _dev(pair.I0), _dev(pair.I1), _dev(pair.M)) as ctx:
        E = [ctx.step()["total"] for _ in range(8)]
    # a rejected step returns the energy of the restored field again (equal up to the FP64
    # atomic summation order)
    assert all(b <= a * (1 + 1e-12) for a, b in zip(E, E[1:])), E
    assert E[-1] < 0.5 * E[0]
