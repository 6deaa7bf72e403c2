"""GPU parity of the §2.2 preprocessing through the C ABI against the FP64 oracle: the
histogram matching of the Image-LDDMM pipeline (every FP64 step in the order of the oracle, so
the float32 result must equal the oracle's rounded to float32) and the ball morphology of the
mask generation (bit-exact)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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
def OP():
    from oracle import preprocess
    return preprocess


@pytest.fixture(scope="module")
def brain():
    from paper_1605_02060_gb300 import synth
    return synth.brain_pair(shape=(57, 40, 66), base_shape=(114, 80, 132), seed=1)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("bins,points", [(32, 8), (16, 3), (64, 0)])
def test_histogram_match_equals_oracle(L, OP, brain, bins, points):
    pair, atlas = brain
    I0, M0 = atlas.astype(np.float32), pair.I0
    I1, M1 = pair.image1, pair.I1
    got = L.histogram_match(_dev(I0), _dev(M0), _dev(I1), _dev(M1), bins=bins, points=points)
    ref = OP.histogram_match(I0, M0, I1, M1, bins, points).astype(np.float32)
    assert np.array_equal(got.cpu().numpy(), ref)


def test_histogram_match_identity_and_empty_mask(L, brain):
    pair, atlas = brain
    I0, M0 = _dev(atlas.astype(np.float32)), _dev(pair.I0)
    out = L.histogram_match(I0, M0, I0, M0)
    m = pair.I0 > 0.5
    assert np.array_equal(out.cpu().numpy()[m], atlas.astype(np.float32)[m])
    assert not out.cpu().numpy()[~m].any()
    with pytest.raises(L.LddmmError) as ei:
        L.histogram_match(I0, torch.zeros_like(M0), I0, M0)
    assert ei.value.code == L.LDDMM_ERR_INVALID_ARG


@pytest.mark.parametrize("t,ro,rc", [(0.025, 1, 2), (0.1, 0, 1), (0.025, 2, 3)])
def test_mask_morphology_equals_oracle(L, OP, brain, t, ro, rc):
    pair, _ = brain
    got = L.mask_morphology(_dev(pair.image1), t, ro, rc)
    ref = OP.mask_morphology(pair.image1, t, ro, rc)
    assert np.array_equal(got.cpu().numpy().astype(bool), ref)


def test_full_size_preprocessing(L, OP):
    """264x160x228: the target mask from the target intensities and the matched atlas image."""
    from paper_1605_02060_gb300 import synth
    pair, atlas = synth.brain_pair(shape=(228, 160, 264), base_shape=(114, 80, 132), seed=1)
    got = L.mask_morphology(_dev(pair.image1), 0.025, 1, 3)
    ref = OP.mask_morphology(pair.image1, 0.025, 1, 3)
    assert np.array_equal(got.cpu().numpy().astype(bool), ref)
    out = L.histogram_match(_dev(atlas.astype(np.float32)), _dev(pair.I0), _dev(pair.image1),
                            _dev(pair.I1))
    r = OP.histogram_match(atlas, pair.I0, pair.image1, pair.I1).astype(np.float32)
    assert np.array_equal(out.cpu().numpy(), r)
