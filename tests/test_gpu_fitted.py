"""The workloads with their fitted occupancy networks (2000 Adam steps of BCE
on 65,536 points against the capsules' occupancy, fitted once by the oracle's
trainer: tests/golden/fit_occupancy.py) through the CUDA path against the
FP64 oracle: the same exact localization rules as the constructed networks
(tests/parity_rules.py), the render, and the MIXED form's band values."""
import numpy as np
import pytest

from oracle import field, localize
from paper_2007_13988_gb300 import synth

from gpu_common import OCC_TOL, Ctx, check_localization, check_mixed_values, check_render, localized

pytestmark = pytest.mark.gpu

MIXED = 2


def occ_oracle(w, P):
    return field.occupancy(w.occ_net, w.occ_map, w.calib, P)


@pytest.fixture(scope="module")
def tiny():
    c = Ctx(synth.tiny_fitted())
    yield c
    c.close()


@pytest.fixture(scope="module")
def full():
    c = Ctx(synth.full_fitted())
    yield c
    c.close()


@pytest.fixture(scope="module")
def tiny_oracle(tiny):
    w = tiny.w
    return localize.hierarchical(lambda P: occ_oracle(w, P), w.n0, w.num_levels)


@pytest.fixture(scope="module")
def full_oracle_256(full):
    w = full.w
    return localize.hierarchical(lambda P: occ_oracle(w, P), w.n0, w.num_levels)


def test_query_fitted_nets(tiny, full):
    for c in (tiny, full):
        P = synth.query_points(4099, seed=77)
        err = np.max(np.abs(c.query(P) - occ_oracle(c.w, P)))
        assert err <= OCC_TOL, err


def test_localize_tiny_fitted(tiny, tiny_oracle):
    res, _, vol = check_localization(tiny, tiny_oracle, lambda P: occ_oracle(tiny.w, P))
    print("tiny fitted localization:", res, [l.n_eval for l in tiny_oracle])


def test_render_tiny_fitted(tiny, tiny_oracle):
    print("tiny fitted render:", check_render(tiny, localized(tiny, tiny_oracle), 64))


def test_localize_full_fitted_256(full, full_oracle_256):
    res, _, vol = check_localization(full, full_oracle_256, lambda P: occ_oracle(full.w, P))
    assert vol.n == 256
    print("full fitted localization:", res, [l.n_eval for l in full_oracle_256],
          [l.conflict_rounds for l in full_oracle_256])


def test_render_full_fitted_512(full, full_oracle_256):
    print("full fitted render:", check_render(full, localized(full, full_oracle_256), 512))


def test_mixed_full_fitted_band_values(full, full_oracle_256):
    vol = full.localize(precision=MIXED)
    res = check_mixed_values(full, vol, full_oracle_256, lambda P: occ_oracle(full.w, P))
    print("full fitted MIXED:", res, "rechecked", list(vol.rechecked_per_level)[:4])
    assert res["in_band"] > 0
