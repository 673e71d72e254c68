"""Every launch-shape variant of the level sweep and of the persistent task
kernel (CTAs per SM, whole or half tiles per thread group) reproduces the
oracle exactly: variants change where the work runs, never the arithmetic."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2609_35529_b300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_35529_b300 import build, vlbm
    build.build()
    return vlbm


@pytest.mark.parametrize("schedule", [0, 1])
@pytest.mark.parametrize("variant", range(5))
def test_every_sweep_variant_matches_oracle(V, variant, schedule):
    assert V.num_variants() == 5
    refs = I.box_refs(48, 40, 3, [(0, 8, 8, 24, 24)])
    refs[1][24:40, 24:56] = 1
    cs = I.smooth_random(48, 40, 3, refs, seed=40 + variant, amp=0.2, beta=1.0, steps=9)
    g = V.Hierarchy.from_case(cs)
    g.set_tuning(variant=variant, schedule=schedule)
    o = O.Hierarchy(cs.nx0, cs.ny0, cs.nlev, 2, cs.bc, cs.gamma, cs.c, cs.beta)
    o.set_layout(cs.refs)
    for l in range(cs.nlev):
        o.set_state(l, cs.W[l])
    g.advance(cs.steps)
    o.advance(cs.steps)
    for l in range(cs.nlev):
        gin, gref = g.layout(l)
        act = (gin == 1) & (gref == 0)
        assert np.array_equal(g.get_populations(l)[:, act], o.get_f(l)[:, act]), (variant, l)


def test_unknown_variant_is_rejected(V):
    cs = I.smooth_random(16, 16, 1, [], seed=1, beta=0.8)
    g = V.Hierarchy.from_case(cs)
    with pytest.raises(V.VlbmError):
        g.set_tuning(variant=5)
