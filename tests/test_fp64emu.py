"""The integer-pipe binary64 routines used inside the sweep agree bit for bit
with the FP64 unit (addition, subtraction, multiplication, halving), and
every sweep variant reproduces the oracle exactly."""
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


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_emulated_binary64_is_bit_exact(V, seed):
    bad, first = V.selftest_fp64(seed, 1 << 26)
    assert all(v == 0 for v in bad.values()), (bad, first)


@pytest.mark.parametrize("variant", range(15))
def test_every_sweep_variant_matches_oracle(V, variant):
    # beta = 1 so that every variant applies (1 - 2 beta = -1)
    refs = I.box_refs(48, 40, 3, [(0, 8, 8, 24, 24)])
    refs[1][24:40, 24:56] = 1
    cs = I.smooth_random(48, 40, 3, refs, seed=40 + variant, amp=0.2, beta=1.0, steps=9)
    g = V.Hierarchy.from_case(cs)
    g.set_tuning(variant=variant)
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


def test_variant_needing_beta_one_is_rejected(V):
    cs = I.smooth_random(16, 16, 1, [], seed=1, beta=0.8)
    g = V.Hierarchy.from_case(cs)
    with pytest.raises(V.VlbmError):
        g.set_tuning(variant=6)
