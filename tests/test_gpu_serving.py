"""The serving path against the oracle: a reduced request trace (the same
recipe as the 512-request trace -- Riemann quadrant problems and vortices,
one to three levels, static or adaptive -- with sides up to 256) served by
the continuous-batching loop on both engine schedules; the batched results
of the smallest requests equal the oracle's bit for bit, and every request's
result equals its run alone."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_35529_b300 import build, serve
    build.build()
    return serve


@pytest.mark.parametrize("schedule", [0, 1])
def test_served_requests_equal_the_oracle_and_their_runs_alone(S, schedule):
    import serving_oracle_sample as sample
    out, reqs = S.run(["--requests", "48", "--nmax", "256", "--keep-sample", "10",
                       "--engine-schedule", str(schedule)])
    mix = out["alone_vs_mix"]
    assert mix["compared"] == len(reqs) and mix["bitwise_equal"] == len(reqs)
    kept = [r for r in reqs if r.result is not None]
    assert len(kept) == 10
    assert any(r.adaptive for r in kept) or any(r.nlev > 1 for r in kept)
    for r in kept:
        assert sample.agreement(r.result, sample.run_oracle(r)) == 0.0, r.rid
