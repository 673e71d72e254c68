"""Host logic of the serving loop (no GPU): the continuous-batching loop and
the one-at-a-time loop run against a fake engine that refuses admissions at
random (as the real one does when a hierarchy's exact byte count exceeds the
budget), finishes residents at their step counts and reports the steps it
took.  Every request must finish exactly once, with its payload prepared
once, whatever the refusals."""
import random

import numpy as np
import pytest

from paper_2609_35529_b300 import serve as S


class FakeH:
    def __init__(self, r, cs):
        self.r, self.cs, self.nlev, self.closed = r, cs, cs.nlev, False
        self.steps = 0

    def info(self):
        return {"lups_per_step": 1000}

    def advance(self, n):
        self.steps += n

    def regrid(self):
        pass

    def get_conserved(self, l):
        return np.zeros((4, 2, 2)), np.ones((2, 2), bool)

    def get_populations(self, l):
        return np.zeros((16, 2, 2))

    def host_times(self):
        return {"tasks": 1.0}

    def close(self):
        self.closed = True


class FakeEngine:
    def __init__(self, budget, stream=None, refuse=0.3, seed=0, schedule=0):
        self.rng = random.Random(seed)
        self.refuse = refuse
        self.res = {}
        self.next = 0
        self.admitted = []

    def admit(self, h, steps, every=0):
        if self.res and self.rng.random() < self.refuse:
            return None
        s = self.next
        self.next += 1
        self.res[s] = [h, steps, 0]
        self.admitted.append(h.r.rid)
        return s

    def advance(self, max_steps):
        if not self.res:
            return [], 0
        k = min(max_steps, min(t - d for _, t, d in self.res.values()))
        fin = []
        for s, v in self.res.items():
            v[2] += k
            if v[2] == v[1]:
                fin.append(s)
        return fin, k

    def slot_stats(self, s):
        return self.res[s][2], 1000 * self.res[s][2]

    def release(self, s):
        del self.res[s]

    def close(self):
        pass


@pytest.fixture
def fakes(monkeypatch):
    made = []

    def start(r, stream, cs=None):
        cs = cs if cs is not None else S.make_case(r)
        h = FakeH(r, cs)
        made.append(h)
        return h, cs

    calls = {"n": 0}
    real_make = S.make_case

    def counting_make(r):
        calls["n"] += 1
        return real_make(r)

    monkeypatch.setattr(S, "_start", start)
    monkeypatch.setattr(S, "make_case", counting_make)
    monkeypatch.setattr(S.V, "Engine", FakeEngine)
    return made, calls


@pytest.mark.timeout(120)
@pytest.mark.parametrize("spread", [0.0, 0.002])
def test_batched_loop_finishes_every_request_once(fakes, spread):
    made, calls = fakes
    reqs = S.make_requests(24, seed=3, nmax=256)
    calls["n"] = 0
    for i, r in enumerate(reqs):
        r.arrival = i * spread
        r.steps = 5 + (i * 7) % 23
    tts, mlups, wall = S.serve_batched(reqs, budget=1 << 40)
    assert len(tts) == len(reqs) and np.all(tts >= 0)
    assert all(r.done_at is not None for r in reqs)
    assert calls["n"] == len(reqs)  # one payload per request, kept across refusals
    live = [h for h in made if not h.closed]
    assert not live


@pytest.mark.timeout(120)
def test_one_at_a_time_loop_finishes_every_request(fakes):
    made, calls = fakes
    reqs = S.make_requests(10, seed=4, nmax=256)
    calls["n"] = 0
    for i, r in enumerate(reqs):
        r.arrival = 0.0
    tts, mlups, wall = S.serve_one_at_a_time(reqs)
    assert len(tts) == len(reqs) and all(r.done_at is not None for r in reqs)
    assert calls["n"] == len(reqs)
    assert all(h.closed for h in made)


@pytest.mark.timeout(120)
def test_both_loops_feed_the_alone_vs_mix_comparison(fakes):
    made, calls = fakes
    reqs = S.make_requests(8, seed=5, nmax=256)
    for r in reqs:
        r.arrival = 0.0
        r.steps = 6
    S.serve_batched(reqs, budget=1 << 40, verify=True)
    S.serve_one_at_a_time(reqs, verify=True)
    assert S.alone_vs_mix(reqs) == {"compared": len(reqs), "bitwise_equal": len(reqs)}


def test_result_digest_sees_every_bit():
    """The alone-vs-mix comparison's digest: equal results give equal
    digests, one flipped bit, two swapped cells or two swapped fields give
    another."""
    from paper_2609_35529_b300.serve import digest
    rng = np.random.default_rng(3)
    W = rng.standard_normal((4, 16, 24))
    act = rng.random((16, 24)) > 0.3
    d0 = digest(W, act)
    assert digest(W.copy(), act) == d0
    W2 = W.copy()
    W2.view(np.uint64)[2, 5, 7] ^= np.uint64(1)
    if act[5, 7]:
        assert digest(W2, act) != d0
    else:
        assert digest(W2, act) == d0  # masked cells do not count
    cells = np.argwhere(act)
    (a0, b0), (a1, b1) = cells[0], cells[1]
    W3 = W.copy()
    W3[:, a0, b0], W3[:, a1, b1] = W[:, a1, b1], W[:, a0, b0]
    assert digest(W3, act) != d0
    W4 = W.copy()
    W4[0, a0, b0], W4[1, a0, b0] = W[1, a0, b0], W[0, a0, b0]  # two fields of one cell
    assert digest(W4, act) != d0


@pytest.mark.timeout(120)
def test_batched_loop_respects_the_work_cap(fakes, monkeypatch):
    """With an admission cap on the residents' cell updates per step, a
    request is admitted only while the residents (itself included) stay
    within the cap, or when nothing else is resident; every request still
    finishes exactly once, in arrival order of admission."""
    made, calls = fakes
    reqs = S.make_requests(16, seed=6, nmax=256)
    for r in reqs:
        r.arrival = 0.0
        r.steps = 4 + r.rid % 5
    per = {r.rid: r.lups / max(1, r.steps) for r in reqs}
    cap = 2.5 * max(per.values())
    loads = []
    real_admit = FakeEngine.admit

    def admit(self, h, steps, every=0):
        s = real_admit(self, h, steps, every)
        if s is not None:
            loads.append((len(self.res), sum(per[v[0].r.rid] for v in self.res.values())))
        return s

    monkeypatch.setattr(FakeEngine, "admit", admit)
    tts, mlups, wall = S.serve_batched(reqs, budget=1 << 40, work_cap=cap)
    assert all(r.done_at is not None for r in reqs)
    assert len(loads) == len(reqs)
    assert all(n == 1 or w <= cap for n, w in loads)
    assert max(n for n, _ in loads) < len(reqs)  # the cap held some requests back
    assert not [h for h in made if not h.closed]
