"""Host logic of the serving loop that needs no GPU: the seeded request stream."""
import numpy as np

from paper_2609_08800_gb300 import serve


def test_poisson_stream_shape():
    a = serve.poisson_stream(200, 5.0, seed=1)
    b = serve.poisson_stream(200, 5.0, seed=1)
    assert [(r.kind, r.n, r.T, r.adjoint, r.arrival) for r in a] == [(r.kind, r.n, r.T, r.adjoint, r.arrival) for r in b]
    arr = np.array([r.arrival for r in a])
    assert np.all(np.diff(arr) > 0) and arr[-1] <= 5.0
    assert abs(len(a) - 1000) < 4 * np.sqrt(1000)          # Poisson count within 4 sigma
    n = np.array([r.n for r in a])
    T = np.array([r.T for r in a])
    assert n.min() >= 1 and n.max() <= 512 and T.min() >= 20 and T.max() <= 200
    # log-uniform: about half the requests below sqrt(513) worlds
    assert 0.4 < np.mean(n < np.sqrt(513)) < 0.6
    assert 0.4 < np.mean([r.adjoint for r in a]) < 0.6
    kinds = [r.kind for r in a]
    for k in ("box", "robot", "terrain"):
        assert 0.25 < kinds.count(k) / len(kinds) < 0.42


def test_summarize_censors_unfinished_requests():
    """Requests left unfinished at a cutoff count with latency cutoff - arrival (a lower
    bound), so the censored percentiles bound the stream's from below."""
    done = [serve.Request(rid=k, kind="box", n=1, T=20, adjoint=False, arrival=0.1 * k) for k in range(4)]
    for k, r in enumerate(done):
        r.latency = 1.0 + k
    late = [serve.Request(rid=10 + k, kind="box", n=2, T=30, adjoint=True, arrival=1.0 + k) for k in range(3)]
    st = serve.summarize(done, 10.0, late, cutoff=3.5)
    assert st["requests"] == 4 and st["world_steps"] == 80
    assert st["unfinished"] == 3 and st["not_arrived"] == 0
    cens = np.array([1.0, 2.0, 3.0, 4.0, 2.5, 1.5, 0.5])
    assert st["censored_p50_s"] == np.percentile(cens, 50) and st["censored_p99_s"] == np.percentile(cens, 99)
    st2 = serve.summarize(done, 10.0, late, cutoff=1.5)
    assert st2["unfinished"] == 1 and st2["not_arrived"] == 2
