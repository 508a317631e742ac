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
