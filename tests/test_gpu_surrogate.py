"""What the trained surrogate gains over the method without it (reduced
scale: 0.5 s rollouts, 16,384 training robots).

The plain search simulates every mutant; the screened search simulates only
the mutants the network ranks highest.  Here all 1024 mutants of a generation
are simulated (ground truth) and the network's pick of 64 is compared with a
random pick of 64 (the search without the network): it must capture far more
of the truly best 64 and have a higher mean simulated fitness."""
import numpy as np
import pytest

from paper_1911_10274_gb300 import surrogate as S

pytestmark = pytest.mark.gpu
STEPS = 5000


@pytest.fixture(scope="module")
def trained():
    rng = np.random.default_rng(0)
    morphs = [S.random_morph(rng) for _ in range(16384)]
    y = S.fitness(morphs, STEPS)
    X = S.encode(morphs)
    sur = S.Surrogate(seed=0)
    hist = sur.fit(X[:-512], y[:-512], epochs=8, batch=1024)
    return sur, morphs, y, X, hist


def test_surrogate_learns_and_generalises(trained):
    sur, morphs, y, X, hist = trained
    assert hist[-1] < hist[0]
    rho = S.spearman(sur.predict(X[-512:]), y[-512:])
    # held-out rank correlation; its standard error at n = 512 is about 0.044
    assert rho > 0.1, rho


def test_surrogate_screening_beats_random_screening(trained):
    sur, morphs, y, X, _ = trained
    rng = np.random.default_rng(7)
    parents = [morphs[i] for i in np.argsort(-y)[:16]]
    kids = [S.mutate(rng, parents[k % 16]) for k in range(1024)]
    truth = S.fitness(kids, STEPS)
    best64 = set(np.argsort(-truth)[:64])
    pick = np.argsort(-sur.predict(S.encode(kids)))[:64]
    recall = len(best64 & set(pick)) / 64
    # a random pick of 64 catches 64/1024 = 6.25% of the best 64 on average
    assert recall >= 3 * 64 / 1024, recall
    rand = rng.choice(1024, 64, replace=False)
    assert truth[pick].mean() > truth[rand].mean()
    assert truth[pick].max() >= np.quantile(truth, 0.95)
