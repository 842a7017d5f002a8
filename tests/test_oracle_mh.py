"""Algorithm 7 (Metropolis-Hastings lazy resampling) in the oracle, pinned to the exact law
of its Markov chain: B steps from (n, n), uniform proposals over the N^2 pairs accepted
with probability min(1, omega* / omega).  The law after B steps is e_(n,n) P^B with P the
chain's transition matrix; for large B it is the normalised weight matrix itself."""
import numpy as np
from scipy import stats

from oracle import core


def _exact_law(w, start, B):
    S = w.size
    wf = w.ravel()
    P = np.zeros((S, S))
    for s in range(S):
        for t in range(S):
            if t == s:
                continue
            a = (1.0 if wf[t] > 0 else 0.0) if wf[s] == 0 else min(1.0, wf[t] / wf[s])
            P[s, t] = a / S
        P[s, s] = 1.0 - P[s].sum()
    p = np.zeros(S)
    p[start] = 1.0
    return p @ np.linalg.matrix_power(P, B)


def _draws(w, n_start, B, G, seed=11, gid=5):
    """G draws of the chain started at (n_start, n_start): slots n = n_start + N k."""
    N = w.shape[0]
    with np.errstate(divide="ignore"):
        logW = np.log(w)
    li, ri = core.mh_pairs(logW, seed, gid, 0, N * G, B)
    sel = np.arange(N * G) % N == n_start
    return li[sel] * N + ri[sel]


def _chi2_pvalue(flat, law):
    obs = np.bincount(flat, minlength=law.size).astype(float)
    exp = law * flat.size
    keep = exp > 0
    assert obs[~keep].sum() == 0          # no draw of a pair the chain cannot reach
    return stats.chisquare(obs[keep], exp[keep]).pvalue


def test_zero_steps_return_the_start():
    w = np.array([[1.0, 2.0], [0.5, 3.0]])
    li, ri = core.mh_pairs(np.log(w), 3, 1, 0, 6, 0)
    assert list(li) == [0, 1, 0, 1, 0, 1] and list(ri) == [0, 1, 0, 1, 0, 1]


def test_few_steps_follow_the_chain_law():
    w = np.array([[1.0, 2.0, 0.0], [3.0, 0.5, 1.0], [0.0, 1.0, 2.0]])
    for n_start, B in ((1, 1), (1, 3), (0, 2)):
        flat = _draws(w, n_start, B, 40000)
        law = _exact_law(w, n_start * 3 + n_start, B)
        assert _chi2_pvalue(flat, law) > 1e-3, (n_start, B)


def test_many_steps_reach_the_weight_law():
    w = np.array([[1.0, 2.0, 0.0], [3.0, 0.5, 1.0], [0.0, 1.0, 2.0]])
    flat = _draws(w, 2, 200, 30000)
    assert _chi2_pvalue(flat, (w / w.sum()).ravel()) > 1e-3


def test_chain_started_on_a_zero_weight_pair():
    # slots n = 1 mod 3 start at (1, 1), which weighs 0: any proposal of positive weight is
    # taken, a zero-weight one leaves the chain where it is
    w = np.array([[1.0, 2.0, 0.0], [3.0, 0.0, 1.0], [0.0, 1.0, 2.0]])
    for B in (1, 2):
        flat = _draws(w, 1, B, 40000)
        law = _exact_law(w, 1 * 3 + 1, B)
        assert _chi2_pvalue(flat, law) > 1e-3, B
    assert abs(_exact_law(w, 4, 1)[4] - 3.0 / 9) < 1e-12   # the three zero pairs keep it there
