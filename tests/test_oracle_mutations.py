"""Each plausible mistake planted in the oracle is caught by some pin.

A mistake is planted by rewriting one line of a copy of the oracle's
source and loading the copy as a separate module (on the CPU); the pins in
``tests/pins.py`` must then fail at least once.  This shows that the pins
constrain every step of the oracle, not just its happy path.
"""
import importlib.util
import inspect
import types

import pytest

import oracle.communicability as oc
from tests import pins

MUTATIONS = [
    # transposed operand: first column instead of first row of Q
    ("c = Q @ (np.exp(lam - theta) * Q[0, :])", "c = Q @ (np.exp(lam - theta) * Q[:, 0])"),
    # dropped factor beta0 = ||1||
    ("y = beta0 * (V.T @ c)", "y = (V.T @ c)"),
    # shift applied with the wrong sign
    ("c = Q @ (np.exp(lam - theta) * Q[0, :])", "c = Q @ (np.exp(lam + theta) * Q[0, :])"),
    # ensemble weights with the shift reversed (eq. 5)
    ("S[:n] += math.exp(theta - theta_star) * y", "S[:n] += math.exp(theta_star - theta) * y"),
    # ensemble drops the last realisation
    ("for (n, _, _), (theta, y, _) in zip(graphs, parts):",
     "for (n, _, _), (theta, y, _) in list(zip(graphs, parts))[:-1]:"),
    # top-k tie rule reversed
    ("order = np.lexsort((idx, -S))[:k]", "order = np.lexsort((-idx, -S))[:k]"),
    # top-k ascending instead of descending
    ("order = np.lexsort((idx, -S))[:k]", "order = np.lexsort((idx, S))[:k]"),
    # missing 1/k in the Taylor term
    ("term = term @ X / k", "term = term @ X"),
    # one squaring too few
    ("for _ in range(s):\n        E = E @ E", "for _ in range(s - 1):\n        E = E @ E"),
    # Lanczos vector not normalised
    ("V[j + 1] = w / beta[j]", "V[j + 1] = w"),
    # breakdown step off by one
    ("m_eff = j + 1\n", "m_eff = j\n"),
    # wrong off-diagonal in T
    ("T = np.diag(alpha) + np.diag(beta_off[: k - 1], 1) + np.diag(beta_off[: k - 1], -1)",
     "T = np.diag(alpha) + np.diag(beta_off[1:k], 1) + np.diag(beta_off[1:k], -1)"),
    # alpha taken before subtracting the previous vector and without A
    ("alpha[j] = V[j] @ w", "alpha[j] = V[j] @ (A @ V[j]) + 0.5"),
    # start vector not normalised
    ("V[0] = b / beta0", "V[0] = b / n"),
    # walk-count brute force: factorial off by one
    ("fact *= k\n", "fact *= k + 1\n"),
    # sub-graph centrality: last instead of first quadrature coefficient
    ("c0.append(float(c[0]))", "c0.append(float(c[-1]))"),
    # sub-graph centrality: start vector on the wrong node
    ("b[int(i)] = 1.0", "b[(int(i) + 1) % n] = 1.0"),
    # restarted Krylov: coupling above instead of below the diagonal
    ("H[o, o - 1] = couple[i - 1]", "H[o - 1, o] = couple[i - 1]"),
    # restarted Krylov: coupling with the wrong residual norm
    ("couple.append(beta[m - 1])", "couple.append(beta[m - 2])"),
    # restarted Krylov: next cycle restarts from the last kept vector
    ("v = V[m]\n", "v = V[m - 1]\n"),
    # restarted Krylov: first row instead of first column of exp(H)
    ("c = expm_taylor(H - theta * np.eye(K))[:, 0]", "c = expm_taylor(H - theta * np.eye(K))[0, :]"),
]


def _mutant(old, new):
    src = inspect.getsource(oc)
    assert src.count(old) >= 1, old
    mod = types.ModuleType("oracle_mutant")
    exec(compile(src.replace(old, new, 1), "oracle_mutant", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("old,new", MUTATIONS, ids=[f"m{i}" for i in range(len(MUTATIONS))])
def test_planted_mistake_is_caught(old, new):
    mod = _mutant(old, new)
    failures = 0
    for check in pins.ALL_CHECKS:
        try:
            check(mod)
        except Exception:  # any failure, including a crash, counts as caught
            failures += 1
    assert failures > 0, f"no pin caught: {new!r}"


def test_unmutated_copy_passes():
    mod = _mutant("BREAKDOWN_RTOL = 1e-12", "BREAKDOWN_RTOL = 1e-12")
    for check in pins.ALL_CHECKS:
        check(mod)
