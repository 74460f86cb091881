"""The FP64 adjoint oracle against its pins, and planted mistakes caught."""
import inspect
import types

import pytest

import oracle.adjoint as oa
from tests import pins_adjoint


@pytest.mark.parametrize("check", pins_adjoint.ADJ_CHECKS, ids=lambda f: f.__name__)
def test_adjoint_pin(check):
    check(oa)


MUTATIONS = [
    # second half of the symmetric edge gradient dropped
    ('g = np.einsum("ek,ek->e", P[i], U[j]) + np.einsum("ek,ek->e", P[j], U[i])',
     'g = 2 * np.einsum("ek,ek->e", P[i], U[j])'),
    # roles of the two bases swapped in M's weights
    ("M = b0w * b01 * (Qw * Qw[0, :]) @ Phi @ (Q1 * Q1[0, :]).T",
     "M = b0w * b01 * (Qw * Q1[0, :]) @ Phi @ (Q1 * Qw[0, :]).T"),
    # missing ||w||
    ("M = b0w * b01 * (Qw * Qw[0, :])", "M = b01 * (Qw * Qw[0, :])"),
    # divided difference with the wrong exponent
    ("Phi = np.exp(nu[None, :] - theta) * np.expm1(d) / d",
     "Phi = np.exp(mu[:, None] - theta) * np.expm1(d) / d"),
    # block exponential with the coupling block transposed
    ("big[:n, n:] = np.outer(w, np.ones(n))", "big[:n, n:] = np.outer(np.ones(n), w)"),
    # Daleckii-Krein without the divided differences
    ("return Q @ (divided_exp(lam) * C) @ Q.T", "return Q @ (np.exp(lam)[:, None] * C) @ Q.T"),
    # edge gradient misses G_ji
    ("return G[i, j] + G[j, i]", "return 2 * G[i, j]"),
    # ensemble: the shift applied the wrong way round
    ("math.exp(t - theta_star) * g for t, g in parts",
     "math.exp(theta_star - t) * g for t, g in parts"),
    # ensemble: the last realisation dropped
    ("np.concatenate([math.exp(t - theta_star) * g for t, g in parts])",
     "np.concatenate([math.exp(t - theta_star) * g for t, g in parts[:-1]])"),
    # ensemble: nodes past the realisation's range not filtered out
    ("sel = np.asarray([x for x in nodes if x < n], dtype=np.int64)",
     "sel = np.asarray([x for x in nodes], dtype=np.int64)"),
    # ensemble: nodes past the range wrapped into it instead of dropped
    ("sel = np.asarray([x for x in nodes if x < n], dtype=np.int64)",
     "sel = np.asarray([x % n for x in nodes], dtype=np.int64)"),
    # ensemble: the common shift is the smallest instead of the largest
    ("theta_star = max(p[0] for p in parts)", "theta_star = min(p[0] for p in parts)"),
]


@pytest.mark.parametrize("old,new", MUTATIONS, ids=[f"m{i}" for i in range(len(MUTATIONS))])
def test_planted_adjoint_mistake_is_caught(old, new):
    src = inspect.getsource(oa)
    assert src.count(old) >= 1, old
    mod = types.ModuleType("oracle.adjoint_mutant")
    mod.__package__ = "oracle"
    exec(compile(src.replace(old, new, 1), "oracle_adjoint_mutant", "exec"), mod.__dict__)
    failures = 0
    for check in pins_adjoint.ADJ_CHECKS:
        try:
            check(mod)
        except Exception:
            failures += 1
    assert failures > 0, f"no pin caught: {new!r}"
