"""Pins of the oracle's coupling (ramp) rows against things other than themselves (no GPU).

The multi-stage problems (general form, Sec. I, eqs. (5)-(6); multi-period, Sec. IV, eq. (15);
security-constrained, Sec. V-A, eq. (20); stochastic, Sec. VI-A, eq. (31)) bound the difference
of each state's generator real power from that of one other state:
    r[b][k] = Pg_k(x_b) - Pg_k(x_parent(b)).
The pins:
  * hand-computed rows and transpose products on a four-state forest (a three-period chain plus
    one contingency of the base case), with binary-exact values;
  * telescoping: along a chain of periods the rows add up to the last period's Pg minus the
    first's;
  * relabelling the states (a permutation of the batch, parents mapped with it) permutes the rows;
  * the transpose product satisfies <C u, nu> = <u, C^T nu> for random forests, u and nu;
  * only the Pg columns enter: the other variables leave the rows unchanged, and C^T nu is zero
    outside the Pg columns; adding one vector to every state's Pg leaves the rows unchanged;
  * invalid parent indices are refused.
test_oracle_mutants.py plants sign, stride and offset mistakes in the two functions and checks
that these pins catch each one.
"""
import numpy as np
import pytest

NB, NG = 1, 2
N = 2 * NB + 2 * NG


def hand_case():
    """States 0 (base / first period), 1 and 2 (next periods), 3 (a contingency of the base)."""
    parent = np.array([-1, 0, 1, 0], np.int32)
    Pg = np.array([[1.0, 2.0], [1.5, 1.25], [0.5, 3.0], [1.0, 2.5]])
    x = np.zeros((4, N))
    x[:, :NB] = [[0.1], [-0.2], [0.3], [0.05]]          # Va: must not enter
    x[:, NB:2 * NB] = [[1.01], [0.97], [1.03], [0.99]]  # Vm: must not enter
    x[:, 2 * NB:2 * NB + NG] = Pg
    x[:, 2 * NB + NG:] = [[7.0, -7.0], [3.0, 4.0], [-1.0, 2.0], [5.0, 5.0]]   # Qg: must not enter
    return parent, x


def test_hand_rows(oracle_mod):
    parent, x = hand_case()
    r = oracle_mod.coupling(parent, x, NB, NG)
    expect = np.array([[0.0, 0.0], [0.5, -0.75], [-1.0, 1.75], [0.0, 0.5]])
    np.testing.assert_array_equal(r, expect)


def test_hand_transpose(oracle_mod):
    parent, _ = hand_case()
    nu = np.array([[9.0, 9.0], [1.0, 2.0], [3.0, 4.0], [5.0, 6.0]])   # row 0 does not exist
    out = oracle_mod.coupling_jtv(parent, nu, N, NB)
    expect = np.zeros((4, N))
    pg = slice(2 * NB, 2 * NB + NG)
    expect[0, pg] = [-6.0, -8.0]    # -nu1 - nu3: parent of states 1 and 3
    expect[1, pg] = [-2.0, -2.0]    # +nu1 - nu2
    expect[2, pg] = [3.0, 4.0]      # +nu2
    expect[3, pg] = [5.0, 6.0]      # +nu3
    np.testing.assert_array_equal(out, expect)


def test_chain_telescopes(oracle_mod):
    rng = np.random.default_rng(5)
    T, nb, ng = 9, 4, 3
    n = 2 * nb + 2 * ng
    x = rng.normal(size=(T, n))
    parent = np.arange(-1, T - 1, dtype=np.int32)
    r = oracle_mod.coupling(parent, x, nb, ng)
    pg = slice(2 * nb, 2 * nb + ng)
    np.testing.assert_allclose(r.sum(axis=0), x[T - 1, pg] - x[0, pg], rtol=0, atol=1e-13)
    np.testing.assert_array_equal(r[0], 0.0)


def random_forest(rng, B, roots):
    """Parents of a random forest over B states with the given number of roots."""
    order = rng.permutation(B)
    parent = np.full(B, -1, np.int32)
    for j in range(roots, B):
        parent[order[j]] = order[rng.integers(0, j)]
    return parent


def test_relabelling_permutes_rows(oracle_mod):
    rng = np.random.default_rng(6)
    B, nb, ng = 12, 3, 4
    n = 2 * nb + 2 * ng
    parent = random_forest(rng, B, 2)
    x = rng.normal(size=(B, n))
    r = oracle_mod.coupling(parent, x, nb, ng)
    perm = rng.permutation(B)           # new state j is old state perm[j]
    inv = np.argsort(perm)
    parent2 = np.array([inv[parent[p]] if parent[p] >= 0 else -1 for p in perm], np.int32)
    r2 = oracle_mod.coupling(parent2, x[perm], nb, ng)
    np.testing.assert_array_equal(r2, r[perm])


@pytest.mark.parametrize("seed,B,roots", [(7, 1, 1), (8, 16, 1), (9, 40, 5), (10, 64, 64)])
def test_transpose_identity(oracle_mod, seed, B, roots):
    rng = np.random.default_rng(seed)
    nb, ng = 5, 3
    n = 2 * nb + 2 * ng
    parent = random_forest(rng, B, roots)
    u = rng.normal(size=(B, n))
    nu = rng.normal(size=(B, ng))
    Cu = oracle_mod.coupling(parent, u, nb, ng)
    CTnu = oracle_mod.coupling_jtv(parent, nu, n, nb)
    lhs = float(np.sum(Cu * nu))
    rhs = float(np.sum(u * CTnu))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_only_generator_power_enters(oracle_mod):
    rng = np.random.default_rng(11)
    B, nb, ng = 10, 4, 3
    n = 2 * nb + 2 * ng
    parent = random_forest(rng, B, 2)
    x = rng.normal(size=(B, n))
    r = oracle_mod.coupling(parent, x, nb, ng)
    other = np.ones(n, bool)
    other[2 * nb:2 * nb + ng] = False
    y = x.copy()
    y[:, other] += rng.normal(size=(B, int(other.sum())))
    np.testing.assert_array_equal(oracle_mod.coupling(parent, y, nb, ng), r)
    z = x.copy()
    z[:, 2 * nb:2 * nb + ng] += rng.normal(size=ng)   # the same shift for every state
    np.testing.assert_allclose(oracle_mod.coupling(parent, z, nb, ng), r, rtol=0, atol=1e-14)
    np.testing.assert_array_equal(r[parent < 0], 0.0)
    out = oracle_mod.coupling_jtv(parent, rng.normal(size=(B, ng)), n, nb)
    np.testing.assert_array_equal(out[:, other], 0.0)


@pytest.mark.parametrize("bad", [[-2, 0], [0, 0], [-1, 2], [1, 0, 5]])
def test_invalid_parents_refused(oracle_mod, bad):
    B = len(bad)
    with pytest.raises(ValueError):
        oracle_mod.coupling(np.array(bad, np.int32), np.zeros((B, N)), NB, NG)
    with pytest.raises(ValueError):
        oracle_mod.coupling_jtv(np.array(bad, np.int32), np.zeros((B, NG)), N, NB)
