"""CPU: the persistent schedule's work list, decoded on the host by the kernels' own decoder
(exago_test_work_list; no GPU needed).

For random and edge-case shapes -- B states of Tbr branch items and Tbu bus items, bus items
trailing branch items by a lag of states -- every (kind, state, tile) item appears exactly once,
and every wait a persistent launch makes points to a smaller ticket, which is what makes the
launch deadlock-free:
  * a bus item of state b comes after all branch items of b;
  * a branch item of state b >= ring comes after all bus items of state b - ring, for every ring
    the host may choose (ring > lag);
and the states whose bus items follow the last branch item are the closing run of lag states
plus the last group's one.
"""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def ex():
    from paper_2203_10587_gb300 import build, exago
    build.build()
    exago.lib()
    return exago


def check(ex, B, Tbr, Tbu, lag):
    kind, state, tile = ex.exago_test_work_list(B, Tbr, Tbu, lag)
    n = B * (Tbr + Tbu)
    assert len(kind) == n
    key = kind.astype(np.int64) * (n + 1) + state.astype(np.int64) * (Tbr + Tbu) + tile
    assert len(np.unique(key)) == n, "an item appears twice"
    br, bu = kind == 1, kind == 0
    assert br.sum() == B * Tbr and bu.sum() == B * Tbu
    assert np.all(tile[br] < Tbr) and np.all(tile[bu] < Tbu) and np.all((state >= 0) & (state < B))
    if Tbr == 0:
        return
    t = np.arange(n)
    last_br = np.full(B, -1)
    np.maximum.at(last_br, state[br], t[br])
    first_br = np.full(B, n)
    np.minimum.at(first_br, state[br], t[br])
    first_bu = np.full(B, n)
    np.minimum.at(first_bu, state[bu], t[bu])
    last_bu = np.full(B, -1)
    np.maximum.at(last_bu, state[bu], t[bu])
    assert np.all(first_bu > last_br), "a bus item precedes one of its state's branch items"
    for ring in (lag + 1, lag + 2, 2 * lag + 1):
        b = np.arange(ring, B)
        assert np.all(first_br[b] > last_bu[b - ring]), f"ring {ring}: slot reused too early"
    tail_states = np.unique(state[t > last_br.max()])
    assert len(tail_states) == (lag if B == lag else lag + 1)


@pytest.mark.parametrize("B,Tbr,Tbu,lag", [
    (1, 3, 2, 1), (1, 0, 4, 1), (2, 5, 3, 1), (2, 5, 3, 2), (512, 43, 32, 40), (512, 43, 32, 1),
    (50, 7, 9, 49), (41, 2, 3, 40), (3, 1, 1, 2), (300, 22, 16, 48),
])
def test_work_list_cases(ex, B, Tbr, Tbu, lag):
    check(ex, B, Tbr, Tbu, lag)


def test_work_list_random(ex):
    rng = np.random.default_rng(7)
    for _ in range(200):
        B = int(rng.integers(1, 200))
        check(ex, B, int(rng.integers(0, 12)), int(rng.integers(1, 12)), int(rng.integers(1, B + 1)))


def test_work_list_rejects_bad_arguments(ex):
    for args in ((0, 1, 1, 1), (4, 1, 0, 1), (4, 1, 1, 0), (4, 1, 1, 5), (4, -1, 1, 1)):
        with pytest.raises(ex.ExagoError) as ei:
            ex.exago_test_work_list(*args)
        assert ei.value.name == "EXAGO_EINVAL"
