"""Host logic of kde_sum_batches (uneven query batches against one reference
tree): consecutive batches grouped under a query budget, a group whose call
reports DFGT_ECAPACITY halved and retried, every batch's rows returned in
order.  The trees and sums are fakes, so no GPU is needed."""
import pytest
import torch

import paper_1102_2878_gb300 as dfgt


class FakeTree:
    def __init__(self, ctx, q, **kw):
        self.q = q
        self.n = q.shape[0]

    def close(self):
        pass


def fake_rows(q, hs):
    return torch.stack([q[:, 0].double() * (i + 1) for i in range(len(hs))])


@pytest.mark.parametrize("log", [False, True])
def test_groups_and_capacity_halving(monkeypatch, log):
    calls = []
    limit = 7  # a query tree above 7 points "overflows"

    def fake_sum(ctx, qt, rt, hs, eps):
        calls.append(qt.n)
        if qt.n > limit:
            raise dfgt.DFGTError(4, "frontier exceeds the capacity")
        return fake_rows(qt.q, hs), {"rounds": 1, "ms_base": 0.5}

    def fake_sum_log(ctx, qt, rt, hs, eps):
        G, st = fake_sum(ctx, qt, rt, hs, eps)
        return G, torch.log(G + 1.0), st

    monkeypatch.setattr(dfgt, "Tree", FakeTree)
    monkeypatch.setattr(dfgt, "kde_sum", fake_sum)
    monkeypatch.setattr(dfgt, "kde_sum_log", fake_sum_log)
    sizes = [3, 3, 2, 4, 5]
    batches = [torch.arange(m, dtype=torch.float32).reshape(-1, 1) + 100 * b for b, m in enumerate(sizes)]
    hs = [1.0, 2.0]
    outs, st = dfgt.kde_sum_batches(None, batches, None, hs, 1e-2, max_queries=8, log=log)
    # groups of at most 8 queries: [0, 1, 2] (8, overflows, halved into [0] and
    # [1, 2]), [3], [4]
    assert calls == [8, 3, 5, 4, 5]
    assert st == {"rounds": 4, "ms_base": 2.0}
    assert len(outs) == len(batches)
    for b, out in zip(batches, outs):
        G = out[0] if log else out
        assert torch.equal(G, fake_rows(b, hs))
        if log:
            assert torch.equal(out[1], torch.log(G + 1.0))


def test_single_batch_over_capacity_raises(monkeypatch):
    def fake_sum(ctx, qt, rt, hs, eps):
        raise dfgt.DFGTError(4, "frontier exceeds the capacity")

    monkeypatch.setattr(dfgt, "Tree", FakeTree)
    monkeypatch.setattr(dfgt, "kde_sum", fake_sum)
    with pytest.raises(dfgt.DFGTError, match="DFGT_ECAPACITY"):
        dfgt.kde_sum_batches(None, [torch.zeros(4, 1)], None, [1.0], 1e-2)


def test_other_errors_are_not_retried(monkeypatch):
    calls = []

    def fake_sum(ctx, qt, rt, hs, eps):
        calls.append(qt.n)
        raise dfgt.DFGTError(5, "a grid barrier wait timed out")

    monkeypatch.setattr(dfgt, "Tree", FakeTree)
    monkeypatch.setattr(dfgt, "kde_sum", fake_sum)
    with pytest.raises(dfgt.DFGTError, match="DFGT_ETIMEOUT"):
        dfgt.kde_sum_batches(None, [torch.zeros(2, 1), torch.zeros(2, 1)], None, [1.0], 1e-2)
    assert calls == [4]


def test_adjacent_batches_are_used_in_place(monkeypatch):
    # batches that are consecutive slices of one tensor form their group's
    # query set without a copy; separate tensors are concatenated
    seen = []

    def fake_sum(ctx, qt, rt, hs, eps):
        seen.append((qt.q.data_ptr(), qt.q.shape))
        return fake_rows(qt.q, hs), {"rounds": 1}

    monkeypatch.setattr(dfgt, "Tree", FakeTree)
    monkeypatch.setattr(dfgt, "kde_sum", fake_sum)
    base = torch.arange(24, dtype=torch.float32).reshape(12, 2)
    parts = list(torch.split(base, [3, 4, 5]))
    outs, _ = dfgt.kde_sum_batches(None, parts, None, [1.0], 1e-2, max_queries=7)
    assert seen[0] == (base.data_ptr(), torch.Size([7, 2]))  # batches 0 and 1 in place
    assert seen[1][1] == torch.Size([5, 2])
    for b, G in zip(parts, outs):
        assert torch.equal(G, fake_rows(b, [1.0]))
    seen.clear()
    apart = [torch.zeros(3, 2), torch.ones(4, 2)]
    dfgt.kde_sum_batches(None, apart, None, [1.0], 1e-2)
    assert seen[0][1] == torch.Size([7, 2]) and seen[0][0] not in (apart[0].data_ptr(), apart[1].data_ptr())
