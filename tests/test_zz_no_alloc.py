"""The allocation-free entry point, checked against the library's own cycle end.

mcgb_bank_offsets_noalloc serves callers that cannot give the library device
memory (their GPU memory belongs to another allocator, or they may not allocate
while running): it takes device pointers and keeps its scratch in a fixed array
inside the library.  Its result must equal what mcgb_run_eigenvalue's own bank
ordering produced: the first position of each history's sites in the
(parent, child) ordered bank, and the bank size.  Two calls in a row share the
array; both must be right.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _expected_first(n_fis, parents, n):
    first = np.zeros(n, dtype=np.int64)
    first[1:] = np.cumsum(n_fis)[:-1]
    # the ordered bank from the existing entry point: parent j's sites start at first[j]
    starts = {}
    for pos, p in enumerate(parents):
        starts.setdefault(int(p), pos)
    return first, starts


def test_noalloc_bank_offsets_match_the_library_cycle_end():
    import torch

    import paper_2501_05440_gb300 as m
    m.build()
    torch.cuda.init()
    n = 30000
    pb = W.pin_cell_mg(n=n, inactive=1, active=1)
    c = m.Context(record_histories=True)
    m.load_problem(c, pb).run()
    h, bank = c.get_histories(), c.get_bank()
    nfis = h["n_fis"]
    assert int(nfis.sum()) == len(bank["parent"])
    first_ref, starts = _expected_first(nfis, bank["parent"], n)
    for j, pos in starts.items():
        assert first_ref[j] == pos

    stream = torch.cuda.current_stream()
    d_in = torch.from_numpy(nfis.astype(np.int32)).cuda()
    for call in range(2):
        d_first = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        d_total = torch.full((1,), -7, dtype=torch.int32, device="cuda")
        m.bank_offsets_noalloc(d_in.data_ptr(), n, d_first.data_ptr(), d_total.data_ptr(),
                               stream.cuda_stream)
        torch.cuda.synchronize()
        assert np.array_equal(d_first.cpu().numpy().astype(np.int64), first_ref), call
        assert int(d_total.item()) == len(bank["parent"]), call
    # a second, larger input spanning several scan tiles with a ragged end
    rng = np.random.default_rng(5)
    big = rng.integers(0, 4, size=4096 * 37 + 123).astype(np.int32)
    d_big = torch.from_numpy(big).cuda()
    d_first = torch.empty(len(big), dtype=torch.int32, device="cuda")
    d_total = torch.empty(1, dtype=torch.int32, device="cuda")
    m.bank_offsets_noalloc(d_big.data_ptr(), len(big), d_first.data_ptr(), d_total.data_ptr(),
                           stream.cuda_stream)
    torch.cuda.synchronize()
    ref = np.concatenate([[0], np.cumsum(big)[:-1]])
    assert np.array_equal(d_first.cpu().numpy(), ref)
    assert int(d_total.item()) == int(big.sum())


def test_noalloc_rejects_oversized_input():
    import paper_2501_05440_gb300 as m
    with pytest.raises(m.McgbError) as e:
        m.bank_offsets_noalloc(1, 4096 * 4096 + 1, 1, 1, 0)
    assert e.value.code == -1
