"""GPU parity of the batched products (many independent C_p = A_p * B_p in
one plan): every product of the batch against the CPU oracle, each product
the same alone and in the batch, empty products, and a bad product caught."""
import numpy as np
import pytest
import torch

import oracle
from paper_1804_01698_gb300 import inputs
from paper_1804_01698_gb300.inputs import CSR
from gpu_helpers import assert_matches_oracle, gpu_product

pytestmark = pytest.mark.gpu


def mixed_batch(dtype):
    prods = []
    for A in inputs.er_batch(24, seed=501, n_lo=64, n_hi=4000, k_lo=2, k_hi=32):
        prods.append((A, A))
    for g in (3, 6, 9):                                  # AMG-style A * P
        prods.append((inputs.poisson7(g), inputs.aggregation(g)))
    prods.append((inputs.rmat(11, 16, seed=502), inputs.rmat(11, 16, seed=502)))
    z = CSR(0, 5, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    b5 = inputs.er_exact(5, 2, seed=503, ncols=7)
    prods.insert(5, (z, b5))                             # a product with no rows
    e = CSR(4, 5, np.zeros(5, np.int32), np.zeros(0, np.int32), np.zeros(0))
    prods.insert(9, (e, b5))                             # rows but no entries
    if dtype == torch.int64:
        prods = [(a.with_vals(np.round(a.vals * 3).astype(np.int64)), b.with_vals(np.round(b.vals * 3).astype(np.int64)))
                 for a, b in prods]
    return prods


@pytest.mark.parametrize("dt", [torch.float64, torch.int64, torch.float32])
@pytest.mark.parametrize("sorted_output", [True, False])
def test_batch_matches_oracle_per_product(dt, sorted_output):
    from paper_1804_01698_gb300 import binding as sg
    prods = mixed_batch(dt)
    npdt = {torch.float64: np.float64, torch.float32: np.float32, torch.int64: np.int64}[dt]
    if dt == torch.float32:   # small integers: exact in float32
        prods = [(a.with_vals(np.round(a.vals * 3)), b.with_vals(np.round(b.vals * 3))) for a, b in prods]
    prods = [(a.astype(npdt), b.astype(npdt)) for a, b in prods]
    dAs = [sg.to_device(a, "cuda", dt) for a, _ in prods]
    dBs = [sg.to_device(b, "cuda", dt) for _, b in prods]
    with sg.Batch(dAs, dBs, sorted_output) as batch:
        batch.symbolic()
        batch.numeric()
        st = batch.plan_stats()
        torch.cuda.synchronize()
        assert st["status"] == 0
        rp_host = batch.c_row_ptr.cpu().numpy()
        for p, (a, b) in enumerate(prods):
            assert_matches_oracle(batch.product(p, rp_host), a, b, sorted_output)


def test_each_product_is_the_same_alone_and_in_the_batch():
    from paper_1804_01698_gb300 import binding as sg
    prods = mixed_batch(torch.int64)
    dAs = [sg.to_device(a) for a, _ in prods]
    dBs = [sg.to_device(b) for _, b in prods]
    with sg.Batch(dAs, dBs, True) as batch:
        batch.symbolic()
        batch.numeric()
        torch.cuda.synchronize()
        rp_host = batch.c_row_ptr.cpu().numpy()
        for p, (a, b) in enumerate(prods):
            alone, _ = gpu_product(a, b, torch.int64, True)
            inb = batch.product(p, rp_host)
            assert torch.equal(alone.row_ptr, inb.row_ptr)
            assert torch.equal(alone.col_idx, inb.col_idx)
            assert torch.equal(alone.vals, inb.vals)


def test_bad_product_is_reported():
    from paper_1804_01698_gb300 import binding as sg
    good = inputs.er_exact(50, 3, seed=511)
    bad = inputs.er_exact(50, 3, seed=512)
    ci = bad.col_idx.copy()
    ci[4] = 50                                           # one past the last column
    bad = CSR(bad.nrows, bad.ncols, bad.row_ptr, ci, bad.vals)
    dg, db = sg.to_device(good), sg.to_device(bad)
    with pytest.raises(sg.SpgemmError) as ei:
        sg.Batch([dg, db], [dg, dg], True)
    assert ei.value.status == -2


@pytest.mark.parametrize("where", ["col_idx", "row_ptr_end"])
def test_bad_index_in_a_later_pack_chunk_is_reported(where):
    """The pack kernel splits a large product over several blocks; a bad
    entry far into the product (past the first 8192-element chunk) is
    still found."""
    from paper_1804_01698_gb300 import binding as sg
    small = inputs.er_exact(50, 3, seed=521)
    big = inputs.er_exact(20000, 3, seed=522)           # 20001 row pointers, 60000 entries
    if where == "col_idx":
        ci = big.col_idx.copy()
        ci[40000] = -1
        big = CSR(big.nrows, big.ncols, big.row_ptr, ci, big.vals)
    else:
        rp = big.row_ptr.copy()
        rp[-1] -= 1                                      # last row pointer != nnz
        big = CSR(big.nrows, big.ncols, rp, big.col_idx, big.vals)
    ds, db = sg.to_device(small), sg.to_device(big)
    with pytest.raises(sg.SpgemmError) as ei:
        sg.Batch([ds, db], [ds, sg.to_device(inputs.er_exact(20000, 2, seed=523))], True)
    assert ei.value.status == -2
