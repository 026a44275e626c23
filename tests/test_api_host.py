"""Host-side API logic (no GPU): pyttb's mode specification for ttv."""
import pytest

import paper_2510_01495_gb300 as ttv


def test_all_modes_by_default():
    assert ttv.resolve_dims(3, 3) == ([0, 1, 2], [0, 1, 2])


def test_dims_sorted_and_vectors_paired_in_listed_order():
    # vectors given for modes 2 then 0: mode 0 takes vector 1, mode 2 vector 0
    assert ttv.resolve_dims(4, 2, dims=[2, 0]) == ([0, 2], [1, 0])
    assert ttv.resolve_dims(4, 1, dims=3) == ([3], [0])


def test_one_vector_per_tensor_mode_selects_by_mode():
    assert ttv.resolve_dims(4, 4, dims=[3, 1]) == ([1, 3], [1, 3])
    assert ttv.resolve_dims(4, 4, exclude_dims=[2]) == ([0, 1, 3], [0, 1, 3])


def test_exclude_dims_is_the_complement():
    assert ttv.resolve_dims(4, 3, exclude_dims=2) == ([0, 1, 3], [0, 1, 2])
    assert ttv.resolve_dims(5, 1, exclude_dims=[0, 1, 3, 4]) == ([2], [0])


@pytest.mark.parametrize("args", [
    dict(d=3, nvec=1, dims=[0], exclude_dims=[1]),      # both
    dict(d=3, nvec=4),                                  # more vectors than modes
    dict(d=3, nvec=2, dims=[0]),                        # count mismatch
    dict(d=3, nvec=2, dims=[0, 0]),                     # repeated mode
    dict(d=3, nvec=1, dims=[3]),                        # out of range
    dict(d=3, nvec=1, exclude_dims=[-1, 0]),            # out of range
])
def test_invalid_specifications(args):
    with pytest.raises(ValueError):
        ttv.resolve_dims(args.pop("d"), args.pop("nvec"), **args)


def test_sptensor_arrays_of_sparse_and_dense_results():
    import torch
    subs = torch.tensor([[0, 1], [2, 0]], dtype=torch.int64)
    vals = torch.tensor([1.5, -2.0], dtype=torch.float64)
    s, v, shp = ttv.Result(subs, vals, (3, 2), False).to_sptensor_arrays()
    assert s.tolist() == [[0, 1], [2, 0]] and v.tolist() == [[1.5], [-2.0]] and shp == (3, 2)
    dense = torch.tensor([[0.0, 1.5], [0.0, 0.0], [-2.0, 0.0]], dtype=torch.float64)
    s, v, shp = ttv.Result(None, dense, (3, 2), True).to_sptensor_arrays()
    # the nonzero cells, in row-major (pyttb unique) order, values as a column
    assert s.tolist() == [[0, 1], [2, 0]] and v.tolist() == [[1.5], [-2.0]] and shp == (3, 2)


def test_out_structured_view_matches_the_c_struct():
    """The binding reads every batch result's size, order, shape and format in
    one pass over the ttv_out array through a numpy view: the view's fields
    must sit where the ctypes struct (the C layout) has them."""
    import ctypes
    import numpy as np
    from paper_2510_01495_gb300 import Out, _OUT_DTYPE, TTV_MAX_D
    assert _OUT_DTYPE.itemsize == ctypes.sizeof(Out)
    arr = (Out * 3)()
    arr[1].nnz, arr[1].is_dense, arr[1].order = 77, 1, 2
    arr[1].shape[0], arr[1].shape[1] = 5, 6
    arr[2].nnz, arr[2].order, arr[2].shape[TTV_MAX_D - 1] = -1, TTV_MAX_D, 9
    a = np.frombuffer(arr, dtype=_OUT_DTYPE, count=3)
    assert a["nnz"].tolist() == [0, 77, -1]
    assert a["is_dense"].tolist() == [0, 1, 0]
    assert a["order"].tolist() == [0, 2, TTV_MAX_D]
    assert a["shape"][1].tolist()[:2] == [5, 6] and a["shape"][2].tolist()[-1] == 9


def test_batch_results_are_formed_on_access():
    """BatchResults: a view per problem of the batch's buffers, sized by the
    run's result count; sparse rows and dense arrays; slices and iteration."""
    import torch
    from paper_2510_01495_gb300 import BatchResults
    ov0, os0 = torch.arange(10, dtype=torch.float64), torch.arange(20, dtype=torch.int64).view(10, 2)
    ov1 = torch.arange(6, dtype=torch.float64)
    meta = [(ov0, os0, (4, 4), [0]), (ov1, None, (2, 3), [1])]
    info = [(3, False, 2, (4, 4, 0, 0, 0, 0, 0, 0)), (6, True, 2, (2, 3, 0, 0, 0, 0, 0, 0))]
    res = BatchResults(meta, info)
    assert len(res) == 2
    r0, r1 = res
    assert not r0.is_dense and r0.shape == (4, 4) and r0.vals.tolist() == [0.0, 1.0, 2.0]
    assert r0.subs.tolist() == [[0, 1], [2, 3], [4, 5]]
    assert r1.is_dense and r1.subs is None and tuple(r1.vals.shape) == (2, 3)
    assert [r.shape for r in res[0:2]] == [(4, 4), (2, 3)]
