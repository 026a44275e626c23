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
