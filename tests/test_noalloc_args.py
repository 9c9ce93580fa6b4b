"""Argument checks of the allocation-free entry point's binding, on the CPU: the library cannot see
the sizes of the arrays it is given, so the binding checks shape, length, type and device first."""

import pytest

from paper_2002_02150_gb300.fcas import array_desc, check_noalloc_arrays

TH = (True, "float64", True, 0, (5, 4))
FIT = (True, "float64", True, 0, (5,))
TC = (True, "int64", True, 0, (5,))


def test_valid_arguments_give_the_particle_count():
    assert check_noalloc_arrays(TH, FIT, TC, 0) == 5
    assert check_noalloc_arrays(TH, (True, "float64", True, 0, (9,)), TC, 0) == 5   # longer outputs are fine


@pytest.mark.parametrize("args,err,match", [
    (((True, "float64", True, 0, (5, 3)), FIT, TC), ValueError, "shape"),
    (((True, "float64", True, 0, (20,)), FIT, TC), ValueError, "shape"),
    ((TH, (True, "float64", True, 0, (4,)), TC), ValueError, "need 5 elements"),
    ((TH, FIT, (True, "int64", True, 0, (4,))), ValueError, "need 5 elements"),
    ((TH, FIT, (True, "int64", True, 1, (5,))), ValueError, "cuda:1"),
    (((True, "float64", True, 1, (5, 4)), FIT, TC), ValueError, "cuda:1"),
    ((TH, FIT, (True, "int32", True, 0, (5,))), TypeError, "int64"),
    ((TH, (True, "float32", True, 0, (5,)), TC), TypeError, "float64"),
    (((True, "float64", False, 0, (5, 4)), FIT, TC), TypeError, "contiguous"),
    (((False, "float64", True, None, (5, 4)), FIT, TC), TypeError, "CUDA"),
])
def test_each_rejection(args, err, match):
    with pytest.raises(err, match=match):
        check_noalloc_arrays(*args, current_device=0)


def test_host_arrays_are_described_as_host_memory():
    import numpy as np
    import torch
    assert array_desc(np.zeros((3, 4)))[:2] == (False, "float64")
    assert array_desc(torch.zeros(3, dtype=torch.int64))[:2] == (False, "int64")
    with pytest.raises(TypeError):
        check_noalloc_arrays(array_desc(np.zeros((3, 4))), FIT, TC, current_device=0)
