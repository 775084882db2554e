"""The binding refuses malformed tpcf_count arguments before anything reaches the C ABI.

The library receives raw pointers and cannot know buffer sizes, so a float32
catalogue, a transposed array or offsets that do not match the randoms would
make its kernels read past the caller's allocation.  These checks run on the
host with CPU tensors (no GPU needed): validate_count_args is the same function
Context.tpcf_count calls first.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def tp():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2205_11852_gb300 as tp
    return tp


DEV = None


def _ok():
    return {"data": torch.zeros(5, 3, dtype=torch.float64), "randoms": torch.zeros(8, 3, dtype=torch.float64),
            "offsets": [0, 4, 8]}


def test_well_formed_mocks_pass(tp):
    host, M = tp.validate_count_args([_ok(), _ok()], 10, torch.device("cuda", 0))
    assert host and M == 2
    u = {"data_u32": torch.zeros(3, 5, dtype=torch.int32), "randoms_u32": torch.zeros(3, 8, dtype=torch.int32),
         "offsets": [0, 3, 8]}
    assert tp.validate_count_args([u], 10, torch.device("cuda", 0)) == (True, 2)


@pytest.mark.parametrize("bad,what", [
    ({"data": torch.zeros(5, 3, dtype=torch.float32)}, "dtype"),
    ({"data": torch.zeros(3, 5, dtype=torch.float64)}, "shape"),
    ({"randoms": torch.zeros(6, 3, dtype=torch.float64)}, "offsets[-1]"),
    ({"randoms": torch.zeros(16, 3, dtype=torch.float64)[::2]}, "contiguous"),
    ({"offsets": [0, 4, 7]}, "offsets[-1]"),
    ({"offsets": [1, 4, 8]}, "start at 0"),
    ({"offsets": [0, 6, 4, 8]}, "non-decreasing"),
    ({"data_u32": torch.zeros(5, 3, dtype=torch.int32)}, "one of"),
    ({"data": None, "data_u32": torch.zeros(5, 3, dtype=torch.int32)}, "shape"),
    ({"data": None, "data_u32": torch.zeros(3, 5, dtype=torch.int64)}, "dtype"),
])
def test_malformed_mocks_refused(tp, bad, what):
    mk = _ok()
    mk.update(bad)
    if mk.get("data") is None:
        mk.pop("data")
    with pytest.raises(tp.TpcfArgError) as e:
        tp.validate_count_args([mk], 10, torch.device("cuda", 0))
    assert e.value.code == tp.TPCF_ERR_ARG
    assert what in str(e.value)


def test_mixed_subset_counts_refused(tp):
    a, b = _ok(), _ok()
    b["offsets"] = [0, 8]
    with pytest.raises(tp.TpcfArgError):
        tp.validate_count_args([a, b], 10, torch.device("cuda", 0))


def test_output_tensors_checked(tp):
    out = {"dd": torch.zeros(1, 10, dtype=torch.int32)}
    with pytest.raises(tp.TpcfArgError) as e:
        tp.validate_count_args([_ok()], 10, torch.device("cpu"), out)
    assert "dd" in str(e.value)
