"""Host-side argument checks of the Python binding (no GPU needed).

The C ABI takes raw pointers and sizes, so it cannot see whether a buffer is
as large as the plan's layout says.  The binding checks every tensor it hands
over (shape, dtype, contiguity, device) and the number of per-plan entries,
and raises before any pointer crosses the boundary.
"""

import pytest

torch = pytest.importorskip("torch")

from paper_1203_4587_gb300 import binding  # noqa: E402


def c64(*shape):
    return torch.zeros(shape, dtype=torch.complex64)


def test_need_accepts_the_exact_layout():
    t = c64(3, 2, 8, 5)
    assert binding._need(t, (3, 2, 8, 5), "k", "cpu") is t
    assert binding._need(t, (3, 2, 8, 5), "k", None) is t


@pytest.mark.parametrize("bad,err", [
    (c64(3, 2, 8, 6), ValueError),                                   # one column too many
    (c64(3, 2, 8), ValueError),                                      # a dimension missing
    (torch.zeros((3, 2, 8, 5), dtype=torch.complex128), TypeError),  # complex128 is twice the bytes
    (torch.zeros((3, 2, 8, 5), dtype=torch.float32), TypeError),
    (c64(3, 2, 5, 8).transpose(2, 3), ValueError),                   # right shape, strided view
    ("not a tensor", TypeError),
])
def test_need_rejects(bad, err):
    with pytest.raises(err):
        binding._need(bad, (3, 2, 8, 5), "k", "cpu")


def test_need_checks_the_device():
    with pytest.raises(ValueError, match="cuda tensor is expected"):
        binding._need(c64(2, 3), (2, 3), "out", "cuda")


def test_need_count():
    assert binding._need_count((a for a in "xy"), 2, "kspaces") == ["x", "y"]
    for n in (1, 3):
        with pytest.raises(ValueError, match="entries for"):
            binding._need_count(["x", "y"], n, "kspaces")


@pytest.mark.parametrize("shape,ok", [
    ((4, 32), True), ((4, 32, 16), True),
    ((4, 31), False), ((4, 32, 15), False), ((4,), False), ((4, 32, 16, 1), False),
])
def test_mask_shapes(shape, ok):
    assert binding._mask_shape_ok(shape, True, 32, 16) == ok
