"""Host-side argument checks of Index.search_noalloc (no GPU needed): the
C entry point takes raw pointers, so a wrong dtype, shape, layout or device
must be refused in the binding before any pointer reaches the library."""
import pytest

torch = pytest.importorskip("torch")

from paper_2308_15014_gb300 import check_noalloc_args  # noqa: E402

d, L, k, nq = 16, 3, 5, 7


def _ok():
    return (torch.zeros(nq, d), torch.zeros(nq, L, dtype=torch.int32),
            torch.zeros(nq, k, dtype=torch.int64), torch.zeros(nq, k))


@pytest.mark.parametrize("i,bad,msg", [
    (0, torch.zeros(nq, d, dtype=torch.float64), "float32"),
    (0, torch.zeros(nq, d, dtype=torch.float16), "float32"),
    (0, torch.zeros(nq, d + 1), "shape"),
    (0, torch.zeros(d, nq).t(), "contiguous"),
    (1, torch.zeros(nq, L, dtype=torch.int64), "int32"),
    (1, torch.zeros(nq - 1, L, dtype=torch.int32), "shape"),
    (2, torch.zeros(nq, k, dtype=torch.int32), "int64"),
    (2, torch.zeros(nq, k - 1, dtype=torch.int64), "shape"),
    (3, torch.zeros(nq, k, dtype=torch.float64), "float32"),
    (3, torch.zeros(nq + 1, k), "shape"),
    (3, [[0.0] * k] * nq, "torch tensor"),
])
def test_noalloc_refuses_bad_arguments(i, bad, msg):
    args = list(_ok())
    args[i] = bad
    with pytest.raises(ValueError, match=msg):
        check_noalloc_args(args[0], args[1], k, args[2], args[3], d, L)


def test_noalloc_refuses_host_tensors():
    Q, Qb, ids, dist = _ok()
    with pytest.raises(ValueError, match="CUDA"):
        check_noalloc_args(Q, Qb, k, ids, dist, d, L)
