"""Dense dot product (Eq. 1) and matrix-vector product (Eq. 2) on the GPU
against the CPU oracle, element by element, at sizes that span several CTAs
and column chunks with ragged tails, up to the paper's largest sizes."""
import numpy as np
import pytest
import torch

import oracle
import paper_2510_01495_gb300 as ttv
import synthetic as S
from parity import assert_close

pytestmark = pytest.mark.gpu


def vec(seed, n, lo=0.0, hi=1.0, dtype=torch.float64, device="cpu"):
    return S.uniform(seed, 1, n, lo, hi, device=device).to(dtype)


def check_dot(x, y, what):
    got = float(ttv.dot(x.cuda(), y.cuda()).cpu())
    xs, ys = x.cpu().double().numpy(), y.cpu().double().numpy()
    ref = oracle.dot(xs, ys)
    A = oracle.dot(np.abs(xs), np.abs(ys))
    assert_close([got], [ref], [A], what=what)
    return got


@pytest.mark.parametrize("n", [0, 1, 2, 3, 255, 1000, 1001, 123_457, 2_000_001])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_dot_sizes(cuda_lib, n, dtype):
    check_dot(vec(n + 1, n, dtype=dtype), vec(n + 2, n, -1.0, 1.0, dtype=dtype), f"dot n={n} {dtype}")


def test_dot_unaligned_and_deterministic(cuda_lib):
    x, y = vec(5, 300_001), vec(6, 300_001)
    dx, dy = x.cuda(), y.cuda()
    # views starting one element in: not 16-byte aligned, elementwise loads
    a = float(ttv.dot(dx[1:], dy[1:]).cpu())
    assert_close([a], [oracle.dot(x[1:].numpy(), y[1:].numpy())], [oracle.dot(x[1:].numpy(), y[1:].numpy())],
                 what="unaligned")
    r1, r2 = ttv.dot(dx, dy), ttv.dot(dx, dy)
    assert torch.equal(r1, r2)


def test_dot_paper_size(cuda_lib):
    n = 100_000_000          # the paper's largest vector (Sec. 4.1)
    check_dot(vec(7, n, device="cuda"), vec(8, n, device="cuda"), "dot n=1e8")


def check_matvec(A, x, what):
    y = ttv.matvec(A.cuda() if not A.is_cuda else A, x.cuda()).cpu().numpy()
    Ah = A.cpu().double().numpy()
    xh = x.cpu().double().numpy()
    ref = oracle.matvec(Ah, xh)
    absref = oracle.matvec(np.abs(Ah), np.abs(xh))
    assert_close(y, ref, absref, what=what)


@pytest.mark.parametrize("shape", [(1, 1), (1, 1000), (1000, 1), (2, 3), (100, 100), (100, 100_000),
                                   (100_000, 100), (3000, 3001), (77, 4097)])
@pytest.mark.parametrize("order", ["C", "F"])
def test_matvec_shapes(cuda_lib, shape, order):
    n1, n2 = shape
    A = vec(n1 * 7 + n2, n1 * n2, -1.0, 1.0).reshape(n1, n2)
    if order == "F":
        A = A.t().contiguous().t()
    check_matvec(A, vec(n2, n2), f"matvec {shape} {order}")


def test_matvec_float32_views_and_determinism(cuda_lib):
    A = vec(11, 500 * 800, dtype=torch.float32).reshape(500, 800)
    x = vec(12, 800, dtype=torch.float32)
    check_matvec(A, x, "float32")
    dA = A.cuda()
    check_matvec(dA[::3, :], x, "every third row")              # row stride 3*800, column stride 1
    check_matvec(dA.t()[:, ::2], vec(13, 250, dtype=torch.float32), "transposed, every second column")
    y1, y2 = ttv.matvec(dA, x.cuda()), ttv.matvec(dA, x.cuda())
    assert torch.equal(y1, y2)
    with pytest.raises(ttv.TTVError) as e:
        ttv.matvec(dA[:, ::2], vec(14, 400, dtype=torch.float32).cuda())
    assert e.value.name == "TTV_ERR_UNSUPPORTED"


def test_matvec_empty(cuda_lib):
    y = ttv.matvec(torch.zeros((4, 0), dtype=torch.float64, device="cuda"),
                   torch.zeros(0, dtype=torch.float64, device="cuda"))
    assert y.cpu().tolist() == [0.0] * 4
    assert ttv.matvec(torch.zeros((0, 5), dtype=torch.float64, device="cuda"),
                      torch.ones(5, dtype=torch.float64, device="cuda")).numel() == 0


@pytest.mark.parametrize("shape", [(1_000_000, 100), (100, 1_000_000), (10_000, 10_000)])
def test_matvec_paper_sizes(cuda_lib, shape):
    """The largest matrices of the paper's three matrix-vector experiments
    (Sec. 4.2), stored row-major and column-major."""
    n1, n2 = shape
    dA = vec(n1 + n2, n1 * n2, device="cuda").reshape(n1, n2)
    x = vec(3, n2)
    check_matvec(dA, x, f"{shape} C")
    check_matvec(dA.t().contiguous().t(), x, f"{shape} F")
