"""Per-kernel parity of one product (rpca_dense_pass) in both forms against an FP64 product.

FP32 form: |C - C64| <= 4e-6 * (|A| |B|) + 1e-30 (FP32 accumulation over K <= 1e5 in
short chains).  Split-BF16 form: a = a_hi + a_lo keeps 16 significant bits of
each factor, so each product term carries a relative error below 3 * 2^-16 plus
FP32 accumulation: |C - C64| <= 6e-5 * (|A| |B|).
"""
import numpy as np
import pytest

from gpu_util import cuda, to_dev, to_np

pytestmark = pytest.mark.gpu

SHAPES = [  # m, n, w   (ragged m, n; several K tiles; widths 8..256)
    (256, 128, 16), (300, 200, 8), (1000, 333, 104), (129, 1000, 32), (4097, 130, 112),
    (2000, 1000, 16), (777, 2049, 224), (5000, 64, 256), (128, 128, 128),
]


def _ref(A, B, adjoint):
    A64 = A.astype(np.float64)
    B64 = B.astype(np.float64)
    C = (A64.T @ B64) if adjoint else (A64 @ B64)
    absC = (np.abs(A64).T @ np.abs(B64)) if adjoint else (np.abs(A64) @ np.abs(B64))
    return C, absC


@pytest.mark.parametrize("precision,rtol", [("fp32", 4e-6), ("bf16x3", 6e-5)])
@pytest.mark.parametrize("adjoint", [False, True])
@pytest.mark.parametrize("m,n,w", SHAPES)
def test_pass_matches_fp64(m, n, w, adjoint, precision, rtol):
    cuda()
    import paper_1412_3510_gb300 as rp
    rng = np.random.default_rng(m * 31 + n + w)
    A = rng.standard_normal((m, n)).astype(np.float32)
    B = rng.standard_normal((m if adjoint else n, w)).astype(np.float32)
    C = to_np(rp.rpca_dense_pass(to_dev(A), to_dev(B), adjoint=adjoint, precision=precision))
    ref, absref = _ref(A, B, adjoint)
    err = np.abs(C - ref)
    assert np.all(err <= rtol * absref + 1e-30), float((err / absref).max())


def test_bf16x3_differs_from_fp32_and_unaligned_falls_back():
    cuda()
    import torch
    import paper_1412_3510_gb300 as rp
    rng = np.random.default_rng(5)
    A = to_dev(rng.standard_normal((512, 300)).astype(np.float32))
    B = to_dev(rng.standard_normal((300, 64)).astype(np.float32))
    c32 = rp.rpca_dense_pass(A, B, precision="fp32")
    ctc = rp.rpca_dense_pass(A, B, precision="bf16x3")
    assert not torch.equal(c32, ctc)                      # the tensor-core form really ran
    big = torch.zeros(512, 301, device="cuda")
    big[:, :300] = A
    cfb = rp.rpca_dense_pass(big[:, :300], B, precision="bf16x3")   # lda = 301: FP32 fallback
    assert torch.equal(cfb, c32)


def test_bf16x3_special_values():
    cuda()
    import paper_1412_3510_gb300 as rp
    # exactly representable in BF16: the split is exact and so is the product
    A = np.zeros((256, 192), dtype=np.float32)
    A[np.arange(192), np.arange(192)] = 2.0
    A[200:, :] = 0.5
    B = np.arange(192 * 16, dtype=np.float32).reshape(192, 16) % 7 - 3
    C = to_np(rp.rpca_dense_pass(to_dev(A), to_dev(B), precision="bf16x3"))
    assert np.array_equal(C, (A.astype(np.float64) @ B.astype(np.float64)))


@pytest.mark.parametrize("m,n,w,adjoint", [(4096, 20000, 224, False), (120000, 4096, 224, True)])
def test_bf16x3_long_accumulation_has_no_drift(m, n, w, adjoint):
    """All-positive operands make any one-signed accumulation error visible: the
    split-BF16 products over long K must stay unbiased against FP64 (the tensor
    cores' FP32 accumulation drifts toward zero on long chains)."""
    torch = cuda()
    import paper_1412_3510_gb300 as rp
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    A = torch.rand(m, n, device="cuda", generator=g)
    B = torch.rand(m if adjoint else n, w, device="cuda", generator=g)
    C = rp.rpca_dense_pass(A, B, adjoint=adjoint, precision="bf16x3")
    rows = torch.arange(0, C.shape[0], C.shape[0] // 16, device="cuda")[:16]
    ref = (A[:, rows].double().T if adjoint else A[rows].double()) @ B.double()
    rel = ((C[rows].double() - ref) / ref).cpu().numpy()
    assert abs(rel.mean()) < 3e-5, rel.mean()
    assert np.abs(rel).max() < 1e-4, np.abs(rel).max()
