"""The tensor-core head product (tcgen05 + TMA, hand-written for sm_103a)
against a plain PyTorch FP32 matmul of the same 16-bit operands (GPU only).

d = a @ b.T with FP32 accumulation, rounded once to the 16-bit type: each
element is within the unit roundoff of that type (2^-8 relative for BF16,
2^-11 for FP16) of the exact product, plus the summation error of k terms,
charged at 2^-22 per addition (the tensor cores' FP32 accumulation is not
specified as round-to-nearest; the assignment's error bound charges the same).
"""
import numpy as np
import pytest

from paper_2002_09094_gb300 import ivf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


def _check(m, n, k, storage, density=1.0, seed=0, lda_pad=0):
    import torch

    dt = torch.bfloat16 if storage == "bf16" else torch.float16
    g = torch.Generator(device="cuda").manual_seed(seed)
    a_full = torch.randn(m, k + lda_pad, generator=g, device="cuda", dtype=torch.float32)
    if density < 1.0:
        a_full *= (torch.rand(m, k + lda_pad, generator=g, device="cuda") < density).float()
    a_full = a_full.to(dt)
    a = a_full[:, :k]
    b = torch.randn(n, k, generator=g, device="cuda", dtype=torch.float32).to(dt)
    d = torch.full((m, n), float("nan"), device="cuda", dtype=dt)
    ivf.head_product(a, b, d, storage)
    torch.cuda.synchronize()
    ref = a.float() @ b.float().T
    mag = a.float().abs() @ b.float().abs().T
    u16 = 2.0 ** -8 if storage == "bf16" else 2.0 ** -11
    tol = u16 * ref.abs() + (k + 2) * 2.0 ** -22 * mag + 1e-30
    err = (d.float() - ref).abs()
    assert torch.isfinite(d.float()).all()
    bad = (err > tol).sum().item()
    assert bad == 0, (bad, float((err / tol).max()))
    return d, ref


@pytest.mark.parametrize("storage", ["bf16", "f16"])
@pytest.mark.parametrize("m,n,k", [(128, 256, 64), (300, 512, 192), (1000, 1024, 320), (1, 256, 64),
                                   (2047, 768, 1024)])
def test_head_product_matches_fp32_matmul(m, n, k, storage):
    _check(m, n, k, storage, seed=m + n + k)


def test_head_product_sparse_rows_and_padded_leading_dimension():
    """Rows about 2 % dense (like objects' head values) and a row stride
    longer than k (the columns beyond k are never read)."""
    d, ref = _check(777, 512, 256, "bf16", density=0.02, seed=5, lda_pad=64)
    assert (ref == 0).any()


def test_head_product_rejects_unsupported_shapes():
    import torch

    a = torch.zeros(64, 64, device="cuda", dtype=torch.bfloat16)
    b = torch.zeros(100, 64, device="cuda", dtype=torch.bfloat16)   # n not a multiple of 256
    d = torch.zeros(64, 100, device="cuda", dtype=torch.bfloat16)
    with pytest.raises(ivf.IvfError):
        ivf.head_product(a, b, d, "bf16")
    b = torch.zeros(256, 48, device="cuda", dtype=torch.bfloat16)   # k not a multiple of 64
    a = torch.zeros(64, 48, device="cuda", dtype=torch.bfloat16)
    d = torch.zeros(64, 256, device="cuda", dtype=torch.bfloat16)
    with pytest.raises(ivf.IvfError):
        ivf.head_product(a, b, d, "bf16")
