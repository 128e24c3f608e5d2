"""GPU parity of the dense contraction tt_contract in every working precision,
including the tcgen05 tensor-core kernels of the TF32 and BF16 forms.

Plain tensor-core inputs (split = 0) are checked against the exact product of
the inputs rounded the way the kernel's packer rounds them (TF32: round to
nearest, ties away, 10 stored mantissa bits; BF16: round to nearest even, 7
stored bits): any layout, swizzle, descriptor or K-slice error gives O(1)
relative errors, while FP32 accumulation of k products stays below
k * 2^-24 relative to (|A||B|)_ij (asserted at 1e-4, above that worst case
for k <= 1024 and far below any layout error).  Split inputs must reach FP32
accuracy: ||C - AB||_F <= 4e-6 ||(|A||B|)||_F.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPES = [(1024, 112, 3072), (3072, 96, 1024), (1024, 3072, 112), (200, 40, 70), (130, 17, 33),
          (300, 600, 100), (64, 8, 16), (129, 257, 65)]


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03483_gb300 import api as A
    from paper_2408_03483_gb300 import capi
    capi.load()
    return A


def tf32_rna(x):
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x1000) & 0xFFFFE000).astype(np.uint32)
    return b.view(np.float32)


def bf16_rne(x):
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return b.view(np.float32)


def operands(m, n, k, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((m, k)), rng.standard_normal((k, n))


def run(api, A, B, precision, split, alpha=1.0, beta=0.0, C0=None):
    import torch
    Ad = torch.from_numpy(A).cuda()
    Bd = torch.from_numpy(B).cuda()
    C = None
    if C0 is not None:
        C = torch.from_numpy(np.asfortranarray(C0)).cuda()
        C = C.t().contiguous().t()
    out = api.tt_contract(Ad, Bd, precision=precision, split=split, alpha=alpha, beta=beta, C=C)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("m,n,k", SHAPES)
@pytest.mark.parametrize("precision", ["tf32", "bf16"])
def test_tensor_core_plain_inputs_exact_product(api, m, n, k, precision):
    A, B = operands(m, n, k, seed=m + 7 * n + 13 * k)
    C = run(api, A, B, precision, split=False)
    rnd = tf32_rna if precision == "tf32" else bf16_rne
    Ar = rnd(A.astype(np.float32)).astype(np.float64)
    Br = rnd(B.astype(np.float32)).astype(np.float64)
    ref = Ar @ Br
    bound = 1e-4 * (np.abs(Ar) @ np.abs(Br)) + 1e-30
    assert np.all(np.abs(C - ref) <= bound), float(np.max(np.abs(C - ref) / bound))


@pytest.mark.parametrize("m,n,k", SHAPES)
@pytest.mark.parametrize("precision", ["tf32", "bf16", "fp32"])
def test_split_and_fp32_reach_fp32_accuracy(api, m, n, k, precision):
    A, B = operands(m, n, k, seed=1 + m + 3 * n + 5 * k)
    C = run(api, A, B, precision, split=True)
    ref = A @ B
    scale = np.linalg.norm(np.abs(A) @ np.abs(B))
    assert np.linalg.norm(C - ref) <= 4e-6 * scale


@pytest.mark.parametrize("precision", ["fp64", "fp32", "tf32", "bf16"])
def test_alpha_beta_and_leading_dimensions(api, precision):
    import torch
    m, n, k = 300, 70, 200
    A, B = operands(m, n, k, seed=3)
    C0 = np.random.default_rng(4).standard_normal((m, n))
    got = run(api, A, B, precision, split=True, alpha=-1.0, beta=1.0, C0=C0)
    ref = C0 - A @ B
    tol = 1e-12 if precision == "fp64" else 4e-6
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(np.abs(A) @ np.abs(B))
    # operands that are column blocks of larger arrays (lda > m, ldb > k)
    big_a = torch.from_numpy(np.random.default_rng(5).standard_normal((k + 9, m + 11)).T.copy()).cuda()
    big_b = torch.from_numpy(np.random.default_rng(6).standard_normal((n + 3, k + 5)).T.copy()).cuda()
    Ad = torch.as_strided(big_a, (m, k), (1, m + 11))
    Bd = torch.as_strided(big_b, (k, n), (1, k + 5))
    out = api.tt_contract(Ad, Bd, precision=precision, split=True)
    ref = Ad.cpu().numpy() @ Bd.cpu().numpy()
    assert np.linalg.norm(out.cpu().numpy() - ref) <= tol * np.linalg.norm(
        np.abs(Ad.cpu().numpy()) @ np.abs(Bd.cpu().numpy()))
