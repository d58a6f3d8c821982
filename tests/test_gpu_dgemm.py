"""FP64-accurate batched products (the mixed path's refinement engine) against
an extended-precision reference.  Tensor-core Ozaki engine: the 48-bit
rounding of every row of op(A) and column of B bounds the error by
2^-48 (max_k|A_ik| sum_k|B_kj| + sum_k|A_ik| max_k|B_kj|) (2^-46 tested); FP64
engine: n 2^-52 (|A| |B|)_ij."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_00454_gb300 import api, build
    build.build()
    c = api.Context(0)
    yield c
    c.close()


def _mats(n, items, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((items, n, n)) * 10.0 ** rng.uniform(-8, 8, (items, n, 1))  # rows over 16 decades
    B = rng.standard_normal((items, n, n)) * 10.0 ** rng.uniform(-8, 8, (items, 1, n))  # columns likewise
    A[0, 1, :] = 0.0  # an all-zero row
    return A, B


@pytest.mark.parametrize("n", [8, 40, 57, 100, 200, 300])
@pytest.mark.parametrize("trans_a", [False, True])
def test_batched_dgemm_engines(ctx, n, trans_a):
    import torch
    from paper_2106_00454_gb300 import api
    A, B = _mats(n, 3, n + (7 if trans_a else 0))
    opA = np.swapaxes(A, 1, 2) if trans_a else A
    ref = np.matmul(opA.astype(np.longdouble), B.astype(np.longdouble))
    absAB = np.matmul(np.abs(opA), np.abs(B))
    aA, aB = np.abs(opA), np.abs(B)
    scaled = (aA.max(axis=2, keepdims=True) * aB.sum(axis=1, keepdims=True)
              + aA.sum(axis=2, keepdims=True) * aB.max(axis=1, keepdims=True))
    dA = torch.tensor(A, device="cuda:0")
    dB = torch.tensor(B, device="cuda:0")
    for engine, tol, bound in [(api.REFINE_TENSOR, 2.0 ** -46, scaled), (api.REFINE_FP64, n * 2.0 ** -52, absAB)]:
        dC = torch.full_like(dA, float("nan"))
        ctx.batched_dgemm(dA, dB, dC, trans_a=trans_a, engine=engine)
        ctx.sync()
        C = dC.cpu().numpy()
        err = np.abs(C.astype(np.longdouble) - ref)
        assert np.all(np.isfinite(C))
        assert np.all(err <= tol * bound + 1e-300), (engine, float(np.max(err / (bound + 1e-300))))


@pytest.mark.parametrize("n", [800, 1024])
def test_batched_dgemm_long_contraction(ctx, n):
    # five and seven 160-k blocks per tile (the int64 sums at the largest size),
    # and the column split for Kp beyond a shared-memory block
    import torch
    from paper_2106_00454_gb300 import api
    A, B = _mats(n, 1, 11)
    ref = np.matmul(A.astype(np.longdouble), B.astype(np.longdouble))
    aA, aB = np.abs(A), np.abs(B)
    scaled = (aA.max(axis=2, keepdims=True) * aB.sum(axis=1, keepdims=True)
              + aA.sum(axis=2, keepdims=True) * aB.max(axis=1, keepdims=True))
    dA = torch.tensor(A, device="cuda:0")
    dB = torch.tensor(B, device="cuda:0")
    dC = torch.full_like(dA, float("nan"))
    ctx.batched_dgemm(dA, dB, dC, engine=api.REFINE_TENSOR)
    ctx.sync()
    err = np.abs(dC.cpu().numpy().astype(np.longdouble) - ref)
    assert np.all(err <= 2.0 ** -46 * scaled + 1e-300)


def test_batched_dgemm_extreme_scales(ctx):
    """Tiles whose results leave the normal FP64 range: rows scaled by 2^-530 times
    columns scaled by 2^-530 give subnormal products, 2^530 times 2^530 overflow to
    infinity; within the same 32-row groups other rows stay normal (the exact
    out-of-range conversion then covers the whole group)."""
    import torch
    from paper_2106_00454_gb300 import api
    n = 100
    rng = np.random.default_rng(5)
    A = rng.standard_normal((2, n, n))
    B = rng.standard_normal((2, n, n))
    A[0, :20] *= 2.0 ** -530
    B[0, :, :50] *= 2.0 ** -530
    A[1, :20] *= 2.0 ** 530
    B[1, :, :50] *= 2.0 ** 530
    ref = np.matmul(A.astype(np.longdouble), B.astype(np.longdouble))
    aA, aB = np.abs(A), np.abs(B)
    with np.errstate(over="ignore"):  # the bound overflows where the products do
        scaled = (aA.max(axis=2, keepdims=True) * aB.sum(axis=1, keepdims=True)
                  + aA.sum(axis=2, keepdims=True) * aB.max(axis=1, keepdims=True))
    dA = torch.tensor(A, device="cuda:0")
    dB = torch.tensor(B, device="cuda:0")
    dC = torch.full_like(dA, float("nan"))
    ctx.batched_dgemm(dA, dB, dC, engine=api.REFINE_TENSOR)
    ctx.sync()
    C = dC.cpu().numpy()
    big = np.abs(ref) >= np.longdouble(2.0) ** 1024
    assert big[1, :20, :50].all() and not big[0].any()
    assert np.all(np.isinf(C[big])) and np.all(np.sign(C[big]) == np.sign(ref[big]))
    fin = ~big
    assert np.all(np.isfinite(C[fin]))
    err = np.abs(C[fin].astype(np.longdouble) - ref[fin])
    tiny = np.abs(ref[fin]) < np.longdouble(2.0) ** -1022
    assert tiny.sum() > 0  # subnormal results are present
    assert np.all(err <= 2.0 ** -46 * scaled[fin] + 2.0 ** -1073)
