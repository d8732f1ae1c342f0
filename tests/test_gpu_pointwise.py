"""GPU parity of the pointwise products (zx_pointwise) with the oracle's product mod 2^N + 1.

Both methods -- the schoolbook warp kernel (method 1) and the second Schoenhage-Strassen level
on the transform kernels (method 2) -- must give the oracle's canonical residue bit for bit, on
structured residues (0, 1, 2^N, 2^N - 1, powers of two, long runs of ones and zeros) and uniform
ones, on every ring size the recursion plans for; squaring (a == b) included. A large batch
compares the two methods with each other and samples the oracle.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

RINGS = [2048, 4096, 8192, 12288, 16384, 20480, 32768]


@pytest.fixture(scope="module")
def tg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0810_3203_gb300 as m
    m.load()
    return m


def stride_of(N):
    W = N // 64 + 1
    return W + (W & 1)


def operands(N, n, seed):
    """n cells: structured residues first, then uniform ones."""
    s = stride_of(N)
    k = n // 2
    x = np.zeros((n, s), np.uint64)
    x[:k] = workloads.structured_residues(seed, k, N, stride=s).reshape(k, s)
    x[k:] = workloads.residues(seed + 1, n - k, N, stride=s).reshape(n - k, s)
    return x.reshape(-1)


def run(tg, a, b, n, N, method, square=False):
    s = stride_of(N)
    A = torch.from_numpy(a.view(np.int64).copy()).cuda()
    B = A if square else torch.from_numpy(b.view(np.int64).copy()).cuda()
    tg.pointwise(A, B, n, N, s, method)
    torch.cuda.synchronize()
    return A.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("N", RINGS)
@pytest.mark.parametrize("method", [1, 2])
def test_pointwise_matches_oracle(tg, orc, N, method):
    n, s = 48, stride_of(N)
    a, b = operands(N, n, 100 + N // 1024), operands(N, n, 200 + N // 1024)
    # shuffle b so that every structured shape meets every other kind
    b = b.reshape(n, s)[np.random.default_rng(N).permutation(n)].reshape(-1)
    got = run(tg, a, b, n, N, method)
    A, B, G = (orc.cells_to_ints(v, N, n, s) for v in (a, b, got))
    for i in range(n):
        assert G[i] == orc.ring_mul(A[i], B[i], N), (N, method, i)


@pytest.mark.parametrize("N", [4096, 32768])
def test_squaring_in_place(tg, orc, N):
    n, s = 32, stride_of(N)
    a = operands(N, n, 300)
    got = run(tg, a, None, n, N, 2, square=True)
    A, G = orc.cells_to_ints(a, N, n, s), orc.cells_to_ints(got, N, n, s)
    for i in range(n):
        assert G[i] == orc.ring_mul(A[i], A[i], N), i


@pytest.mark.parametrize("N,n", [(32768, 3000), (8192, 20000)])
def test_methods_agree_at_size(tg, orc, N, n):
    s = stride_of(N)
    a = workloads.residues(11, n, N, stride=s)
    b = workloads.residues(12, n, N, stride=s)
    r1 = run(tg, a, b, n, N, 1)
    r2 = run(tg, a, b, n, N, 2)
    assert np.array_equal(r1, r2)
    for i in (0, 1, n // 2, n - 1):
        A, B = orc.cells_to_ints(a[i * s:(i + 1) * s], N, 1, s)[0], orc.cells_to_ints(b[i * s:(i + 1) * s], N, 1, s)[0]
        assert orc.cells_to_ints(r2[i * s:(i + 1) * s], N, 1, s)[0] == orc.ring_mul(A, B, N), i


def test_empty_and_errors(tg):
    x = torch.zeros(stride_of(4096) * 2, dtype=torch.int64, device="cuda")
    tg.pointwise(x, x, 0, 4096, stride_of(4096), 2)
    with pytest.raises(tg.TftError) as ei:
        tg.pointwise(x, x, 1, 4096, 10, 1)
    assert ei.value.code == tg.ZX_EINVAL
    with pytest.raises(tg.TftError) as ei:
        tg.pointwise(x, x, 1, 4096, stride_of(4096), 3)
    assert ei.value.code == tg.ZX_EINVAL
