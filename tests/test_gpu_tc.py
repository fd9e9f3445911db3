"""The tensor-core contraction of the 16-bit accumulate walk (tcgen05 MMA, kind::f16, operands in
128-byte-swizzled K-major shared memory, FP32 accumulator in TMEM): an exact product of small
dyadic numbers through icgs_selftest_tc, in BF16 and FP16, for both MMA widths the walk uses."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def icgs():
    from paper_2604_17155_gb300 import build as B
    B.build()
    from paper_2604_17155_gb300 import icgs as I
    I.load()
    return I


@pytest.mark.parametrize("M", [64, 128])
@pytest.mark.parametrize("N", [32, 80])
@pytest.mark.parametrize("bf16", [True, False])
def test_tc_contraction_exact(icgs, M, N, bf16):
    rng = np.random.default_rng(N + 7 * bf16 + M)
    # multiples of 1/8 in [-2, 2]: exact in 16 bits; every partial sum is exact in FP32
    A = rng.integers(-16, 17, (M, 256)) / 8.0
    B = rng.integers(-16, 17, (N, 256)) / 8.0
    dt = torch.bfloat16 if bf16 else torch.float16
    At = torch.tensor(A, dtype=dt, device="cuda")
    Bt = torch.tensor(B, dtype=dt, device="cuda")
    D = icgs.selftest_tc(At, Bt, bf16=bf16).cpu().numpy()
    ref = A @ B.T
    bad = np.argwhere(D != ref)
    assert bad.size == 0, f"{len(bad)} mismatches, first {bad[:5].tolist()}: {D[tuple(bad[0])]} vs {ref[tuple(bad[0])]}"


@pytest.mark.parametrize("M", [64, 128])
def test_tc_structure_rows_and_columns(icgs, M):
    """One-hot operands: D[m][n] = 1 exactly where A's row m and B's row n pick the same pixel,
    which pins the row/column/pixel mapping independently of the arithmetic."""
    A = np.zeros((M, 256))
    B = np.zeros((80, 256))
    for m in range(M):
        A[m, (m * 37) % 256] = 1.0
    for n in range(80):
        B[n, (n * 37 + (n % 3)) % 256] = 1.0
    D = icgs.selftest_tc(torch.tensor(A, dtype=torch.bfloat16, device="cuda"),
                         torch.tensor(B, dtype=torch.bfloat16, device="cuda"), bf16=True).cpu().numpy()
    np.testing.assert_array_equal(D, A @ B.T)


def test_tc_m64_rows_in_tmem_lanes(icgs):
    """An M = 64 product places row m in TMEM lane (m % 16) + 32 (m // 16): with A's row m picking
    pixel m and B's row 0 holding pixel index + 1, lane L of the raw read-back holds m + 1 in
    column 0 exactly for the lanes that carry a row."""
    A = np.zeros((64, 256))
    A[np.arange(64), np.arange(64)] = 1.0
    B = np.zeros((32, 256))
    B[0] = np.arange(256) + 1.0
    D, lanes = icgs.selftest_tc(torch.tensor(A, dtype=torch.bfloat16, device="cuda"),
                                torch.tensor(B, dtype=torch.bfloat16, device="cuda"), bf16=True, lanes=True)
    col0 = lanes[:, 0].cpu().numpy()
    found = {m: [L for L in range(128) if col0[L] == m + 1] for m in (0, 1, 15, 16, 17, 31, 32, 47, 48, 63)}
    print("row -> lanes holding it", found)
    expected = np.array([(m % 16) + 32 * (m // 16) for m in range(64)])
    np.testing.assert_array_equal(col0[expected], np.arange(64) + 1.0)
    np.testing.assert_array_equal(D.cpu().numpy(), A @ B.T)
