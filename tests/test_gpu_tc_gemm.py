"""The tensor-core (tcgen05, split TF32) dense products of the mixed-precision
M~ factorisation, against a plain PyTorch FP64 product, and the factorisation
built on them (M~^-1 applied to M~ x returns x).

Tolerance of a product: each operand is split x = hi + lo into TF32 parts
(|lo| <= 2^-11 |x|) and hi.hi + hi.lo + lo.hi are accumulated in FP32; the
dropped lo.lo term and the FP32 accumulation over K terms bound the error
by about (2^-22 + K 2^-24) sum_k |a_k b_k|: asserted below as 1e-5 of the
largest |A| |B|^T entry (a single TF32 product, 2^-11, would miss it).
"""
import numpy as np
import pytest

from oracle import mobility
from synthetic import Body, Workload, sphere_markers

from ._util import gpu_grid, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abi():
    from paper_1505_07865_gb300 import abi as a

    assert torch.cuda.is_available()
    return a


@pytest.mark.parametrize("M,N,K,lda_pad,alpha,beta", [
    (128, 128, 32, 0, 1.0, 0.0),
    (256, 384, 160, 4, -1.5, 0.5),
    (512, 128, 1024, 8, 1.0, 1.0),
])
def test_tc_gemm_matches_fp64(abi, M, N, K, lda_pad, alpha, beta):
    g = torch.Generator(device="cpu").manual_seed(M + N + K)
    Ab = torch.randn(M, K + lda_pad, generator=g, dtype=torch.float32)
    Bb = torch.randn(N, K + lda_pad, generator=g, dtype=torch.float32)
    C0 = torch.randn(M, N, generator=g, dtype=torch.float32)
    A, B = Ab.cuda(), Bb.cuda()
    C = C0.clone().cuda()
    abi.op_gemm_tf32x3(A[:, :K], B[:, :K], C, alpha=alpha, beta=beta)
    torch.cuda.synchronize()
    ref = beta * C0.double() + alpha * (Ab[:, :K].double() @ Bb[:, :K].double().T)
    scale = (Ab[:, :K].double().abs() @ Bb[:, :K].double().abs().T).max().item() * abs(alpha)
    err = (C.cpu().double() - ref).abs().max().item()
    assert err < 1e-5 * scale, (err, scale)


def test_tc_gemm_rejects_unaligned_sizes(abi):
    A = torch.zeros(100, 32, device="cuda")
    B = torch.zeros(128, 32, device="cuda")
    C = torch.zeros(100, 128, device="cuda")
    with pytest.raises(abi.IbrError) as e:
        abi.op_gemm_tf32x3(A, B, C)
    assert e.value.code == abi.EINVAL


@pytest.mark.parametrize("N,R", [(700, 0.25), (2000, 0.3)])
def test_tc_mobility_inverse_large_block(abi, N, R):
    # one sphere on a 64^3 grid: a dense 3N x 3N M~ (2100 and 6000: ragged and
    # near the largest single block) from the tabulated pair mobility (positive
    # definite, no shift), factorised in split TF32; checked against the FP64
    # block the library built
    rel = sphere_markers(R, N)
    wl = Workload("tc_big", (64, 64, 64), (1.0, 1.0, 1.0),
                  bodies=[Body(np.array([0.5, 0.5, 0.5]), rel, np.zeros(6))], tol=1e-8)
    G = gpu_grid(abi, wl, abi.MIXED)
    try:
        o = abi.solve_opts_default()
        o.mob_model = abi.MOB_PAIR
        abi.prepare(G, o)
        n = 3 * N
        Mt = torch.zeros(n * n, dtype=torch.float64, device="cuda")
        abi.op_mtilde(G, 0, Mt)
        torch.cuda.synchronize()
        M = Mt.cpu().numpy().reshape(n, n)
        x = np.random.default_rng(4).standard_normal(n)
        out = torch.zeros(n, dtype=torch.float64, device="cuda")
        abi.op_mtilde_solve(G, torch.from_numpy(M @ x).cuda(), out)
        torch.cuda.synchronize()
        kappa = np.linalg.cond(M)
        assert rel_err(out.cpu().numpy(), x) < 1e-3 * max(1.0, kappa / 1e3), kappa
    finally:
        abi.destroy_grid(G)
