"""The network's tensor-core product (fno_gemm_bf16: tcgen05.mma on BF16
operands staged by TMA, FP32 accumulators in tensor memory) against a plain
PyTorch FP32 product of the same BF16 values.

Shapes cover one and many tiles, ragged M, N and K tails (TMA zero fill,
guarded stores), K shorter than one stage and much longer than the
pipeline, shared and batched operands, transposed output strides and
beta = 1 accumulation, odd and unaligned row pitches, and the network's
own shapes.  The FP32 reference
sums the same exactly representable products in another order, so the
difference is FP32 rounding of sums of K terms."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    yield
    torch.cuda.synchronize()


CASES = [
    # (M, N, K, batch, shared_y, transposed_out, beta)
    (128, 32, 64, 1, False, False, 0.0),
    (128, 64, 16, 1, False, False, 0.0),
    (300, 40, 100, 1, False, False, 0.0),
    (257, 200, 520, 2, False, False, 0.0),
    (1000, 256, 256, 1, False, True, 0.0),
    (640, 300, 72, 3, True, False, 1.0),
    (64, 32, 16384, 4, False, False, 0.0),
    (32768, 32, 256, 1, False, False, 0.0),   # x-transform of a training batch
    (16384, 32, 32, 4, True, True, 1.0),      # channel mixing, written transposed, accumulated
    (4096, 2048, 32, 1, False, False, 1.0),   # inverse x-transform at nx = 2048
    (200, 37, 48, 2, False, False, 1.0),      # N and the row pitch odd
    (130, 74, 40, 1, False, False, 0.0),      # row pitch 74: rows 8-byte aligned only
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[:4])) + ("s" if c[4] else "")
                         + ("t" if c[5] else "") + ("b" if c[6] else ""))
def test_gemm_against_fp32_reference(case):
    import torch
    from paper_1307_6703_gb300.fno import fno_gemm_bf16
    M, N, K, B, shared_y, tout, beta = case
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N * 3 + K)
    ldx = ((K + 7) // 8) * 8 + 8          # padded pitches (multiples of 8)
    ldy = ((K + 7) // 8) * 8
    X = (torch.randn(B, M, ldx, generator=g) * 0.5).to(torch.bfloat16).cuda()
    Y = (torch.randn(1 if shared_y else B, N, ldy, generator=g) * 0.5).to(torch.bfloat16).cuda()
    Xk, Yk = X[:, :, :K].float(), Y[:, :, :K].float()
    ref = torch.matmul(Xk, Yk.transpose(1, 2))  # [B, M, N] in FP32
    C0 = torch.randn(B, M, N, generator=g).cuda()
    if beta:
        ref = ref + beta * C0
    if tout:  # C stored as [B][N][M]
        Cbuf = C0.transpose(1, 2).contiguous()
        cm, cn, sC = 1, M, M * N
    else:
        Cbuf = C0.clone()
        cm, cn, sC = N, 1, M * N
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    fno_gemm_bf16(X, ldx, M * ldx, Y, ldy, 0 if shared_y else N * ldy, Cbuf, cm, cn, sC,
                  M, N, K, B, beta, err)
    torch.cuda.synchronize()
    assert err.item() == 0
    out = Cbuf.transpose(1, 2) if tout else Cbuf
    scale = float(ref.abs().max())
    diff = float((out - ref).abs().max()) / scale
    print(f"{case}: max |diff| / max |ref| = {diff:.2e}")
    assert diff <= 2e-5 * max(1.0, np.sqrt(K / 64.0))


def test_gemm_rejects_bad_arguments():
    import torch
    from paper_1307_6703_gb300 import LBError
    from paper_1307_6703_gb300.fno import fno_gemm_bf16
    X = torch.zeros(64, 64, dtype=torch.bfloat16, device="cuda")
    C = torch.zeros(64, 64, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    for bad in (dict(ldx=60), dict(K=0), dict(ldx=32), dict(M=0)):
        a = dict(ldx=64, K=64, M=64)
        a.update(bad)
        with pytest.raises(LBError):
            fno_gemm_bf16(X, a["ldx"], 0, X, 64, 0, C, 64, 1, 0, a["M"], 64, a["K"], 1, 0.0, err)
