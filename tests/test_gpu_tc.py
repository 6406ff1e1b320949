"""tcgen05 BF16 GEMM (nsk_gemm_bf16) against an FP64 CPU product of the same BF16 inputs.

The products of two BF16 numbers are exact in FP32, so the only error is the FP32
accumulation: |C - C_ref| <= 2e-5 * (|A| |B|^T) elementwise (about K * 2^-24 relative
to the sum of magnitudes, K <= 256, with margin).
"""
import numpy as np
import pytest

from paper_1912_12059_gb300 import nsk

pytestmark = pytest.mark.gpu


def _bf16(shape, gen, scale=1.0):
    import torch

    return (torch.from_numpy(gen.standard_normal(shape) * scale).to(torch.bfloat16))


def _ref(A, B):
    a = A.double().numpy()
    b = B.double().numpy()
    return a @ b.T, np.abs(a) @ np.abs(b).T


@pytest.mark.parametrize("M,N,K,k_split", [(128, 64, 64, 0), (300, 256, 80, 0), (1000, 80, 256, 64),
                                           (77, 16, 16, 0), (513, 240, 192, 128)])
def test_gemm_store_and_split_k(gpu, M, N, K, k_split):
    import torch

    g = np.random.default_rng(M + N + K)
    A, B = _bf16((M, K), g), _bf16((N, K), g)
    bias = torch.from_numpy(g.standard_normal(N)).float()
    ref, mag = _ref(A, B)
    Ad, Bd = A.to(gpu), B.to(gpu)
    err = torch.zeros(1, dtype=torch.int32, device=gpu)
    if k_split:
        out = torch.zeros((M, N), dtype=torch.float32, device=gpu)
        assert nsk.gemm_bf16(Ad, Bd, epilogue=1, out=out, k_split=k_split, err=err) == 0
        want = ref
    else:
        out = torch.full((M, N), float("nan"), dtype=torch.float32, device=gpu)
        assert nsk.gemm_bf16(Ad, Bd, epilogue=0, bias=bias.to(gpu), out=out, err=err) == 0
        want = ref + bias.double().numpy()[None, :]
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    got = out.cpu().double().numpy()
    assert np.all(np.abs(got - want) <= 2e-5 * mag + 1e-6)


def test_gemm_gelu_and_transpose(gpu):
    import math

    import torch

    g = np.random.default_rng(5)
    M, N, K = 200, 256, 80
    A, B = _bf16((M, K), g, 0.3), _bf16((N, K), g, 0.3)
    bias = torch.from_numpy(g.standard_normal(N) * 0.1).float()
    z = torch.empty((M, N), dtype=torch.float32, device=gpu)
    h = torch.empty((M, N), dtype=torch.bfloat16, device=gpu)
    ht = torch.empty((N, 208), dtype=torch.bfloat16, device=gpu)  # row stride 208 >= M
    assert nsk.gemm_bf16(A.to(gpu), B.to(gpu), epilogue=2, bias=bias.to(gpu), out=z, hout=h, hout_t=ht) == 0
    torch.cuda.synchronize()
    ref, mag = _ref(A, B)
    zr = ref + bias.double().numpy()[None, :]
    assert np.all(np.abs(z.cpu().double().numpy() - zr) <= 2e-5 * mag + 1e-6)
    erf = np.vectorize(math.erf)
    hr = 0.5 * zr * (1 + erf(zr / math.sqrt(2)))
    hb = h.cpu().double().numpy()
    assert np.all(np.abs(hb - hr) <= 2 ** -8 * np.abs(hr) + 1e-4)  # BF16 rounding of the output
    assert np.array_equal(ht[:, :M].cpu().float().numpy().T, h.cpu().float().numpy())


def test_gemm_dgelu_and_bias_grad(gpu):
    import math

    import torch

    g = np.random.default_rng(6)
    M, N, K = 384, 64, 256
    A, B = _bf16((M, K), g, 0.2), _bf16((N, K), g, 0.2)
    zin = torch.from_numpy(g.standard_normal((M, N))).float()
    dz = torch.empty((M, N), dtype=torch.bfloat16, device=gpu)
    dzt = torch.empty((N, M), dtype=torch.bfloat16, device=gpu)
    bg = torch.zeros(N, dtype=torch.float32, device=gpu)
    assert nsk.gemm_bf16(A.to(gpu), B.to(gpu), epilogue=3, hout=dz, hout_t=dzt, zin=zin.to(gpu), bias_grad=bg) == 0
    torch.cuda.synchronize()
    ref, mag = _ref(A, B)
    zz = zin.double().numpy()
    erf = np.vectorize(math.erf)
    gp = 0.5 * (1 + erf(zz / math.sqrt(2))) + zz * np.exp(-0.5 * zz * zz) / math.sqrt(2 * math.pi)
    want = ref * gp
    got = dz.cpu().double().numpy()
    assert np.all(np.abs(got - want) <= 2 ** -8 * np.abs(want) + 3e-5 * mag * np.abs(gp) + 1e-5)
    assert np.array_equal(dzt.cpu().float().numpy().T, dz.cpu().float().numpy())
    assert np.allclose(bg.cpu().double().numpy(), want.sum(axis=0), rtol=1e-3, atol=1e-3)
