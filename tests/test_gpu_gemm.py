"""The tcgen05 BF16 GEMM against an FP64 product of the same BF16 operands."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_2501_14030_gb300 import nrr

pytestmark = pytest.mark.gpu


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 to the nearest BF16 (ties to even); returns float32."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return (u.astype(np.uint32) << 16).view(np.float32)


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (128, 128, 128),
                                   (256, 512, 512), (384, 192, 320),
                                   (256, 16384, 512), (512, 64, 256)])
def test_gemm_matches_fp64_product(gpu, M, N, K):
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = bf16_round(rng.standard_normal((M, K)).astype(np.float32))
    B = bf16_round(rng.standard_normal((N, K)).astype(np.float32))
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    Ad = torch.from_numpy(A).cuda().to(torch.bfloat16)
    Bd = torch.from_numpy(B).cuda().to(torch.bfloat16)
    D = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    nrr.gemm_bf16_tn(Ad, Bd, D)
    torch.cuda.synchronize()
    out = D.cpu().numpy().astype(np.float64)
    # FP32 accumulation of K exact BF16 products: |err| <= K eps32 sum|a b|
    bound = K * 6e-8 * (np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T)
    assert np.all(np.isfinite(out))
    assert np.all(np.abs(out - ref) <= bound + 1e-30)


def test_gemm_rejects_bad_shapes(gpu):
    A = torch.zeros((100, 64), dtype=torch.bfloat16, device="cuda")
    B = torch.zeros((64, 64), dtype=torch.bfloat16, device="cuda")
    D = torch.zeros((100, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(nrr.NrrError) as e:
        nrr.gemm_bf16_tn(A, B, D)
    assert e.value.status == nrr.ERR_INVALID_ARG


def _operands(M, N, K, seed):
    rng = np.random.default_rng(seed)
    A = bf16_round(rng.standard_normal((M, K)).astype(np.float32))
    B = bf16_round(rng.standard_normal((N, K)).astype(np.float32))
    return A, B


@pytest.mark.parametrize("M,N,K,bn,splits", [
    (256, 512, 16384, 128, 0),    # the input gradient of a 16384-wide layer
    (256, 512, 16384, 128, 19),
    (256, 512, 4096, 64, 5),      # k-block ranges of unequal length
    (128, 256, 512, 256, 1),
    (256, 16384, 512, 256, 1),
    (384, 768, 1024, 256, 3),
    (128, 128, 512, 128, 8),      # one k-block per split
])
def test_gemm_tiles_and_splits_match_fp64_product(gpu, M, N, K, bn, splits):
    A, B = _operands(M, N, K, M + N + K + bn + splits)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    Ad = torch.from_numpy(A).cuda().to(torch.bfloat16)
    Bd = torch.from_numpy(B).cuda().to(torch.bfloat16)
    D = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    nrr.gemm_bf16_tn_async(Ad, Bd, D, bn=bn, splits=splits, persistent=0)
    nrr.gemm_status()
    out = D.cpu().numpy().astype(np.float64)
    # each split and the final sum add FP32 roundings: still within K eps32
    bound = K * 6e-8 * (np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T)
    assert np.all(np.isfinite(out))
    assert np.all(np.abs(out - ref) <= bound + 1e-30)


def test_gemm_split_k_is_deterministic(gpu):
    """The split partial sums are added in a fixed order: repeated calls give
    identical bits."""
    M, N, K = 256, 512, 8192
    A, B = _operands(M, N, K, 5)
    Ad = torch.from_numpy(A).cuda().to(torch.bfloat16)
    Bd = torch.from_numpy(B).cuda().to(torch.bfloat16)
    outs = []
    for _ in range(3):
        D = torch.empty((M, N), dtype=torch.float32, device="cuda")
        nrr.gemm_bf16_tn_async(Ad, Bd, D, bn=128, splits=16)
        outs.append(D)
    nrr.gemm_status()
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])


def test_gemm_async_calls_need_one_status_check(gpu):
    """Many enqueued products, one read-back of the error flag at the end."""
    M, N, K = 256, 1024, 512
    A, B = _operands(M, N, K, 9)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    Ad = torch.from_numpy(A).cuda().to(torch.bfloat16)
    Bd = torch.from_numpy(B).cuda().to(torch.bfloat16)
    Ds = [torch.empty((M, N), dtype=torch.float32, device="cuda") for _ in range(8)]
    for i, D in enumerate(Ds):
        nrr.gemm_bf16_tn_async(Ad, Bd, D, bn=(64, 128, 256)[i % 3])
    nrr.gemm_status()
    bound = K * 6e-8 * (np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T)
    for D in Ds:
        assert np.all(np.abs(D.cpu().numpy().astype(np.float64) - ref) <= bound)


@pytest.mark.parametrize("M,N,K,bn", [
    (2048, 4096, 512, 256),   # 256 tiles: some CTAs take two
    (4096, 4096, 256, 256),   # 512 tiles: both accumulators reused
    (4096, 2048, 512, 128),
    (1024, 1024, 1024, 64),   # fewer tiles than SMs: one each
    (384, 192, 320, 64),
])
def test_persistent_gemm_matches_fp64_product(gpu, M, N, K, bn):
    A, B = _operands(M, N, K, M + 3 * N + K + bn)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    Ad = torch.from_numpy(A).cuda().to(torch.bfloat16)
    Bd = torch.from_numpy(B).cuda().to(torch.bfloat16)
    D = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    nrr.gemm_bf16_tn_async(Ad, Bd, D, bn=bn, splits=1, persistent=1)
    nrr.gemm_status()
    out = D.cpu().numpy().astype(np.float64)
    bound = K * 6e-8 * (np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T)
    assert np.all(np.isfinite(out))
    assert np.all(np.abs(out - ref) <= bound + 1e-30)


@pytest.mark.parametrize("bn", [64, 128, 256])
def test_persistent_gemm_equals_one_cta_per_tile_bitwise(gpu, bn):
    """The persistent kernel, alone or in 2-CTA clusters that share B by
    multicast, issues the same MMAs over K in the same order into an FP32
    accumulator as one CTA per tile: identical bits, whatever the
    tile-to-CTA assignment."""
    M, N, K = 2048, 2048, 512
    A, B = _operands(M, N, K, 77 + bn)
    Ad = torch.from_numpy(A).cuda().to(torch.bfloat16)
    Bd = torch.from_numpy(B).cuda().to(torch.bfloat16)
    Ds = [torch.empty((M, N), dtype=torch.float32, device="cuda") for _ in range(3)]
    for D, pers in zip(Ds, (0, 1, 2)):
        nrr.gemm_bf16_tn_async(Ad, Bd, D, bn=bn, splits=1, persistent=pers)
    nrr.gemm_status()
    assert torch.equal(Ds[1], Ds[0])
    assert torch.equal(Ds[2], Ds[0])


@pytest.mark.parametrize("M,N,K,bn", [
    (4096, 4096, 256, 256),   # 1024 tile pairs over 76 clusters
    (768, 512, 1024, 128),    # fewer pairs than clusters
    (8192, 16384, 512, 256),  # the large shape of the rate table
])
def test_cluster_gemm_matches_fp64_product(gpu, M, N, K, bn):
    A, B = _operands(M, N, K, M + N + K + 2 * bn)
    Ad = torch.from_numpy(A).cuda().to(torch.bfloat16)
    Bd = torch.from_numpy(B).cuda().to(torch.bfloat16)
    D = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    nrr.gemm_bf16_tn_async(Ad, Bd, D, bn=bn, splits=1, persistent=2)
    nrr.gemm_status()
    rows = np.random.default_rng(3).choice(M, size=min(M, 512), replace=False)
    ref = A[rows].astype(np.float64) @ B.astype(np.float64).T
    bound = K * 6e-8 * (np.abs(A[rows]).astype(np.float64) @ np.abs(B).astype(np.float64).T)
    out = D.cpu().numpy()[rows].astype(np.float64)
    assert np.all(np.isfinite(D.cpu().numpy()))
    assert np.all(np.abs(out - ref) <= bound + 1e-30)
