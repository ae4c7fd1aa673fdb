"""The allocation-free projection entry point trbl_block_dot_noalloc.

It serves callers that must not allocate device memory during the call (see
include/trbl.h).  Its scratch is a fixed device array compiled into the
library, so this file runs last: if it fails, every other test has already
run.  Each case calls the new entry point through the C ABI twice in a row,
on different inputs, and checks both results against an FP64 product on
the host (numpy) and against the allocating entry point trbl_block_dot,
within the projection tests' tolerance (rounding bounded by
rtol * |B|^T |W|).  One case nearly fills the scratch, so only one row
chunk fits and the whole sum runs through a single chunk."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
trbl = pytest.importorskip("paper_1902_02064_gb300")

pytestmark = pytest.mark.gpu
RTOL = {torch.float64: 1e-12, torch.float32: 1e-5}


def _call_noalloc(B, W):
    C = torch.full((B.shape[1], W.shape[1]), float("nan"), dtype=torch.float64, device="cuda")
    dt = trbl.TRBL_F64 if B.dtype == torch.float64 else trbl.TRBL_F32
    trbl.trbl_block_dot_noalloc(B.data_ptr(), B.stride(0), B.shape[1], W.data_ptr(), W.stride(0), W.shape[1],
                                B.shape[0], dt, C.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return C


def _host_fp64(B, W):
    """C = B^T W in FP64 on the host, and the rounding scale |B|^T |W|."""
    Bh = B.cpu().double().numpy()
    Wh = W.cpu().double().numpy()
    return Bh.T @ Wh, np.abs(Bh).T @ np.abs(Wh)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_noalloc_matches_fp64_host_product_twice(dtype):
    # (D, m, q): many row chunks; a ragged small case; m * q * 8 bytes close
    # to the 8 MiB scratch (one row chunk fits)
    cases = ((1, (120001, 300, 32)), (2, (777, 9, 5)), (3, (301, 16000, 64)))
    assert 16000 * 64 * 8 <= trbl.TRBL_NOALLOC_SCRATCH_BYTES < 2 * 16000 * 64 * 8
    for seed, (D, m, q) in cases:
        B = torch.from_numpy(synth.random_block(D, m, 40 + seed)).to(dtype).cuda()
        W = torch.from_numpy(synth.random_block(D, q, 50 + seed)).to(dtype).cuda()
        C = _call_noalloc(B, W)
        C_ref = trbl.block_dot(B, W)
        torch.cuda.synchronize()
        exact, bound = _host_fp64(B, W)
        Ch = C.cpu().numpy()
        assert np.isfinite(Ch).all()
        assert np.all(np.abs(Ch - exact) <= RTOL[dtype] * bound + 1e-300), (D, m, q)
        assert torch.all((C - C_ref).abs() <= 2 * RTOL[dtype] * torch.from_numpy(bound).cuda() + 1e-300)


def test_noalloc_rejects_oversized_products():
    D, m, q = 64, 20000, 64  # m * q * 8 bytes exceeds the fixed scratch
    B = torch.zeros((D, m), dtype=torch.float32, device="cuda")
    W = torch.zeros((D, q), dtype=torch.float32, device="cuda")
    C = torch.zeros((m, q), dtype=torch.float64, device="cuda")
    with pytest.raises(trbl.TrblError) as e:
        trbl.trbl_block_dot_noalloc(B.data_ptr(), m, m, W.data_ptr(), q, q, D, trbl.TRBL_F32, C.data_ptr(), 0)
    assert e.value.code == trbl.TRBL_ERR_ARG and "scratch" in str(e.value)
