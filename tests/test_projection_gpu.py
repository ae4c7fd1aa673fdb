"""Parity of trbl_block_dot (C = B^T W, the block projection of Alg. 3/4 and
of the reorthogonalisation, Sec. III C/D) with numpy in FP64.

Tolerance: |C - B^T W|_ij <= rtol * (|B|^T |W|)_ij with rtol = 1e-12 for
FP64 data and 1e-5 for FP32 data (FP32 products summed in FP32 inside row
chunks, chunk sums in FP64)."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
trbl = pytest.importorskip("paper_1902_02064_gb300")

pytestmark = pytest.mark.gpu
RTOL = {torch.float64: 1e-12, torch.float32: 1e-5}


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("D,m,q", [(1, 1, 1), (1000, 7, 3), (33333, 130, 32), (200001, 300, 16), (5000, 64, 64)])
def test_block_dot_matches_numpy(dtype, D, m, q):
    B = synth.random_block(D, m, 11)
    W = synth.random_block(D, q, 12)
    Bt = torch.from_numpy(B).to(dtype)
    Wt = torch.from_numpy(W).to(dtype)
    C = trbl.block_dot(Bt.cuda(), Wt.cuda()).cpu().numpy()
    Bd, Wd = Bt.double().numpy(), Wt.double().numpy()
    ref = Bd.T @ Wd
    bound = np.abs(Bd).T @ np.abs(Wd)
    assert np.all(np.abs(C - ref) <= RTOL[dtype] * bound + 1e-300)


def test_block_dot_strided_and_errors():
    D, m, q = 4097, 40, 8
    big = torch.from_numpy(synth.random_block(D, 64, 3)).cuda()
    B = big[:, 5:5 + m]
    W = big[:, 50:50 + q]
    C = trbl.block_dot(B, W)
    ref = B.cpu().numpy().T @ W.cpu().numpy()
    assert np.allclose(C.cpu().numpy(), ref, rtol=0, atol=1e-11)
    with pytest.raises(trbl.TrblError):
        trbl.trbl_block_dot(B.data_ptr(), 64, m, W.data_ptr(), 64, 65, D, trbl.TRBL_F64, C.data_ptr(), 0)
    host = np.zeros((D, q))
    with pytest.raises(trbl.TrblError):
        trbl.trbl_block_dot(B.data_ptr(), 64, m, host.ctypes.data, q, q, D, trbl.TRBL_F64, C.data_ptr(), 0)


@pytest.mark.parametrize("D,m,q", [(1, 1, 1), (100003, 1024, 1), (70001, 300, 2), (5000, 17, 3), (33333, 600, 4)])
def test_narrow_fp64_dot_and_update(D, m, q):
    """FP64 projections with q (resp. n) <= 4 columns -- the one-vector
    Lanczos arm and the column-wise QR -- through the narrow kernels, against
    numpy: C = B^T W and Out = alpha B U + beta Out."""
    B = torch.from_numpy(synth.random_block(D, m, 61)).cuda()
    W = torch.from_numpy(synth.random_block(D, q, 62)).cuda()
    C = trbl.block_dot(B, W).cpu().numpy()
    Bh, Wh = B.cpu().numpy(), W.cpu().numpy()
    ref = Bh.T @ Wh
    assert np.all(np.abs(C - ref) <= 1e-12 * (np.abs(Bh).T @ np.abs(Wh)) + 1e-300)
    U = synth.random_block(m, q, 63)
    O0 = synth.random_block(D, q, 64)
    Out = torch.from_numpy(O0.copy()).cuda()
    trbl.block_update(B, torch.from_numpy(U).cuda(), Out, -1.0, 0.5)
    ref = -(Bh @ U) + 0.5 * O0
    bound = np.abs(Bh) @ np.abs(U) + 0.5 * np.abs(O0)
    assert np.all(np.abs(Out.cpu().numpy() - ref) <= 1e-12 * bound + 1e-300)


@pytest.mark.parametrize("q", [8, 16, 32, 64])
@pytest.mark.parametrize("D,ld", [(1, 0), (127, 0), (100003, 0), (33333, 5), (300000, 1)])
def test_gram_kernel_matches_numpy(q, D, ld):
    """The Gram matrix W^T W of FP32 data (the block Cholesky QR's input)
    through the dedicated kernel: contiguous blocks, blocks inside a wider
    array (leading dimension q + ld, unaligned rows when q + ld is not a
    multiple of 4), ragged row counts; symmetric to the last bit because
    (i, j) and (j, i) see the same products in the same order."""
    full = torch.from_numpy(synth.random_block(D, q + ld, 40 + q)).float().cuda()
    W = full[:, :q]
    G = trbl.block_dot(W, W).cpu().numpy()
    Wd = W.double().cpu().numpy()
    ref = Wd.T @ Wd
    bound = np.abs(Wd).T @ np.abs(Wd)
    assert np.all(np.abs(G - ref) <= 4e-6 * bound + 1e-300)
    assert np.array_equal(G, G.T)
    G2 = trbl.block_dot(W, W).cpu().numpy()
    assert np.array_equal(G, G2)
