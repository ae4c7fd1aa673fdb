"""Parity of the tensor-core (tcgen05, split-TF32) block projections with
numpy in FP64: C = B^T W (trbl_block_dot_tc; the coefficients
"alpha_k := V_k^T W" and those of the reorthogonalisation, Sec. III C/D) and
the update Out = alpha In U + beta Out (trbl_block_update; "W -= V C" and
W R^-1), and the mixed-precision solver on both projection paths.

Tolerance: each product a b is formed from TF32 parts with relative error
below 2^-21, and tensor-core FP32 sums run over at most 128 rows
(projection; compensated FP32, then FP64, beyond) or the K columns
(update); for random data the realised
error is far inside |err| <= 1e-5 * (|B|^T |W|) (resp. |In| |U| + |beta Out|),
the bound the CUDA-core FP32 kernels are held to."""
import json
import os

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
trbl = pytest.importorskip("paper_1902_02064_gb300")

pytestmark = pytest.mark.gpu
RTOL = 1e-5
HERE = os.path.dirname(__file__)


def _f32(a):
    return torch.from_numpy(np.ascontiguousarray(a)).float()


def _dev_ld4(t):
    """CUDA copy of a 2-D tensor whose rows start 16-byte aligned (leading
    dimension rounded up to a multiple of 4), as the tensor-core path needs."""
    n = t.shape[1]
    buf = torch.zeros((t.shape[0], (n + 3) // 4 * 4), dtype=t.dtype, device="cuda")
    buf[:, :n] = t.cuda()
    return buf[:, :n]


@pytest.mark.parametrize("D,m,q", [(1, 1, 1), (1000, 7, 3), (4097, 128, 32), (33333, 130, 32),
                                   (200001, 300, 16), (262147, 1024, 32), (70001, 33, 8)])
def test_block_dot_tc_matches_numpy(D, m, q):
    B = _f32(synth.random_block(D, m, 21))
    W = _f32(synth.random_block(D, q, 22))
    C = trbl.block_dot(_dev_ld4(B), _dev_ld4(W), tensor_cores=True).cpu().numpy()
    Bd, Wd = B.double().numpy(), W.double().numpy()
    ref = Bd.T @ Wd
    bound = np.abs(Bd).T @ np.abs(Wd)
    err = np.abs(C - ref)
    assert np.all(err <= RTOL * bound + 1e-300), float((err / bound).max())
    # and against the CUDA-core path
    Ccc = trbl.block_dot(B.cuda(), W.cuda()).cpu().numpy()
    assert np.all(np.abs(C - Ccc) <= 2 * RTOL * bound + 1e-300)


def test_block_dot_tc_strided_view_and_gram():
    D = 50003
    big = _f32(synth.random_block(D, 96, 5)).cuda()
    B = big[:, 4:4 + 64]   # 16-byte aligned start, ld 96
    W = big[:, 64:64 + 32]
    C = trbl.block_dot(B, W, tensor_cores=True).cpu().numpy()
    ref = B.double().cpu().numpy().T @ W.double().cpu().numpy()
    bound = np.abs(B.double().cpu().numpy()).T @ np.abs(W.double().cpu().numpy())
    assert np.all(np.abs(C - ref) <= RTOL * bound)
    G = trbl.block_dot(W, W, tensor_cores=True).cpu().numpy()   # Gram matrix of the block QR
    assert np.allclose(G, G.T, rtol=0, atol=1e-6 * np.abs(G).max())


@pytest.mark.parametrize("tensor_cores", [True, False])
def test_gram_diagonal_is_unbiased(tensor_cores):
    """Diagonal of the Gram matrix W^T W (the block QR's column norms) over
    a million rows: the relative errors of its 32 entries, all of one sign
    if the FP32 sums are biased, must average below 1e-6 and stay below
    3e-6.  The tensor cores' FP32 accumulation rounds toward zero, so long
    accumulations inside tensor memory shrink every positive sum; the
    projection drains its accumulators often enough to keep that below
    FP32 rounding noise (a 2,048-row segment gave -1.6e-5)."""
    D = 1 << 20
    W = _f32(synth.random_block(D, 32, 41))
    Wd = W.double().numpy()
    ref = np.einsum("ij,ij->j", Wd, Wd)
    G = trbl.block_dot(_dev_ld4(W), _dev_ld4(W), tensor_cores=tensor_cores).cpu().numpy()
    rel = np.diag(G) / ref - 1.0
    assert abs(rel.mean()) <= 1e-6, rel.mean()
    assert np.abs(rel).max() <= 3e-6, np.abs(rel).max()


def test_tensor_core_paths_propagate_nan():
    """A NaN with the all-ones payload that CUDA's arithmetic produces, placed
    in W, makes exactly its column of C = B^T W NaN; placed in In, exactly
    its row of the update.  (Rounding to TF32 by adding half a unit to the
    bit pattern carries such a payload into the sign bit and turns the NaN
    into -0, which would hide it.)"""
    nan = torch.tensor([0x7FFFFFFF], dtype=torch.int32).view(torch.float32)[0]
    D = 4097
    B = _f32(synth.random_block(D, 64, 51))
    W = _f32(synth.random_block(D, 32, 52))
    W[100, 5] = nan
    C = trbl.block_dot(_dev_ld4(B), _dev_ld4(W), tensor_cores=True).cpu().numpy()
    assert np.all(np.isnan(C[:, 5])) and np.all(np.isfinite(np.delete(C, 5, axis=1)))
    In = _f32(synth.random_block(D, 300, 53))
    In[7, 3] = nan
    U = synth.random_block(300, 16, 54)
    Out = trbl.block_update(_dev_ld4(In), torch.from_numpy(U), torch.zeros((D, 16), device="cuda"), 1.0, 0.0,
                            algo=trbl.TRBL_PROJ_TENSOR).cpu().numpy()
    assert np.all(np.isnan(Out[7])) and np.all(np.isfinite(np.delete(Out, 7, axis=0)))


def test_block_dot_tc_rejects_unsupported_shapes():
    B = torch.zeros((100, 8), device="cuda")
    W = torch.zeros((100, 40), device="cuda")
    with pytest.raises(trbl.TrblError) as e:
        trbl.block_dot(B, W, tensor_cores=True)
    assert e.value.code == trbl.TRBL_ERR_ARG
    Wb = torch.zeros((100, 9), device="cuda")[:, 1:9]   # 4-byte offset: not 16-byte aligned
    with pytest.raises(trbl.TrblError) as e:
        trbl.block_dot(B, Wb, tensor_cores=True)
    assert e.value.code == trbl.TRBL_ERR_ARG


@pytest.mark.parametrize("algo", [0, 1])
@pytest.mark.parametrize("D,K,n,alpha,beta", [(1, 1, 1, 1.0, 0.0), (1000, 7, 5, -1.0, 1.0),
                                              (33333, 32, 32, 1.0, 0.0), (200001, 100, 16, -1.0, 1.0),
                                              (65537, 640, 32, -1.0, 1.0), (4099, 300, 1, 0.5, -2.0)])
def test_block_update_matches_numpy(algo, D, K, n, alpha, beta):
    In = _f32(synth.random_block(D, K, 31))
    U = synth.random_block(K, n, 32) / np.sqrt(K)
    Out0 = _f32(synth.random_block(D, n, 33))
    Out = trbl.block_update(_dev_ld4(In), torch.from_numpy(U), Out0.clone().cuda(), alpha, beta, algo=algo)
    Ind, O0 = In.double().numpy(), Out0.double().numpy()
    ref = alpha * (Ind @ U) + beta * O0
    bound = abs(alpha) * (np.abs(Ind) @ np.abs(U)) + abs(beta) * np.abs(O0)
    err = np.abs(Out.cpu().double().numpy() - ref)
    assert np.all(err <= RTOL * bound + 1e-30), float((err / (bound + 1e-30)).max())


def test_block_update_strided_input_falls_back_correctly():
    D, K, n = 5001, 40, 8
    big = _f32(synth.random_block(D, 43, 7)).cuda()
    In = big[:, 1:1 + K]   # unaligned for TMA: the CUDA-core path takes it
    U = synth.random_block(K, n, 8)
    Out = trbl.block_update(In, torch.from_numpy(U), torch.zeros((D, n), device="cuda"), 1.0, 0.0)
    ref = In.double().cpu().numpy() @ U
    assert np.allclose(Out.cpu().double().numpy(), ref, rtol=0, atol=1e-5 * np.abs(ref).max())


@pytest.mark.parametrize("projections", [0, 1])
def test_mixed_solver_on_both_projection_paths(projections):
    """The 28,503-dim workload to 1e-6 ||H|| in mixed precision, with the
    projections on the tensor cores and on the CUDA cores."""
    gold = json.load(open(os.path.join(HERE, "golden", "eigs_s12_4p4n.json")))
    w, sa, sb, inter = synth.workload("s12_4p4n")
    tb = trbl.Basis(sa, w.nA, sb, w.nB, w.twoM)
    th = trbl.Hamiltonian.from_interaction(tb, inter)
    normH = gold["normH"]
    ev, rs, X, st = trbl.solve(th, 40, 8, 160, 1e-6, precision=trbl.TRBL_PREC_MIXED, normH=normH,
                               projections=projections)
    ref = np.array(gold["evals"][:40])
    assert np.abs(ev - ref).max() <= 1e-6 * normH
    assert rs.max() <= 1e-4 * normH


@pytest.mark.parametrize("D,K,n,beta", [(1000, 7, 33, 0.0), (33333, 130, 129, 0.0), (70001, 64, 256, 0.5),
                                        (200001, 1024, 631, 0.0), (129, 1024, 500, -1.0)])
def test_wide_update_matches_numpy(D, K, n, beta):
    """The wide tensor-core GEMM (thick restart and Ritz vectors, n > 32)
    against numpy in FP64: ragged row and column tiles, K not a multiple of
    32, the restart's shape (K = 1024, n = 631) and a beta term."""
    In = _f32(synth.random_block(D, K, 31))
    U = synth.random_block(K, n, 32) / np.sqrt(K)
    O0 = _f32(synth.random_block(D, n, 33))
    Out = _dev_ld4(O0)
    trbl.block_update(_dev_ld4(In), torch.from_numpy(U).cuda(), Out, 1.0, beta, algo=trbl.TRBL_PROJ_TENSOR)
    Ind, O0d = In.double().numpy(), O0.double().numpy()
    ref = Ind @ U + beta * O0d
    bound = np.abs(Ind) @ np.abs(U) + abs(beta) * np.abs(O0d)
    err = np.abs(Out.cpu().double().numpy() - ref)
    assert np.all(err <= RTOL * bound), float((err / bound).max())
    # typical error near FP32 rounding, far inside the bound
    assert float(np.median(err / bound)) < 1e-6


def test_wide_update_is_unbiased():
    """Rotating orthonormal columns by an orthogonal matrix keeps unit norms:
    the tensor cores' round-toward-zero accumulation, left unchecked over
    K = 1024, would shrink every norm by about 1e-5; with fresh accumulators
    every 32 values of K the mean deviation stays at FP32 rounding level."""
    D, K, n = 60001, 1024, 200
    Q, _ = np.linalg.qr(synth.random_block(D, K, 41))
    Uo, _ = np.linalg.qr(synth.random_block(K, K, 42))
    In = _dev_ld4(_f32(Q))
    Out = torch.zeros((D, n), dtype=torch.float32, device="cuda")
    trbl.block_update(In, torch.from_numpy(np.ascontiguousarray(Uo[:, :n])).cuda(), Out, 1.0, 0.0,
                      algo=trbl.TRBL_PROJ_TENSOR)
    nrm2 = (Out.double() ** 2).sum(0).cpu().numpy()
    assert abs(float(np.mean(nrm2 - 1.0))) < 5e-7, float(np.mean(nrm2 - 1.0))
    assert float(np.abs(nrm2 - 1.0).max()) < 5e-6
