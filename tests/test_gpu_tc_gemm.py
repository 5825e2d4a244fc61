"""The tensor-core GEMM (twa_tc_gemm: tcgen05 MMAs with TF32 operands, FP32 accumulation in tensor
memory, TMA tile loads) against FP64 products, and the surrogate's DFT contractions that use it.

Bound of one output: the tensor cores read each FP32 operand to TF32 (10 explicit mantissa bits), so
each product a b carries a relative error below about 2 x 2^-10, and the FP32 sums add K x 2^-24
of sum |a b|; |C - A B^T| <= 2.5e-3 (|A| |B|^T) elementwise covers both.  A wrong operand layout,
swizzle or descriptor gives errors of the size of C itself.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2310_07119_gb300 import _lib

TOL = 2.5e-3


def _call(A, P, K, lda, Bt, N, Np, C, ldc, acc, err):
    lib = _lib.load()
    return lib.twa_tc_gemm(A, P, K, lda, Bt, N, Np, C, ldc, acc, err, None)


@pytest.mark.parametrize("P,K,N,Np,acc", [(1000, 32, 16, 16, 0), (4096, 128, 64, 64, 0), (333, 64, 48, 48, 1),
                                          (130, 128, 100, 112, 0), (257, 96, 128, 128, 1), (40000, 128, 192, 192, 0),
                                          (5000, 64, 256, 256, 0)])
@pytest.mark.gpu
def test_tc_gemm_matches_fp64_products(P, K, N, Np, acc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(P + K + N)
    a = rng.normal(size=(P, K)).astype(np.float32)
    b = np.zeros((Np, K), dtype=np.float32)
    b[:N] = rng.normal(size=(N, K))
    c0 = rng.normal(size=(P, N)).astype(np.float32) if acc else np.zeros((P, N), dtype=np.float32)
    A, B, C = (torch.from_numpy(x).cuda() for x in (a, b, c0))
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = _call(A.data_ptr(), P, K, K, B.data_ptr(), N, Np, C.data_ptr(), N, acc, err.data_ptr())
    assert rc == 0, _lib.load().twa_last_error(None)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    got = C.double().cpu().numpy()
    ref = c0.astype(np.float64) + a.astype(np.float64) @ b[:N].astype(np.float64).T
    bound = TOL * (np.abs(a).astype(np.float64) @ np.abs(b[:N]).astype(np.float64).T) + 1e-6 * (np.abs(c0) + 1)
    assert np.all(np.abs(got - ref) <= bound), float(np.max(np.abs(got - ref) / bound))
    # the result really is reduced-precision tensor-core arithmetic, not an FP32 product
    assert np.max(np.abs(got - ref)) > 0


@pytest.mark.parametrize("K,Np,lda,off", [(48, 16, 48, 0), (32, 24, 32, 0), (160, 16, 160, 0), (32, 16, 33, 0),
                                          (32, 16, 32, 4), (128, 208, 128, 0)])
def test_tc_gemm_refuses_unsupported_shapes_before_any_launch(K, Np, lda, off):
    lib = _lib.load()
    # fake device addresses: every check fires before anything touches them
    rc = lib.twa_tc_gemm(4096 + off, 64, K, lda, 8192, min(Np, 16), Np, 16384, 16, 0, 256, None)
    assert rc == _lib.TWA_EINVAL
    assert b"twa_tc_gemm" in lib.twa_last_error(None)


@pytest.mark.gpu
def test_surrogate_on_tensor_cores_matches_the_oracle_and_the_cuda_core_path():
    """grid 32, modes 8: both x-axis contractions of the truncated DFT run on the tensor cores."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import fno as ofno
    from paper_2310_07119_gb300.fno import FNO
    cfg = dict(W=4, c_in=4, c_out=1, modes=8, layers=2)
    n, B = 32, 2
    rng = np.random.default_rng(5)
    theta = rng.normal(scale=0.4, size=ofno.num_params(**cfg))
    x = rng.normal(size=(B, cfg["c_in"], n, n, n)).astype(np.float32)
    m = FNO(n, cfg["W"], cfg["modes"], cfg["layers"], cfg["c_in"], cfg["c_out"])
    lib = _lib.load()
    assert lib.twa_fno_tensor_core_shapes(m.h) == 3
    m.set_params(torch.tensor(theta, dtype=torch.float32))
    xg = torch.from_numpy(x).cuda()
    y_tc = m.forward(xg).double().cpu().numpy()
    assert lib.twa_fno_sync_status(m.h, None) == 0
    assert lib.twa_fno_set_tensor_cores(m.h, 0) == 0
    y_cc = m.forward(xg).double().cpu().numpy()
    th = theta.astype(np.float32).astype(np.float64)
    o = 0
    for name, sh in ofno.param_shapes(**cfg):
        k = int(np.prod(sh))
        if name[0] in "PRWQ":
            u = th[o:o + k].astype(np.float32).view(np.uint32).astype(np.uint64)
            th[o:o + k] = (((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16).astype(np.uint32).view(np.float32)
        o += k
    yo = ofno.forward(th, x.astype(np.float64), **cfg)
    scale = np.max(np.abs(yo))
    assert np.max(np.abs(y_cc - yo)) < 1e-4 * scale          # the CUDA-core path, as in the other tests
    assert np.max(np.abs(y_tc - yo)) < 1e-2 * scale          # TF32 operands in two contractions per layer
    assert np.max(np.abs(y_tc - y_cc)) > 0                   # the tensor-core path really ran
    m.close()
