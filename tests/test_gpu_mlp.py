"""The tensor-core GEMM and the warm-start network against the FP64 oracle.

GEMM: bf16 operands, fp32 accumulation; bound |C - AB^T| <= 2e-5 (|A||B|^T)
elementwise (fp32 summation of exact bf16 products).  Network: the oracle
rounds to bf16 at the same points, so outputs differ only through fp32
accumulation order and the bf16 roundings it flips: |dy| <= 2e-3 (outputs span
[0.1, 0.6]); gradients within 2e-2 relative L2 per layer.
"""
import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from paper_2507_04192_gb300 import mpm

pytestmark = pytest.mark.gpu

WIDTHS = [640, 256, 256, 32]


def _gemm(M, N, K, lda=None, ldb=None, ldc=None, seed=0):
    lda, ldb, ldc = lda or K, ldb or K, ldc or N
    g = torch.Generator().manual_seed(seed)
    A = torch.randn(M, lda, generator=g).to(torch.bfloat16)
    B = torch.randn(N, ldb, generator=g).to(torch.bfloat16)
    dA, dB = A.cuda(), B.cuda()
    dC = torch.full((M, ldc), float("nan"), device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    mpm.mpm_gemm_bf16(M, N, K, dA.data_ptr(), lda, dB.data_ptr(), ldb, dC.data_ptr(), ldc, st.data_ptr(), stream)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    a = A[:, :K].double().numpy()
    b = B[:, :K].double().numpy()
    return dC.cpu().double().numpy(), a @ b.T, np.abs(a) @ np.abs(b).T


@pytest.mark.parametrize("M,N,K", [(256, 256, 640), (256, 256, 256), (256, 32, 256), (32, 256, 256),
                                   (256, 640, 256), (130, 40, 72), (1, 8, 8), (300, 136, 1000),
                                   # 128 x 256 tiles (enough of them to fill every SM), full and ragged
                                   (4864, 1024, 256), (5000, 1000, 200)])
def test_gemm_bf16_matches_fp64_product(M, N, K):
    C, ref, mag = _gemm(M, N, K)
    assert np.isfinite(C[:, :N]).all()
    assert (np.abs(C[:, :N] - ref) <= 2e-5 * mag + 1e-30).all()


def test_gemm_strided_operands_and_untouched_padding():
    M, N, K = 144, 48, 96
    C, ref, mag = _gemm(M, N, K, lda=112, ldb=104, ldc=56, seed=1)
    assert (np.abs(C[:, :N] - ref) <= 2e-5 * mag).all()
    assert np.isnan(C[:, N:]).all()          # columns past N are not written


def test_gemm_argument_errors():
    x = torch.zeros(64, dtype=torch.bfloat16, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(mpm.MPMError):
        mpm.mpm_gemm_bf16(8, 8, 8, x.data_ptr(), 4, x.data_ptr(), 8, x.data_ptr(), 8, st.data_ptr())   # lda < K
    with pytest.raises(mpm.MPMError):
        mpm.mpm_gemm_bf16(8, 8, 8, x.data_ptr() + 2, 8, x.data_ptr(), 8, x.data_ptr(), 8, st.data_ptr())  # alignment


def _params(widths, seed):
    rng = np.random.default_rng(seed)
    out = []
    for l in range(len(widths) - 1):
        out.append((rng.standard_normal((widths[l + 1], widths[l])) / np.sqrt(widths[l]),
                    rng.standard_normal(widths[l + 1]) * 0.1))
    return omlp.pack(out).astype(np.float32)


def _data(batch, widths, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((batch, widths[0])).astype(np.float32),
            rng.uniform(0.1, 0.6, (batch, widths[-1])).astype(np.float32))


@pytest.mark.parametrize("batch", [256, 96])
def test_infer_matches_oracle(batch):
    p = _params(WIDTHS, 0)
    x, _ = _data(batch, WIDTHS, 1)
    net = mpm.MLP(WIDTHS, 256)
    net.set_params(p)
    y = net.infer(x)
    net.close()
    ref, _, _ = omlp.forward(p.astype(np.float64), WIDTHS, x.astype(np.float64))
    assert np.abs(y - ref).max() <= 2e-3
    assert np.abs(y - ref).mean() <= 2e-4


def test_gradient_matches_oracle():
    p = _params(WIDTHS, 2)
    x, t = _data(256, WIDTHS, 3)
    net = mpm.MLP(WIDTHS, 256)
    net.set_params(p)
    loss = net.train_step(x, t, lr=0.0, update=False)
    g = net.get_params(which=1).astype(np.float64)
    assert np.array_equal(net.get_params(0), p)          # no update
    net.close()
    ref_loss, ref_g = omlp.loss_and_grad(p.astype(np.float64), WIDTHS, x.astype(np.float64), t.astype(np.float64))
    assert loss == pytest.approx(ref_loss, rel=1e-2)
    o = 0
    for l in range(len(WIDTHS) - 1):
        for n in (WIDTHS[l + 1] * WIDTHS[l], WIDTHS[l + 1]):
            gs, rs = g[o:o + n], ref_g[o:o + n]
            assert np.linalg.norm(gs - rs) <= 2e-2 * np.linalg.norm(rs), (l, n)
            o += n


def test_adam_update_follows_its_definition():
    p = _params(WIDTHS, 4)
    x, t = _data(64, WIDTHS, 5)
    net = mpm.MLP(WIDTHS, 64)
    net.set_params(p)
    net.train_step(x, t, lr=1e-3, update=True)
    g = net.get_params(which=1).astype(np.float64)
    p1 = net.get_params(0).astype(np.float64)
    net.close()
    # first Adam step (bias-corrected): p - lr * g / (|g| + eps)
    ref = p - 1e-3 * g / (np.abs(g) + 1e-8)
    np.testing.assert_allclose(p1, ref, rtol=0, atol=2e-6)


def test_training_fits_a_teacher_network():
    teacher = _params(WIDTHS, 6)
    rng = np.random.default_rng(7)
    x = rng.standard_normal((1024, WIDTHS[0])).astype(np.float32)
    t = omlp.forward(teacher.astype(np.float64), WIDTHS, x.astype(np.float64), bf16_round=False)[0].astype(np.float32)
    net = mpm.MLP(WIDTHS, 256)
    net.set_params(_params(WIDTHS, 8))
    first = last = None
    for it in range(300):
        b = (it % 4) * 256
        loss = net.train_step(x[b:b + 256], t[b:b + 256], lr=1e-3)
        first = loss if first is None else first
        last = loss
    net.close()
    assert np.isfinite(last) and last < 0.2 * first


def test_network_argument_errors():
    with pytest.raises(mpm.MPMError):
        mpm.MLP([640, 250, 32], 256)                      # width not a multiple of 8
    net = mpm.MLP([16, 16, 8], 64)
    with pytest.raises(mpm.MPMError):
        net.train_step(np.zeros((12, 16)), np.zeros((12, 8)), 1e-3)      # batch not a multiple of 8
    with pytest.raises(mpm.MPMError):
        net.infer(np.zeros((72, 16)))                    # above max_batch
    net.close()


# ---- the coordinate network of Eq. nn_apprx (Sec. 5.2): 1 -> 30 -> 30 -> 30 -> 1 with ReLU,
# padded to multiples of 8 (8 -> 32 -> 32 -> 32 -> 8; the padding is inert), linear output

COORD = [8, 32, 32, 32, 8]


def _coord_params(seed):
    rng = np.random.default_rng(seed)
    w = [1, 30, 30, 30, 1]
    layers = []
    for l in range(4):
        W = np.zeros((COORD[l + 1], COORD[l]))
        W[:w[l + 1], :w[l]] = rng.standard_normal((w[l + 1], w[l])) * np.sqrt(2.0 / w[l])
        b = np.zeros(COORD[l + 1])
        b[:w[l + 1]] = rng.standard_normal(w[l + 1]) * 0.1
        layers.append((W, b))
    return omlp.pack(layers).astype(np.float32)


def _coords(batch, seed):
    rng = np.random.default_rng(seed)
    x = np.zeros((batch, 8), dtype=np.float32)
    x[:, 0] = rng.uniform(0.0, 1.0, batch)
    return x


def test_coordinate_network_matches_oracle():
    p = _coord_params(10)
    x = _coords(256, 11)
    net = mpm.MLP(COORD, 256, hidden=mpm.MPM_ACT_RELU, output=mpm.MPM_OUT_LINEAR)
    net.set_params(p)
    y = net.infer(x)
    rng = np.random.default_rng(12)
    dy = np.zeros((256, 8), dtype=np.float32)
    dy[:, 0] = rng.standard_normal(256)
    net.backward(x, dy, lr=0.0, update=False)
    g = net.get_params(which=1).astype(np.float64)
    net.close()
    kw = dict(hidden="relu", out="linear")
    ref, _, _ = omlp.forward(p.astype(np.float64), COORD, x.astype(np.float64), **kw)
    scale = np.abs(ref[:, 0]).max()
    assert np.abs(y[:, 0] - ref[:, 0]).max() <= 5e-3 * scale
    assert np.abs(y[:, 1:]).max() == 0.0                  # padded outputs: zero weights, zero bias
    ref_g = omlp.backward(p.astype(np.float64), COORD, x.astype(np.float64), dy.astype(np.float64), **kw)
    o = 0
    for l in range(len(COORD) - 1):
        for n in (COORD[l + 1] * COORD[l], COORD[l + 1]):
            gs, rs = g[o:o + n], ref_g[o:o + n]
            assert np.linalg.norm(gs - rs) <= 2e-2 * np.linalg.norm(rs) + 1e-12, (l, n)
            assert np.all(gs[rs == 0.0] == 0.0)            # inert padding stays exactly zero
            o += n


def test_async_train_step_equals_the_synchronous_one():
    torch = pytest.importorskip("torch")
    p = _params(WIDTHS, 13)
    x, t = _data(256, WIDTHS, 14)
    a, b = mpm.MLP(WIDTHS, 256), mpm.MLP(WIDTHS, 256)
    a.set_params(p)
    b.set_params(p)
    la = [a.train_step(x, t, lr=1e-3) for _ in range(3)]
    dx, dt = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()                   # the network runs on its own stream
    lb = []
    for _ in range(3):
        b.train_step_async(256, dx.data_ptr(), dt.data_ptr(), 1e-3, loss.data_ptr())
        torch.cuda.synchronize()
        lb.append(float(loss.item()))
    pa, pb = a.get_params(0), b.get_params(0)
    a.close()
    b.close()
    assert lb == pytest.approx(la, rel=1e-6)
    np.testing.assert_array_equal(pa, pb)
