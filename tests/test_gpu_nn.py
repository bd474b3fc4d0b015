"""The learned initialiser's kernels (gbp_nn_*, tcgen05 BF16 GEMM + elementwise
kernels) against the FP64 reference network (oracle/nn_oracle.py).

Tolerances: the GEMM (both kernels: the 128 x 64 tile kernel and, for
shapes of at least 64 whole 128 x 256 tiles, the TMA-fed one) against an FP64 product of
the same BF16-rounded operands (FP32 accumulation: 1e-5 relative; at 8192^3-class
sizes against a PyTorch FP32 product of the same operands); the whole network (every GEMM
operand rounded to BF16, 2^-9 relative each, through six layers) against the
FP64 reference with FP32 weights: 3e-2 relative L2 for outputs and
gradients."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import nn_oracle as NO  # noqa: E402
from paper_2308_08410_gb300 import gbp  # noqa: E402
from paper_2308_08410_gb300.learned_init import ConvMLP, NetConfig  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = gbp.Context(0)
    yield c
    c.close()


def rel_l2(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def bf16_round(x):
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


# the last three are 64, 72 and 320 whole 128 x 256 tiles: the TMA-fed kernel
# (at 320 tiles some CTAs take three, so each of its two accumulators is reused)
@pytest.mark.parametrize("M,N,K", [(300, 100, 130), (128, 64, 64), (1, 43, 256), (1000, 320, 1216),
                                   (1024, 2048, 320), (1152, 2048, 1216), (4096, 2560, 128)])
def test_gemm_bf16(ctx, M, N, K):
    rng = np.random.default_rng(M + N + K)
    Kp = ((K + 63) // 64) * 64
    A = np.zeros((M, Kp), np.float32)
    B = np.zeros((N, Kp), np.float32)
    A[:, :K] = bf16_round(rng.standard_normal((M, K)))
    B[:, :K] = bf16_round(rng.standard_normal((N, K)))
    Ad = torch.from_numpy(A).cuda().to(torch.bfloat16)
    Bd = torch.from_numpy(B).cuda().to(torch.bfloat16)
    C0 = rng.standard_normal((M, N)).astype(np.float32)
    Cd = torch.from_numpy(C0).cuda()
    lib = ctx.lib
    st = lib.gbp_nn_gemm_bf16(ctx.h, M, N, Kp, C.c_void_p(Ad.data_ptr()), Kp, C.c_void_p(Bd.data_ptr()), Kp,
                              C.c_void_p(Cd.data_ptr()), N, 0.5, 2.0)
    assert st == 0
    ref = 0.5 * (A.astype(np.float64) @ B.astype(np.float64).T) + 2.0 * C0
    assert ctx.stats()["status"] == 0
    assert rel_l2(Cd.cpu().numpy(), ref) < 1e-5


def test_gemm_bf16_large_vs_fp32_matmul(ctx):
    """The TMA-fed kernel at the size its throughput is reported at (8192 x
    8192 x 4096: 2048 tiles, 13-14 per CTA) against a plain PyTorch FP32
    product of the same BF16 operands (no TF32): 1e-5 relative L2."""
    M = N = 8192
    K = 4096
    g = torch.Generator(device="cuda").manual_seed(7)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    C0 = torch.randn(M, N, device="cuda", generator=g)
    Cd = C0.clone()
    st = ctx.lib.gbp_nn_gemm_bf16(ctx.h, M, N, K, C.c_void_p(A.data_ptr()), K, C.c_void_p(B.data_ptr()), K,
                                  C.c_void_p(Cd.data_ptr()), N, 0.5, 2.0)
    assert st == 0 and ctx.stats()["status"] == 0
    tf32 = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        ref = 0.5 * (A.float() @ B.float().T) + 2.0 * C0
    finally:
        torch.backends.cuda.matmul.allow_tf32 = tf32
    err = float(torch.linalg.vector_norm(Cd - ref) / torch.linalg.vector_norm(ref))
    assert err < 1e-5, err


def test_network_forward_backward_vs_reference(ctx):
    cfg = NetConfig()
    ref = NO.Net(C_in=cfg.C_in, L_in=cfg.L_in, channels=cfg.channels, n_conv=cfg.n_conv, ksize=cfg.ksize,
                 stride=cfg.stride, pad=cfg.pad, hidden=cfg.hidden, n_out=cfg.n_out)
    params = ref.init(3)
    rng = np.random.default_rng(4)
    params = [(p + 0.05 * rng.standard_normal(p.shape)).astype(np.float32) for p in params]
    Bn = 6
    x = rng.standard_normal((Bn, cfg.L_in, cfg.C_in)).astype(np.float32)
    t = rng.standard_normal((Bn, cfg.n_out)).astype(np.float32)
    net = ConvMLP(ctx, cfg, params, max_batch=8)
    y = net.forward(torch.from_numpy(x).cuda(), Bn).cpu().numpy()
    yr, cache = ref.forward(params, x)
    assert rel_l2(y, yr) < 3e-2, rel_l2(y, yr)
    loss = net.mse(torch.from_numpy(t).cuda(), Bn)
    lr, dy = NO.mse(yr, t)
    assert abs(loss.item() - lr) < 3e-2 * lr
    net.backward(net.dy[:Bn], Bn)
    gr = ref.backward(params, cache, dy)
    gg = net.grads_numpy()
    for i, (a, b) in enumerate(zip(gg, gr)):
        assert rel_l2(a, b) < 3e-2, (i, rel_l2(a, b))


def test_training_reduces_loss(ctx):
    """A few hundred Adam steps on a small regression task with the
    project's kernels only."""
    cfg = NetConfig(C_in=4, L_in=64, channels=32, n_conv=2, hidden=64, n_out=5)
    ref = NO.Net(C_in=cfg.C_in, L_in=cfg.L_in, channels=cfg.channels, n_conv=cfg.n_conv, hidden=cfg.hidden,
                 n_out=cfg.n_out)
    rng = np.random.default_rng(7)
    Bn = 64
    x = rng.standard_normal((Bn, cfg.L_in, cfg.C_in)).astype(np.float32)
    t = np.tanh(x[:, ::13, 0][:, :cfg.n_out]).astype(np.float32)
    net = ConvMLP(ctx, cfg, ref.init(8), max_batch=Bn)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    losses = []
    for _ in range(300):
        net.forward(xd, Bn)
        losses.append(net.mse(td, Bn).item())
        net.backward(net.dy[:Bn], Bn)
        net.adam_step(lr=3e-3)
    assert losses[-1] < 0.2 * losses[0], (losses[0], losses[-1])
