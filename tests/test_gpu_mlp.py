"""The tcgen05 tensor-core GEMM and the surrogate MLP against references.

GEMM: BF16 products are exact in FP32, so C = A B^T must match an FP32
computation from the same BF16 inputs up to summation order (1e-4 of the
largest entry).  MLP: the network keeps activations in BF16 (relative
rounding 2^-9 per stored value, compounding over three layers and the
backward pass), so its loss and gradient are compared with the FP64 reference
evaluated on the same BF16-rounded weights and inputs at 3e-2, normwise."""
import numpy as np
import pytest

from oracle import mlp as ref
from paper_1911_10274_gb300 import titan as T

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


# the last two shapes have at least two waves of 256-wide tiles: the wide-tile kernel
# tile widths: 64 (up to one wave of 128-wide tiles), 128 (between), 256
# (two waves of 256-wide tiles or more)
@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 384, 512), (512, 512, 4096), (4096, 512, 1024),
                                   (4096, 768, 256), (4096, 2560, 256), (2048, 5120, 192)])
def test_tcgen05_gemm_matches_reference(M, N, K):
    g = torch.Generator(device="cuda").manual_seed(M + N + K)
    A = torch.randn(M, K, device="cuda", generator=g).bfloat16()
    B = torch.randn(N, K, device="cuda", generator=g).bfloat16()
    C = torch.full((M, N), float("nan"), device="cuda")
    T.titan_gemm_bf16_tn(A, B, C)
    ref_c = A.double() @ B.double().T
    err = (C.double() - ref_c).abs().max().item()
    assert err <= 1e-4 * ref_c.abs().max().item(), err
    torch.cuda.synchronize()
    T.titan_gemm_check()


def test_gemm_calls_enqueue_without_waiting_and_follow_stream_order():
    """Eight products enqueued back to back on a side stream, each output
    then consumed on that stream: stream order alone orders them."""
    g = torch.Generator(device="cuda").manual_seed(9)
    s = torch.cuda.Stream()
    As = [torch.randn(256, 512, device="cuda", generator=g).bfloat16() for _ in range(8)]
    B = torch.randn(384, 512, device="cuda", generator=g).bfloat16()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        Cs = [torch.empty(256, 384, device="cuda") for _ in range(8)]
        for A, C in zip(As, Cs):
            T.titan_gemm_bf16_tn(A, B, C)                # torch's current stream: s
        tot = sum(C.double() for C in Cs)
    s.synchronize()
    T.titan_gemm_check()
    ref = sum(A.double() @ B.double().T for A in As)
    assert (tot - ref).abs().max().item() <= 1e-4 * ref.abs().max().item()


def test_gemm_rejects_unaligned_shapes():
    A = torch.zeros(100, 64, device="cuda").bfloat16()
    B = torch.zeros(128, 64, device="cuda").bfloat16()
    C = torch.zeros(100, 128, device="cuda")
    with pytest.raises(T.TitanError) as ei:
        T.titan_gemm_bf16_tn(A, B, C)
    assert ei.value.status == T.TITAN_E_INVALID


def _bf16_round(a):
    return torch.as_tensor(a, dtype=torch.float32).bfloat16().float().numpy().astype(np.float64)


# B = 4096 cuts the weight-gradient products into 4 (first layer) and 8 (hidden
# layers) K slices; B = 512 into 2; B = 128 not at all
@pytest.mark.parametrize("n_in,hidden,B", [(128, 128, 128), (1024, 512, 512), (1024, 512, 4096)])
def test_mlp_forward_and_gradient_match_fp64_reference(n_in, hidden, B):
    net = T.MLP(n_in, hidden, seed=3)
    rng = np.random.default_rng(1)
    x = torch.as_tensor(rng.normal(0, 1, (B, n_in)), dtype=torch.float32).bfloat16().cuda()
    t = torch.as_tensor(rng.normal(0, 0.3, B), dtype=torch.float32).cuda()
    p = net.get_params().astype(np.float64)
    # the network multiplies BF16 copies of its weights: the reference uses the same values
    pr = p.copy()
    Wo = net.unpack(np.arange(net.n_params))
    for idx in (Wo[0], Wo[2], Wo[4]):
        pr[idx.ravel()] = _bf16_round(p[idx.ravel()])
    xr = x.float().cpu().numpy().astype(np.float64)
    y = torch.empty(B, device="cuda")
    net.forward(x, y)
    y_ref, _, _ = ref.forward(pr, xr, n_in, hidden)
    yr = y.cpu().numpy()
    assert np.abs(yr - y_ref).max() <= 3e-2 * np.abs(y_ref).max()
    loss = torch.empty(1, device="cuda")
    grad = torch.empty(net.n_params, device="cuda")
    net.gradient(x, t, loss, grad)
    l_ref, g_ref = ref.loss_and_grad(pr, xr, t.cpu().numpy().astype(np.float64), n_in, hidden)
    assert float(loss) == pytest.approx(l_ref, rel=3e-2)
    g = grad.cpu().numpy().astype(np.float64)
    slices = net.unpack(np.arange(net.n_params))
    for sl in slices[:-1]:
        gs, rs = g[sl.ravel()], g_ref[sl.ravel()]
        assert np.linalg.norm(gs - rs) <= 3e-2 * np.linalg.norm(rs) + 1e-12
    # db4 = 2 mean(y - t) nearly cancels: its error is measured against its summands
    tt = t.cpu().numpy().astype(np.float64)
    scale = 2.0 / B * np.abs(y_ref - tt).sum()
    assert abs(g[slices[-1][0]] - g_ref[slices[-1][0]]) <= 3e-2 * scale


def test_mlp_training_reduces_the_loss_on_a_learnable_target():
    net = T.MLP(128, 128, seed=0)
    rng = np.random.default_rng(5)
    B = 512
    X = rng.normal(0, 1, (B, 128))
    t = np.tanh(X[:, :8].sum(axis=1) / 3.0)
    x = torch.as_tensor(X, dtype=torch.float32).bfloat16().cuda()
    tt = torch.as_tensor(t, dtype=torch.float32).cuda()
    loss = torch.empty(1, device="cuda")
    net.gradient(x, tt, loss, None)
    first = float(loss)
    for _ in range(300):
        net.train_step(x, tt, 1e-3, loss)
    net.sync()
    assert float(loss) < 0.2 * first


def test_train_step_is_adam_on_the_gradient_with_the_device_step_count():
    """Three training steps (the first two at one learning rate, the third at
    another) against Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected)
    written out in FP64 on the gradients the network reports at each step's
    parameters: checks the step counter and learning rate the captured step
    reads from device memory."""
    n_in, hidden, B = 256, 128, 1024
    net = T.MLP(n_in, hidden, seed=11)
    rng = np.random.default_rng(2)
    x = torch.as_tensor(rng.normal(0, 1, (B, n_in)), dtype=torch.float32).bfloat16().cuda()
    t = torch.as_tensor(rng.normal(0, 0.3, B), dtype=torch.float32).cuda()
    b1, b2, eps = 0.9, 0.999, 1e-8
    m = np.zeros(net.n_params)
    v = np.zeros(net.n_params)
    loss = torch.empty(1, device="cuda")
    grad = torch.empty(net.n_params, device="cuda")
    for step, lr in enumerate([1e-3, 1e-3, 3e-4], start=1):
        p0 = net.get_params().astype(np.float64)
        net.gradient(x, t, loss, grad)
        g = grad.cpu().numpy().astype(np.float64)
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        want = p0 - lr * (m / (1 - b1 ** step)) / (np.sqrt(v / (1 - b2 ** step)) + eps)
        net.train_step(x, t, lr, loss)
        net.sync()
        got = net.get_params().astype(np.float64)
        # FP32 arithmetic of a step of size <= lr (a few ulp of lr), plus
        # entries whose gradient is near zero, where eps decides the step
        err = np.abs(got - want)
        assert np.median(err) <= 1e-3 * lr
        assert np.quantile(err, 0.999) <= 2e-2 * lr + 1e-6 * np.abs(p0).max()
