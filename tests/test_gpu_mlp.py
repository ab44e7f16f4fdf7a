"""The scheduling MLP's hand-written GPU kernels against the float64 oracle.

fp32 mode: forward outputs and gradients within 1e-5 (relative to the
largest reference magnitude).  bf16 mode rounds weights, inputs and hidden
activations to bf16 (8 significant bits): the oracle is run on the same
bf16-rounded weights and inputs, and the remaining difference comes from the
two rounded hidden layers.  A rounding of a value v changes it by at most
2^-9 |v|; propagated through two layers of 64-term sums it stays below
1 % of the output scale, which the bf16 tolerance below uses with a 2x margin.
"""
import numpy as np
import pytest

from oracle import mlp as ref
from paper_2412_19420_gb300 import datagen

pytestmark = pytest.mark.gpu
fim = pytest.importorskip("paper_2412_19420_gb300.fim")
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    c = fim.fim_create(0)
    yield c
    fim.fim_destroy(c)


def _bf16(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float32).numpy()


def _data(B, seed):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(B, 8)).astype(np.float32)
    t = np.stack([rng.normal(4, 2, B), (rng.random(B) < 0.3)], 1).astype(np.float32)
    p = datagen.mlp_init_weights(seed)
    p += np.random.default_rng(seed + 1).normal(0, 0.05, p.shape).astype(np.float32)
    return p, x, t


def _gpu_fwd_bwd(ctx, p, x, t, bf16):
    B = x.shape[0]
    dp = torch.from_numpy(p).cuda()
    dx = torch.from_numpy(x).cuda()
    dt = torch.from_numpy(t).cuda()
    dy = torch.empty((B, 2), dtype=torch.float32, device="cuda")
    dc = torch.empty((B, 256), dtype=torch.float32, device="cuda")
    dg = torch.empty(fim.FIM_MLP_PARAMS, dtype=torch.float32, device="cuda")
    import ctypes
    loss = ctypes.c_float()
    torch.cuda.synchronize()
    fim._check(fim._lib.fim_mlp_forward(ctx, dp.data_ptr(), dx.data_ptr(), B, dy.data_ptr(), dc.data_ptr(),
                                        int(bf16)), "fwd")
    fim._check(fim._lib.fim_mlp_backward(ctx, dp.data_ptr(), dx.data_ptr(), dy.data_ptr(), dt.data_ptr(),
                                         dc.data_ptr(), B, dg.data_ptr(), ctypes.byref(loss), int(bf16)), "bwd")
    torch.cuda.synchronize()
    return dy.cpu().numpy(), dg.cpu().numpy(), loss.value


def _close(a, b, tol):
    scale = max(1e-30, float(np.max(np.abs(b))))
    return float(np.max(np.abs(a - b))) <= tol * scale


@pytest.mark.parametrize("B", [1, 37, 256, 4099])
def test_fp32_forward_backward_match_oracle(ctx, B):
    p, x, t = _data(B, B)
    y, g, loss = _gpu_fwd_bwd(ctx, p, x, t, bf16=False)
    ry, cache = ref.forward(p.astype(np.float64), x.astype(np.float64))
    rg = ref.backward(p.astype(np.float64), cache, ry, t.astype(np.float64))
    assert _close(y, ry, 1e-5)
    assert loss == pytest.approx(ref.loss(ry, t), rel=1e-5)
    # per parameter block, relative to that block's scale
    o = 0
    for s in ref.SHAPES:
        k = int(np.prod(s))
        assert _close(g[o:o + k], rg[o:o + k], 1e-5), s
        o += k


def test_bf16_forward_backward_within_bound(ctx):
    p, x, t = _data(512, 7)
    y, g, _ = _gpu_fwd_bwd(ctx, p, x, t, bf16=True)
    pb, xb = _bf16(p).astype(np.float64), _bf16(x).astype(np.float64)
    ry, cache = ref.forward(pb, xb)
    rg = ref.backward(pb, cache, ry, t.astype(np.float64))
    assert _close(y, ry, 2e-2)
    assert _close(g, rg, 2e-2)


def test_adam_matches_oracle(ctx):
    rng = np.random.default_rng(3)
    p = rng.normal(size=fim.FIM_MLP_PARAMS).astype(np.float32)
    g = rng.normal(size=fim.FIM_MLP_PARAMS).astype(np.float32)
    m = rng.normal(size=fim.FIM_MLP_PARAMS).astype(np.float32) * 0.1
    v = np.abs(rng.normal(size=fim.FIM_MLP_PARAMS)).astype(np.float32) * 0.1
    dp, dg, dm, dv = (torch.from_numpy(a.copy()).cuda() for a in (p, g, m, v))
    fim._check(fim._lib.fim_mlp_adam(ctx, dp.data_ptr(), dg.data_ptr(), dm.data_ptr(), dv.data_ptr(), 3,
                                     1e-3, 0.9, 0.999, 1e-8), "adam")
    torch.cuda.synchronize()
    # the kernel receives float32 hyper-parameters: give the oracle the same
    # values (1 - 0.999f differs from 0.001 by 1.3e-5 relative)
    f32 = lambda v: float(np.float32(v))  # noqa: E731
    b1, b2, lr, eps = f32(0.9), f32(0.999), f32(1e-3), f32(1e-8)
    rp, rm, rv = ref.adam_step(p.astype(np.float64), g.astype(np.float64), m.astype(np.float64),
                               v.astype(np.float64), 3, lr, b1, b2, eps)
    # each moment is a sum of two float32 products: its error is a few ulp of
    # the larger term, not of the (possibly cancelling) result
    tm = np.abs(b1 * m.astype(np.float64)) + np.abs((1 - b1) * g.astype(np.float64))
    tv = np.abs(b2 * v.astype(np.float64)) + np.abs((1 - b2) * g.astype(np.float64) ** 2)
    assert np.all(np.abs(dm.cpu().numpy() - rm) <= 4e-7 * tm)
    assert np.all(np.abs(dv.cpu().numpy() - rv) <= 4e-7 * tv)
    assert np.allclose(dp.cpu().numpy(), rp, rtol=1e-6, atol=1e-7)


def test_gpu_training_reduces_loss(ctx):
    from paper_2412_19420_gb300 import sched
    p, x, t = _data(2048, 11)
    w, hist = sched.train(ctx, x, t, steps=300, lr=3e-3, batch=512, seed=0, init=p)
    assert hist[-1] < 0.5 * hist[0]
