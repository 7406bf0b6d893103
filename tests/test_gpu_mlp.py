"""GPU parity of the BF16 tensor-core GEMM and MLPs against the FP64 oracle.

Tolerances: the GEMM's inputs are bf16 and its accumulation fp32, so against
an FP64 product of the same bf16 values the error is a few fp32 roundings of
the K-term sum: |d| <= 1e-5 * sum_k |a_k b_k| + 1e-6.  A bf16 output adds one
bf16 rounding (relative 2^-8).  An MLP rounds every layer's activations to
bf16, so against the FP64 oracle (no intermediate rounding, same bf16
weights) the outputs agree to ~1e-2 relative per layer; gradients computed
from bf16 activations and bf16 dZ agree to ~3e-2 relative (norm-wise) and,
element by element, to 5e-2 of the element plus 5e-2 of the tensor's RMS
(the floor covers elements that are sums of cancelling terms, whose bf16
rounding noise scales with the RMS; a wrong, swapped or dropped element is
off by about the RMS itself).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlp as MO
from paper_2605_08528_b300 import sf

pytestmark = pytest.mark.gpu


def bf16(shape, rng, scale=1.0):
    t = torch.as_tensor(rng.normal(0, scale, shape), dtype=torch.float32).to(torch.bfloat16)
    return t.cuda().contiguous(), t.float().numpy().astype(np.float64)


# the last two shapes give every persistent CTA several tiles (both TMEM accumulators reused)
@pytest.mark.parametrize("M,N,K,tile", [(128, 64, 64, 64), (300, 200, 136, 128), (1000, 512, 320, 256),
                                        (77, 3, 512, 64), (4096, 256, 64, 256), (129, 130, 8, 128),
                                        (20000, 512, 320, 256), (40001, 96, 136, 64)])
@pytest.mark.parametrize("act", [sf.ACT_NONE, sf.ACT_ELU, sf.ACT_SILU, sf.ACT_TANH])
def test_gemm_against_fp64(M, N, K, tile, act):
    rng = np.random.default_rng(M * 7 + N + K + act)
    a, an = bf16((M, K), rng)
    b, bn = bf16((N, K), rng, 1 / np.sqrt(K))
    bias = torch.as_tensor(rng.normal(0, 0.1, N), dtype=torch.float32).cuda()
    out = torch.full((M, N), float("nan"), device="cuda")
    outb = torch.zeros((M, N), dtype=torch.bfloat16, device="cuda")
    outt = torch.zeros((N, M), dtype=torch.bfloat16, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    sf.sf_gemm_bf16(a, b, bias, M, N, K, act, out, outb, outt, tile_n=tile, d_err=err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    z = an @ bn.T + bias.cpu().numpy().astype(np.float64)
    ref = MO.act(z, act)
    bound = 1e-5 * (np.abs(an) @ np.abs(bn).T) + 1e-6
    if act != sf.ACT_NONE:   # exp via the hardware intrinsic: ~2 ulp-scale absolute error
        bound = bound * 2 + 4e-6 * np.maximum(1.0, np.abs(ref))
    got = out.cpu().numpy()
    assert np.isfinite(got).all()
    assert (np.abs(got - ref) <= bound).all(), float(np.abs(got - ref).max())
    gb = outb.float().cpu().numpy()
    assert (np.abs(gb - ref) <= np.abs(ref) * 2.0 ** -8 + bound).all()
    assert np.array_equal(outt.float().cpu().numpy(), gb.T)


def make_mlp(dims, hidden, out, rng):
    m = sf.sf_mlp_create(dims, hidden, out)
    params = []
    for l, (i, o) in enumerate(zip(dims[:-1], dims[1:])):
        W = rng.normal(0, 1 / np.sqrt(i), (o, i)).astype(np.float32)
        b = rng.normal(0, 0.05, o).astype(np.float32)
        sf.sf_mlp_set_layer(m, l, W, b)
        Wb = torch.as_tensor(W).to(torch.bfloat16).float().numpy().astype(np.float64)
        params.append((Wb, b.astype(np.float64)))
    return m, params


# outputs of at most 4 run as the fused head of the layer before; at 20,000 rows every
# persistent CTA computes two or more row blocks (both head-partial buffers reused)
@pytest.mark.parametrize("dims,hidden,out,batch", [([320, 512, 512, 3], sf.ACT_ELU, sf.ACT_TANH, 1000),
                                                   ([320, 512, 512, 3], sf.ACT_ELU, sf.ACT_TANH, 20000),
                                                   ([320, 512, 512, 1], sf.ACT_ELU, sf.ACT_NONE, 777),
                                                   ([30, 256, 256, 256, 16], sf.ACT_SILU, sf.ACT_NONE, 4096)])
def test_mlp_forward_against_fp64(dims, hidden, out, batch):
    rng = np.random.default_rng(len(dims) + batch)
    m, params = make_mlp(dims, hidden, out, rng)
    x = rng.normal(0, 1, (batch, dims[0])).astype(np.float32)
    xd = torch.as_tensor(x).cuda()
    y = torch.zeros((batch, dims[-1]), device="cuda")
    sf.sf_mlp_forward(m, xd, batch, y)
    sf.sf_mlp_sync(m)
    xb = torch.as_tensor(x).to(torch.bfloat16).float().numpy().astype(np.float64)
    ref = MO.forward(params, xb, hidden, out)
    got = y.cpu().numpy()
    scale = max(1.0, float(np.abs(ref).max()))
    err = np.abs(got - ref).max() / scale
    print("MLP forward max error (relative to output scale):", err)
    assert err < 2e-2 * (len(dims) - 1)
    sf.sf_mlp_destroy(m)


@pytest.mark.parametrize("dims,hidden,out,batch", [([30, 256, 256, 256, 16], sf.ACT_SILU, sf.ACT_NONE, 1024),
                                                   ([320, 512, 512, 3], sf.ACT_ELU, sf.ACT_TANH, 1736),
                                                   ([30, 64, 5], sf.ACT_ELU, sf.ACT_NONE, 200)])
def test_mlp_gradients_against_fp64(dims, hidden, out, batch):
    """Weight and bias gradients against the FP64 oracle: the bias sums run in
    batch // 256 row splits, at least one (four even ones; six with a short
    last one; one), over column groups wider than some layers (3, 5 outputs)."""
    rng = np.random.default_rng(3)
    m, params = make_mlp(dims, hidden, out, rng)
    x = rng.normal(0, 1, (batch, dims[0])).astype(np.float32)
    t = rng.normal(0, 1, (batch, dims[-1])).astype(np.float32)
    loss = sf.sf_mlp_train_step(m, torch.as_tensor(x).cuda(), torch.as_tensor(t).cuda(), batch, 0.0, update=False)
    xb = torch.as_tensor(x).to(torch.bfloat16).float().numpy().astype(np.float64)
    ref_loss = MO.mse(MO.forward(params, xb, hidden, out), t.astype(np.float64))
    assert abs(loss - ref_loss) <= 2e-2 * ref_loss
    grads = MO.backward(params, xb, t.astype(np.float64), hidden, out)
    for l, (gW, gb) in enumerate(grads):
        _, _, gw_gpu, gb_gpu = sf.sf_mlp_get_layer(m, l, dims[l + 1], dims[l])
        ew = np.linalg.norm(gw_gpu - gW) / np.linalg.norm(gW)
        eb = np.linalg.norm(gb_gpu - gb) / max(np.linalg.norm(gb), 1e-12)
        rw = np.abs(gw_gpu - gW) / (5e-2 * np.abs(gW) + 5e-2 * np.sqrt(np.mean(gW ** 2)))
        rb = np.abs(gb_gpu - gb) / (5e-2 * np.abs(gb) + 5e-2 * np.sqrt(np.mean(gb ** 2)) + 1e-30)
        print("layer", l, "relative gradient error W %.2e b %.2e; element-wise worst W %.2f b %.2f of the bound"
              % (ew, eb, rw.max(), rb.max()))
        assert ew < 3e-2 and eb < 3e-2
        assert rw.max() <= 1.0 and rb.max() <= 1.0, (l, float(rw.max()), float(rb.max()))
    sf.sf_mlp_destroy(m)


def test_mlp_training_fits_a_smooth_map():
    dims = [8, 64, 64, 4]
    rng = np.random.default_rng(5)
    m, _ = make_mlp(dims, sf.ACT_SILU, sf.ACT_NONE, rng)
    A = rng.normal(0, 0.5, (4, 8))
    batch = 512
    losses = []
    for it in range(300):
        x = rng.normal(0, 1, (batch, 8)).astype(np.float32)
        t = np.tanh(x @ A.T).astype(np.float32)
        losses.append(sf.sf_mlp_train_step(m, torch.as_tensor(x).cuda(), torch.as_tensor(t).cuda(), batch, 3e-3))
    sf.sf_mlp_sync(m)
    print("loss %.4f -> %.5f" % (losses[0], losses[-1]))
    assert losses[-1] < 0.1 * losses[0]
    sf.sf_mlp_destroy(m)
