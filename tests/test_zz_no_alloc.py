"""The allocation-free MLP forward (sf_mlp_forward_static) through the C-ABI.

Some callers cannot allocate device memory while they run: code inside a
CUDA graph whose memory was fixed at capture, a process whose device-memory
budget is already spent, or a host application that owns the allocator.  The
static variant keeps its scratch in a fixed array compiled into the library,
so it never calls cudaMalloc.  This file is named to be collected last.

Checks, on two calls in a row: the static result equals the allocating
forward's bit for bit (same GEMM kernels on the same inputs), and both agree
with the FP64 MLP oracle to the MLP forward tolerance; on a fresh handle the
first static call at a never-used batch leaves the device's free memory
unchanged; a batch-0 call primes the device without touching any buffer; a
batch beyond the fixed scratch is refused with a clear error.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlp as MO
from paper_2605_08528_b300 import sf

pytestmark = pytest.mark.gpu

DIMS = [320, 512, 512, 3]
# MLP forward against the FP64 oracle: ~1e-2 of the output scale per layer
TOL_PER_LAYER = 2e-2


def make(rng):
    m = sf.sf_mlp_create(DIMS, sf.ACT_ELU, sf.ACT_TANH)
    params = []
    for l, (i, o) in enumerate(zip(DIMS[:-1], DIMS[1:])):
        W = rng.normal(0, 1 / np.sqrt(i), (o, i)).astype(np.float32)
        b = rng.normal(0, 0.05, o).astype(np.float32)
        sf.sf_mlp_set_layer(m, l, W, b)
        params.append((torch.as_tensor(W).to(torch.bfloat16).float().numpy().astype(np.float64),
                       b.astype(np.float64)))
    return m, params


def test_static_forward_matches_allocating_forward_twice():
    rng = np.random.default_rng(17)
    m, params = make(rng)
    try:
        batch = 1000
        for call in range(2):       # the second call reuses (and must clear) the same scratch
            x = rng.normal(0, 1, (batch, DIMS[0])).astype(np.float32)
            xd = torch.as_tensor(x, device="cuda")
            y_ref = torch.full((batch, 3), float("nan"), device="cuda")
            y_static = torch.full((batch, 3), float("nan"), device="cuda")
            sf.sf_mlp_forward(m, xd, batch, y_ref)
            sf.sf_mlp_forward_static(m, xd, batch, y_static)
            sf.sf_mlp_sync(m)
            a, b = y_ref.cpu().numpy(), y_static.cpu().numpy()
            assert np.isfinite(b).all()
            assert np.array_equal(a.view(np.uint32), b.view(np.uint32)), call
            xb = torch.as_tensor(x).to(torch.bfloat16).float().numpy().astype(np.float64)
            ref = MO.forward(params, xb, MO.ELU, MO.TANH)
            err = np.abs(b - ref).max() / max(1.0, float(np.abs(ref).max()))
            print("static forward, call %d: max error vs FP64 %.2e of the output scale" % (call, err))
            assert err <= TOL_PER_LAYER * (len(DIMS) - 1), (call, err)
        # a batch beyond the fixed scratch is refused with a clear error
        big = sf.sf_mlp_static_scratch_bytes() // (2 * (320 + 512 + 512)) + 64
        xb = torch.zeros((big, DIMS[0]), device="cuda")
        yb = torch.zeros((big, 3), device="cuda")
        with pytest.raises(sf.SFError) as e:
            sf.sf_mlp_forward_static(m, xb, big, yb)
        assert e.value.status == sf.SF_ERR_INVALID_ARG and "scratch" in str(e.value)
    finally:
        sf.sf_mlp_destroy(m)


def test_static_forward_allocates_nothing_on_a_fresh_handle():
    """A fresh handle whose first call is the static forward, at a batch no
    call of that handle has used: the allocating forward would grow several
    MB of batch buffers there, so any hidden allocation would show in the
    device's free memory.  Kernels are loaded beforehand by a warm-up call on
    another handle (lazy module loading takes device memory once)."""
    rng = np.random.default_rng(23)
    warm, _ = make(rng)
    xw = torch.zeros((8, DIMS[0]), device="cuda")
    yw = torch.zeros((8, 3), device="cuda")
    sf.sf_mlp_forward_static(warm, xw, 0, yw)           # batch 0: the address lookup only
    sf.sf_mlp_forward_static(warm, xw, 8, yw)
    sf.sf_mlp_sync(warm)
    m, params = make(rng)
    try:
        batch = 1200
        x = rng.normal(0, 1, (batch, DIMS[0])).astype(np.float32)
        xd = torch.as_tensor(x, device="cuda")
        y = torch.full((batch, 3), float("nan"), device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        sf.sf_mlp_forward_static(m, xd, batch, y)
        sf.sf_mlp_sync(m)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert free1 == free0, (free0, free1)
        xb = torch.as_tensor(x).to(torch.bfloat16).float().numpy().astype(np.float64)
        ref = MO.forward(params, xb, MO.ELU, MO.TANH)
        got = y.cpu().numpy()
        assert np.abs(got - ref).max() / max(1.0, float(np.abs(ref).max())) <= TOL_PER_LAYER * (len(DIMS) - 1)
    finally:
        sf.sf_mlp_destroy(m)
        sf.sf_mlp_destroy(warm)
