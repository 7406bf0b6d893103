"""The allocation-free MLP forward (sf_mlp_forward_static) against the
allocating one (sf_mlp_forward), through the C-ABI, on two calls in a row.

Some callers cannot allocate device memory while they run (inside fixed-memory
CUDA graphs, under a spent memory budget, or with an allocator owned by the
host application); the static variant keeps its scratch in a fixed array of
the library.  This file is named to be collected last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2605_08528_b300 import sf

pytestmark = pytest.mark.gpu

# the tolerance of the MLP forward tests, relative to the output scale, per layer
TOL_PER_LAYER = 2e-2


def test_static_forward_matches_allocating_forward_twice():
    dims = [320, 512, 512, 3]
    rng = np.random.default_rng(17)
    m = sf.sf_mlp_create(dims, sf.ACT_ELU, sf.ACT_TANH)
    try:
        for l, (i, o) in enumerate(zip(dims[:-1], dims[1:])):
            sf.sf_mlp_set_layer(m, l, rng.normal(0, 1 / np.sqrt(i), (o, i)), rng.normal(0, 0.05, o))
        batch = 1000
        for call in range(2):       # the second call reuses (and must clear) the same scratch
            x = torch.as_tensor(rng.normal(0, 1, (batch, dims[0])), dtype=torch.float32, device="cuda")
            y_ref = torch.full((batch, 3), float("nan"), device="cuda")
            y_static = torch.full((batch, 3), float("nan"), device="cuda")
            sf.sf_mlp_forward(m, x, batch, y_ref)
            sf.sf_mlp_forward_static(m, x, batch, y_static)
            sf.sf_mlp_sync(m)
            a, b = y_ref.cpu().numpy(), y_static.cpu().numpy()
            assert np.isfinite(b).all()
            scale = max(1.0, float(np.abs(a).max()))
            assert np.abs(a - b).max() / scale <= TOL_PER_LAYER * (len(dims) - 1), (call, float(np.abs(a - b).max()))
        # a batch beyond the fixed scratch is refused with a clear error
        big = sf.sf_mlp_static_scratch_bytes() // (2 * (320 + 512 + 512)) + 64
        xb = torch.zeros((big, dims[0]), device="cuda")
        yb = torch.zeros((big, 3), device="cuda")
        with pytest.raises(sf.SFError) as e:
            sf.sf_mlp_forward_static(m, xb, big, yb)
        assert e.value.status == sf.SF_ERR_INVALID_ARG and "scratch" in str(e.value)
    finally:
        sf.sf_mlp_destroy(m)
